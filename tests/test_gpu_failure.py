"""Failure detection on the GPU without a fault: a bounded wait that runs out.

With CHW_FLAG_TEST_STALL one CTA of each cluster withholds its first "full" signal and
the kernel's waits give up after a few thousand polls.  The other CTAs' waits run out,
record CHW_ERR_TIMEOUT in the plan's status word and finish; the host reads the status,
and the context stays usable (a normal plan right after gives bit-exact results).
"""

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


@pytest.mark.parametrize("m", [15, 16])
def test_cluster_wait_timeout_is_reported_and_the_context_survives(chw, m):
    import torch

    x = W.normal_f32(m, 8, seed=900 + m)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    p = chw.chw_plan(m, 8, "f32", "end", chw.CHW_FLAG_TEST_STALL)
    assert chw.chw_plan_get_info(p).tier == 2
    chw.chw_forward(p, xd, yd)
    assert chw.chw_last_device_status(p) == chw._lib.CHW_ERR_TIMEOUT
    assert chw.chw_last_device_status(p) == 0  # reading the status clears the latch
    q = chw.chw_plan(m, 8, "f32", "end")
    chw.chw_forward(q, xd, yd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(q) == 0
    assert_bitwise(yd.cpu().numpy(), O.chw_cascade(x, m, np.float32, "end"), "after a timeout")
