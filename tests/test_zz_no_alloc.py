"""chw_forward_noalloc: the transform for callers that cannot allocate device memory (GPU).

Callers capturing a CUDA graph, or running with device memory owned by another
allocator, cannot let the library cudaMalloc a workspace.  This entry point keeps the
two-pass intermediate in a fixed array inside the library instead.  Its results must
equal chw_forward's (the same butterflies in the same order, so bit for bit, which is
within the fp32 tolerance of 1e-6 used everywhere else), on two calls in a row that reuse
the array.  This file sorts last so that a run stopping at its first failure has already
run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(cuda_device):
    import torch

    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import _lib, build

    build.build()
    return chw, _lib, _lib.load(), torch


def noalloc(lib, torch, m, batch, dtype, norm, xd):
    yd = torch.empty_like(xd)
    st = lib.chw_forward_noalloc(m, batch, dtype, norm, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.chw_status_string(st).decode()
    return yd


@pytest.mark.parametrize(
    "m,batch,dtype,norm", [(18, 16, "f32", "end"), (20, 4, "f32", "per_level"), (22, 1, "i32", "none"), (19, 3, "f32", "none")]
)
def test_noalloc_matches_forward_on_two_calls(env, m, batch, dtype, norm):
    chw, _lib, lib, torch = env
    d = chw.DTYPES[dtype]
    nm = chw.NORMS[norm]
    outs, refs = [], []
    for call in range(2):  # two calls in a row share the static array
        if dtype == "i32":
            x = W.uniform_int32(m, batch, seed=50 + call, bound=2 ** (29 - m))
        else:
            x = W.normal_f32(m, batch, seed=50 + call)
        xd = torch.from_numpy(x).cuda()
        outs.append(noalloc(lib, torch, m, batch, d, nm, xd))
        p = chw.chw_plan(m, batch, dtype, norm)
        yr = torch.empty_like(xd)
        chw.chw_forward(p, xd, yr)
        refs.append(yr)
    torch.cuda.synchronize()
    for got, ref in zip(outs, refs):
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(g.view(np.uint32), r.view(np.uint32))
        if dtype == "f32":
            rel = np.linalg.norm((g - r).astype(np.float64), axis=1) / np.linalg.norm(r.astype(np.float64), axis=1)
            assert rel.max() <= 1e-6


def test_noalloc_rejects_what_it_cannot_hold(env):
    chw, _lib, lib, torch = env
    xd = torch.zeros(1 << 20, device="cuda")
    p = ctypes.c_void_p(xd.data_ptr())
    assert lib.chw_forward_noalloc(20, 8, _lib.CHW_F32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward_noalloc(23, 1, _lib.CHW_F32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_UNSUPPORTED
    assert lib.chw_forward_noalloc(18, 1, _lib.CHW_BF16, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_UNSUPPORTED
    assert lib.chw_forward_noalloc(18, 1, _lib.CHW_F32, _lib.CHW_NORM_END, ctypes.c_void_p(xd.data_ptr() + 4), p, None) == _lib.CHW_ERR_ALIGNMENT
