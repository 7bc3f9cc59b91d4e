"""Natural and sequency output orders on the GPU, every tier, against the oracle bit for bit.

The ordered outputs are the dyadic cascade's values stored elsewhere, so the oracle is
the cascade of Theorem 1 permuted (oracle.wht_ordered, pinned to the Sylvester matrix and
to the sign-change definition of sequency order).
"""

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORACLE_DT = {"f32": np.float32, "i32": np.int32}
TIER = {"simple": 0, "fused": 1, "cluster": 2, "two-pass": 3, "tensor-memory": 7}


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


def _x(m, batch, dtype, seed):
    if dtype == "i32":
        return W.uniform_int32(m, batch, seed, bound=1 << max(1, 29 - m))
    return W.normal_f32(m, batch, seed)


def _run(chw, x, m, order, dtype, norm, flags=0, adjoint=False, diag=None, inplace=False):
    import torch

    p = chw.chw_plan(m, x.shape[0], dtype, norm, flags, order=order)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = xd if inplace else torch.empty_like(xd)
    dd = None if diag is None else torch.from_numpy(diag).cuda()
    (chw.chw_adjoint if adjoint else chw.chw_forward)(p, xd, yd, diag=dd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    info = chw.chw_plan_get_info(p)
    return yd.cpu().numpy(), info


def _expected_tier(m, batch, order):
    if m < 5 and (batch << m) % 32:
        return TIER["simple"]
    if m <= 14:
        return TIER["fused"]
    if m <= 16:
        return TIER["tensor-memory"]
    if order == "natural" or m >= 18:
        return TIER["two-pass"]
    return TIER["cluster"]


CASES = [(m, b) for m in range(0, 18) for b in (1, 5)] + [(12, 64), (18, 2), (20, 3), (23, 1), (24, 1)]
MODES = [("f32", "end"), ("f32", "per_level"), ("i32", "none")]


@pytest.mark.parametrize("order", ["natural", "sequency"])
@pytest.mark.parametrize("m,batch", CASES)
@pytest.mark.parametrize("dtype,norm", MODES)
def test_ordered_forward_bitwise(chw, order, m, batch, dtype, norm):
    if order == "natural" and m > 23:
        pytest.skip("natural order takes m <= 23")
    x = _x(m, batch, dtype, 6000 + m)
    y, info = _run(chw, x, m, order, dtype, norm)
    assert info.order == (1 if order == "natural" else 2)
    assert info.tier == _expected_tier(m, batch, order), (info.tier, m, batch, order)
    assert_bitwise(y, O.wht_ordered(x, m, order, ORACLE_DT[dtype], norm), f"{order} m={m} b={batch} {dtype} {norm}")


@pytest.mark.parametrize("order", ["natural", "sequency"])
@pytest.mark.parametrize("m", [15, 16])
@pytest.mark.parametrize("dtype,norm", MODES)
def test_ordered_tensor_memory_many_signals(chw, order, m, dtype, norm):
    # more signals than SMs: CTAs walk several signals with alternating tensor-memory layouts
    x = _x(m, 157, dtype, 6600 + m)
    y, info = _run(chw, x, m, order, dtype, norm)
    assert info.tier == TIER["tensor-memory"]
    rows = [0, 1, 2, 77, 155, 156]
    assert_bitwise(y[rows], O.wht_ordered(x[rows], m, order, ORACLE_DT[dtype], norm), f"{order} m={m} {dtype}")


@pytest.mark.parametrize("m", [15, 16])
def test_sequency_cluster_tier_on_request(chw, m):
    x = _x(m, 3, "f32", 6700 + m)
    y, info = _run(chw, x, m, "sequency", "f32", "end", flags=chw.CHW_FLAG_CLUSTER)
    assert info.tier == TIER["cluster"]
    assert_bitwise(y, O.wht_ordered(x, m, "sequency", np.float32, "end"), f"cluster sequency m={m}")


@pytest.mark.parametrize("order", ["natural", "sequency"])
@pytest.mark.parametrize("m", [0, 1, 3, 7, 11, 13])
def test_ordered_simple_kernel(chw, order, m):
    x = _x(m, 6, "f32", 6100 + m)
    y, info = _run(chw, x, m, order, "f32", "end", flags=chw.CHW_FLAG_FORCE_SIMPLE)
    assert info.tier == 0
    assert_bitwise(y, O.wht_ordered(x, m, order, np.float32, "end"), f"simple {order} m={m}")


@pytest.mark.parametrize("order", ["natural", "sequency"])
@pytest.mark.parametrize("m", [11, 14])
def test_ordered_forced_two_pass(chw, order, m):
    x = _x(m, 8, "f32", 6200 + m)
    y, info = _run(chw, x, m, order, "f32", "per_level", flags=chw.CHW_FLAG_FORCE_MULTIPASS)
    assert info.tier == TIER["two-pass"]
    assert_bitwise(y, O.wht_ordered(x, m, order, np.float32, "per_level"), f"forced two-pass {order} m={m}")


@pytest.mark.parametrize("order", ["natural", "sequency"])
@pytest.mark.parametrize("m,batch", [(4, 3), (10, 16), (14, 4), (15, 5), (16, 3), (19, 2)])
def test_ordered_diag_adjoint_inplace(chw, order, m, batch):
    x = _x(m, batch, "f32", 6300 + m)
    d = W.diag_pm1(m, 6400 + m)
    perm = O.order_permutation(m, order)
    ref = O.wht_ordered(x, m, order, np.float32, "end")
    # forward with D on the stored (ordered) outputs
    y, _ = _run(chw, x, m, order, "f32", "end", diag=d)
    assert_bitwise(y, np.where(d < 0, -ref, ref).astype(np.float32), f"D H {order}")
    # adjoint: the ordered matrices are symmetric, so H^T D y is the ordered forward of D y
    xa, _ = _run(chw, x, m, order, "f32", "end", adjoint=True, diag=d)
    dx = np.where(d < 0, -x, x).astype(np.float32)
    assert_bitwise(xa, O.wht_ordered(dx, m, order, np.float32, "end"), f"H^T D {order}")
    # in place
    yi, _ = _run(chw, x, m, order, "f32", "end", inplace=True)
    assert_bitwise(yi, ref, f"in-place {order}")
    assert perm.shape == (1 << m,)


@pytest.mark.parametrize("order", ["natural", "sequency"])
@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("m", [3, 11, 12])
def test_ordered_16bit_is_permuted_dyadic(chw, order, fmt, m):
    import torch

    tdt = torch.bfloat16 if fmt == "bf16" else torch.float16
    x64 = W.heavy_tailed_f64(m, 8, 6500 + m)
    codes, e_in = W.quantise_pow2(x64, fmt)
    outs = {}
    for o in ("dyadic", order):
        p = chw.chw_plan(m, 8, fmt, "end", order=o)
        xd = torch.from_numpy(codes.view(np.int16)).cuda().view(tdt)
        yd = torch.empty_like(xd)
        ei = torch.from_numpy(e_in).cuda()
        eo = torch.empty_like(ei)
        chw.chw_forward(p, xd, yd, ei, eo)
        torch.cuda.synchronize()
        outs[o] = (yd.view(torch.int16).cpu().numpy().view(np.uint16), eo.cpu().numpy())
    perm = O.order_permutation(m, order)
    assert np.array_equal(outs[order][1], outs["dyadic"][1])
    assert np.array_equal(outs[order][0], outs["dyadic"][0][:, perm])


def test_order_argument_errors(chw):
    with pytest.raises(chw.ChwError, match="m <= 23"):
        chw.chw_plan(24, 1, "f32", "end", order="natural")
    with pytest.raises(chw.ChwError, match="ROWSTACK"):
        chw.chw_plan(16, 2, "f32", "end", chw.CHW_FLAG_ROWSTACK, order="sequency")
    with pytest.raises(chw.ChwError, match="exclude"):
        chw.chw_plan(8, 2, "f32", "end", chw.CHW_FLAG_ORDER_NATURAL | chw.CHW_FLAG_ORDER_SEQUENCY)
