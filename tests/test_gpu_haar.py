"""Haar transform (eq. (2)), its transpose, and the Haar-Walsh transform (eq. (4)) on the GPU.

Every case compares the CUDA path, called through the C ABI, with the CPU oracle on the
same seeded inputs, element by element: bit for bit wherever both sides take the same
operations (all modes here), and the round trips within fp32 tolerance.
"""

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORACLE_DT = {"f32": np.float32, "i32": np.int32}


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


def _inputs(m, batch, dtype, seed):
    if dtype == "i32":
        # |x| <= 2^(28-m) keeps every unnormalised coefficient (up to 2^m |x|) in int32
        return W.uniform_int32(m, batch, seed, bound=1 << max(1, 28 - m))
    return W.normal_f32(m, batch, seed)


def _gpu(chw, fn, plan, a, out=None):
    import torch

    ad = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    od = torch.empty_like(ad) if out is None else out
    fn(plan, ad, od)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(plan) == 0
    return od.cpu().numpy()


CASES = [(m, b) for m in range(0, 15) for b in (1, 3)] + [(5, 300), (12, 9), (13, 2), (14, 5), (16, 3), (20, 2), (22, 1)]
MODES = [("f32", "per_level"), ("f32", "end"), ("f32", "none"), ("i32", "none")]


@pytest.mark.parametrize("m,batch", CASES)
@pytest.mark.parametrize("dtype,norm", MODES)
def test_haar_forward_and_inverse_bitwise(chw, m, batch, dtype, norm):
    x = _inputs(m, batch, dtype, 1000 + m)
    p = chw.chw_plan(m, batch, dtype, norm)
    z = _gpu(chw, chw.chw_haar, p, x)
    assert_bitwise(z, O.haar_forward(x, m, ORACLE_DT[dtype], norm), f"Psi m={m} b={batch} {dtype} {norm}")
    w = _gpu(chw, chw.chw_haar_inverse, p, z)
    assert_bitwise(w, O.haar_inverse(z, m, ORACLE_DT[dtype], norm), f"Psi^T m={m} b={batch} {dtype} {norm}")
    if norm != "none":
        assert np.abs(w - x).max() <= 1e-5 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("m", [26, 27])
def test_haar_multi_pass_large(chw, m):
    # two and three passes (13 + 13, 13 + 13 + 1 levels)
    x = W.uniform_pm1_f32(m, 1, 3000 + m)
    for norm in ("per_level", "end"):
        p = chw.chw_plan(m, 1, "f32", norm)
        z = _gpu(chw, chw.chw_haar, p, x)
        assert_bitwise(z, O.haar_forward(x, m, np.float32, norm), f"Psi m={m} {norm}")
        w = _gpu(chw, chw.chw_haar_inverse, p, z)
        assert_bitwise(w, O.haar_inverse(z, m, np.float32, norm), f"Psi^T m={m} {norm}")


HW_CASES = [(m, b) for m in range(0, 18) for b in (1, 2)] + [(10, 64), (13, 5), (16, 33), (20, 2), (21, 1), (22, 2)]


@pytest.mark.parametrize("m,batch", HW_CASES)
@pytest.mark.parametrize("dtype,norm", MODES)
def test_haar_walsh_bitwise(chw, m, batch, dtype, norm):
    z = _inputs(m, batch, dtype, 2000 + m)
    p = chw.chw_plan(m, batch, dtype, norm, chw.CHW_FLAG_HAAR_WALSH)
    y = _gpu(chw, chw.chw_from_haar, p, z)
    assert_bitwise(y, O.haar_walsh(z, m, ORACLE_DT[dtype], norm), f"HW m={m} b={batch} {dtype} {norm}")


@pytest.mark.parametrize("m,batch", [(3, 4), (12, 8), (16, 4), (18, 1)])
def test_haar_walsh_in_place(chw, m, batch):
    import torch

    z = W.normal_f32(m, batch, 77)
    p = chw.chw_plan(m, batch, "f32", "per_level", chw.CHW_FLAG_HAAR_WALSH)
    zd = torch.from_numpy(z).cuda()
    chw.chw_from_haar(p, zd, zd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    assert_bitwise(zd.cpu().numpy(), O.haar_walsh(z, m, np.float32, "per_level"), "in place")


@pytest.mark.parametrize("m,batch", [(1, 5), (3, 64), (5, 40), (9, 16), (11, 8), (13, 4), (14, 4), (15, 6), (16, 8),
                                     (19, 2)])
@pytest.mark.parametrize("dtype,norm", [("f32", "per_level"), ("i32", "none"), ("f32", "end")])
def test_forward_with_haar_side_output(chw, m, batch, dtype, norm):
    # y is chw_forward's result and z chw_haar's, bit for bit; for m <= 16 both leave one
    # pass (z captured from the cascade's registers), for m = 19 two calls
    import torch

    x = _inputs(m, batch, dtype, 4000 + m)
    p = chw.chw_plan(m, batch, dtype, norm)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    zd = torch.empty_like(xd)
    chw.chw_forward_haar(p, xd, yd, zd)
    y_ref = torch.empty_like(xd)
    chw.chw_forward(p, xd, y_ref)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    dt = ORACLE_DT[dtype]
    assert_bitwise(zd.cpu().numpy(), O.haar_forward(x, m, dt, norm), "side output")
    assert_bitwise(yd.cpu().numpy(), y_ref.cpu().numpy(), "same as chw_forward")
    assert_bitwise(yd.cpu().numpy(), O.chw_cascade(x, m, dt, norm), "cascade")


@pytest.mark.parametrize("m", [12, 16])
def test_forward_with_haar_side_output_in_place_and_tail(chw, m):
    # y == x (in place) and a batch whose last 2^13-word tile is partly empty (m = 12: 3
    # signals in two tiles): nothing past the batch is written
    import torch

    batch = 3
    x = _inputs(m, batch, "f32", 4100 + m)
    p = chw.chw_plan(m, batch, "f32", "end")
    buf = torch.full((batch + 1, 1 << m), 7.0, device="cuda")
    zbuf = torch.full((batch + 1, 1 << m), 9.0, device="cuda")
    xd, zd = buf[:batch], zbuf[:batch]
    xd.copy_(torch.from_numpy(x))
    chw.chw_forward_haar(p, xd, xd, zd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    assert_bitwise(zd.cpu().numpy(), O.haar_forward(x, m, np.float32, "end"), "side output")
    assert_bitwise(xd.cpu().numpy(), O.chw_cascade(x, m, np.float32, "end"), "in place")
    assert np.all(buf[batch].cpu().numpy() == 7.0) and np.all(zbuf[batch].cpu().numpy() == 9.0)


@pytest.mark.parametrize("m", [10, 14, 16])
def test_forward_with_haar_side_output_16_byte_aligned_z(chw, m):
    # z on a 16-byte but not 32-byte boundary: the captures that would leave as 32-byte
    # stores go out as two 16-byte stores, same bits
    import torch

    batch = 5
    x = _inputs(m, batch, "f32", 4200 + m)
    p = chw.chw_plan(m, batch, "f32", "end")
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    zbuf = torch.full((batch * (1 << m) + 8,), 9.0, device="cuda")
    assert zbuf.data_ptr() % 32 == 0
    zd = zbuf[4: 4 + batch * (1 << m)].view(batch, 1 << m)  # 16 bytes past a 32-byte boundary
    chw.chw_forward_haar(p, xd, yd, zd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    assert_bitwise(zd.cpu().numpy(), O.haar_forward(x, m, np.float32, "end"), "side output")
    assert_bitwise(yd.cpu().numpy(), O.chw_cascade(x, m, np.float32, "end"), "cascade")
    rest = zbuf.cpu().numpy()
    assert np.all(rest[:4] == 9.0) and np.all(rest[4 + batch * (1 << m):] == 9.0)


def test_haar_argument_errors(chw):
    import torch

    p = chw.chw_plan(10, 2, "f32", "end")
    x = torch.zeros(2, 1024, device="cuda")
    with pytest.raises(chw.ChwError, match="overlap"):
        chw.chw_haar(p, x, x)
    with pytest.raises(chw.ChwError, match="overlap"):
        chw.chw_haar_inverse(p, x, x)
    with pytest.raises(chw.ChwError, match="CHW_FLAG_HAAR_WALSH"):
        chw.chw_from_haar(p, x, torch.empty_like(x))
    q = chw.chw_plan(10, 2, "bf16", "end")
    xb = torch.zeros(2, 1024, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(chw.ChwError, match="int32 or fp32"):
        chw.chw_haar(q, xb, torch.empty_like(xb))
    with pytest.raises(chw.ChwError):
        chw.chw_plan(10, 2, "bf16", "end", chw.CHW_FLAG_HAAR_WALSH)
