"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

fp32: the kernels perform the butterflies of the cascade (Theorem 1) in an order that
gives every value the same operands, so the results must equal the oracle's fp32
cascade bit for bit (a stronger bar than the normwise relative error <= 1e-6 against the
FP64 definition, which is checked too).  int32: bit-exact against the int64 fast WHT
reduced mod 2^32.
"""

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise, run_forward
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_GATE = 1e-6


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    chw._lib.load()
    return chw


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


def _check_f32(chw, torch, x, m, norm, **kw):
    got, info = run_forward(chw, torch, x, m, "f32", norm, **kw)
    ref32 = O.chw_cascade(x, m, np.float32, norm)
    assert_bitwise(got, ref32, f"m={m} {norm} tier={info.tier}")
    ref = O.wht_fast_dyadic(x.astype(np.float64), m)
    if norm == "none":
        ref = ref * 2.0 ** (m / 2)
    err = O.rel_err_per_signal(got, ref).max()
    assert err <= FP32_GATE, (m, norm, err)
    return info


# ---------------------------------------------------------------- every m, every tier
@pytest.mark.parametrize("m", list(range(0, 18)))
@pytest.mark.parametrize("norm", ["per_level", "end"])
def test_f32_every_m(chw, torch, m, norm):
    # batch chosen so tiles are ragged: not a multiple of the signals per tile
    batch = 3 if m >= 13 else max(3, (1 << (14 - m)) + 5)
    x = W.normal_f32(m, batch, seed=100 + m)
    info = _check_f32(chw, torch, x, m, norm)
    if m in (15, 16):
        assert info.tier == 7 and info.cluster == 1  # one CTA per signal, tensor memory
    elif m == 17:
        assert info.tier == 8 and info.passes == 1 and info.cluster == 2  # two SMs, tensor memory


@pytest.mark.parametrize("m", [15, 16, 17])
@pytest.mark.parametrize("norm", ["per_level", "end"])
def test_cluster_tier_on_request(chw, torch, m, norm):
    x = W.normal_f32(m, 5, seed=140 + m)
    info = _check_f32(chw, torch, x, m, norm, flags=chw.CHW_FLAG_CLUSTER)
    assert info.tier == 2 and info.cluster == 1 << (m - 14)


@pytest.mark.parametrize("m", [15, 16])
@pytest.mark.parametrize("batch", [1, 2, 157, 331])
def test_tmem_tier_batches(chw, torch, m, batch):
    # 157 and 331 signals: more signals than SMs, so CTAs walk several signals and the
    # last round leaves SMs idle; batch 1 and 2 leave most CTAs without work
    x = W.normal_f32(m, batch, seed=170 + m + batch)
    rows = sorted(set(np.random.default_rng(batch).choice(batch, min(batch, 6), replace=False)) | {0, batch - 1})
    got, info = run_forward(chw, torch, x, m, "f32", "end")
    assert info.tier == 7
    assert_bitwise(got[rows], O.chw_cascade(x[rows], m, np.float32, "end"), f"m={m} batch={batch}")


@pytest.mark.parametrize("m", [15, 16])
def test_tmem_tier_norm_none_and_i32_wrap(chw, torch, m):
    x = W.normal_f32(m, 3, seed=180 + m)
    info = _check_f32(chw, torch, x, m, "none")
    assert info.tier == 7
    rng = np.random.default_rng(m)
    xi = rng.integers(-(2**31), 2**31 - 1, size=(3, 1 << m), endpoint=True, dtype=np.int64).astype(np.int32)
    got, info = run_forward(chw, torch, xi, m, "i32", "none")
    assert info.tier == 7
    assert_bitwise(got, O.chw_cascade(xi, m, np.int32, "none"), "int32 wrap")


@pytest.mark.parametrize("m", [15, 16, 17])
@pytest.mark.parametrize("norm", ["per_level", "end"])
def test_rowstack_tier(chw, torch, m, norm):
    x = W.normal_f32(m, 5, seed=150 + m)
    info = _check_f32(chw, torch, x, m, norm, flags=4)
    assert info.tier == 6  # one CTA per signal, rows through L2
    xi = W.uniform_int32(m, 3, seed=160 + m, bound=2 ** (29 - m))
    got, _ = run_forward(chw, torch, xi, m, "i32", "none", flags=4)
    assert np.array_equal(got, O.wht_fast_dyadic(xi.astype(np.int64), m, normalised=False).astype(np.int32))


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 5, 7, 10, 12, 13, 14, 15, 16, 17])
def test_i32_every_m(chw, torch, m):
    batch = 3 if m >= 13 else max(3, (1 << (14 - m)) + 3)
    x = W.uniform_int32(m, batch, seed=200 + m, bound=2 ** max(0, 29 - m))
    got, info = run_forward(chw, torch, x, m, "i32", "none")
    ref = O.wht_fast_dyadic(x.astype(np.int64), m, normalised=False)
    assert np.array_equal(got, ref.astype(np.int32)), (m, info.tier)


def test_i32_wraps_like_int32_ring(chw, torch):
    m = 12
    rng = np.random.default_rng(5)
    x = rng.integers(-(2**31), 2**31 - 1, size=(5, 1 << m), endpoint=True, dtype=np.int64).astype(np.int32)
    got, _ = run_forward(chw, torch, x, m, "i32", "none")
    assert_bitwise(got, O.chw_cascade(x, m, np.int32, "none"), "int32 wrap")


@pytest.mark.parametrize("m", [3, 9, 12])
def test_f32_norm_none(chw, torch, m):
    x = W.normal_f32(m, 7, seed=9)
    _check_f32(chw, torch, x, m, "none")


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_tiny_m_batch_not_multiple_of_a_row(chw, torch, m):
    # 2^m * batch not a multiple of 32 words: the plan takes the plain kernel
    x = W.normal_f32(m, 5, seed=m)
    info = _check_f32(chw, torch, x, m, "per_level")
    assert info.tier == 0


@pytest.mark.parametrize("m", [2, 6, 10, 13])
def test_forced_simple_kernel(chw, torch, m):
    x = W.normal_f32(m, 9, seed=m)
    info = _check_f32(chw, torch, x, m, "end", flags=1)
    assert info.tier == 0


# ---------------------------------------------------------------- two HBM passes
@pytest.mark.parametrize("m", [11, 14])
@pytest.mark.parametrize("norm", ["per_level", "end"])
def test_forced_two_pass(chw, torch, m, norm):
    x = W.normal_f32(m, 6, seed=300 + m)
    info = _check_f32(chw, torch, x, m, norm, flags=2)
    assert info.tier == 3 and info.passes == 2


@pytest.mark.parametrize("m", [18, 19, 20, 21, 22, 23, 24])
def test_two_pass_f32(chw, torch, m):
    x = W.normal_f32(m, 2, seed=400 + m)
    info = _check_f32(chw, torch, x, m, "end")
    assert info.tier == 3 and info.passes == 2


@pytest.mark.parametrize("m", [18, 21, 24])
def test_two_pass_i32_and_per_level(chw, torch, m):
    x = W.uniform_int32(m, 2, seed=500 + m, bound=2 ** max(0, 29 - m))
    got, _ = run_forward(chw, torch, x, m, "i32", "none")
    assert np.array_equal(got, O.wht_fast_dyadic(x.astype(np.int64), m, normalised=False).astype(np.int32))
    xf = W.normal_f32(m, 1, seed=600 + m)
    _check_f32(chw, torch, xf, m, "per_level")


# ---------------------------------------------------------------- in place, adjoint, D
@pytest.mark.parametrize("m", [5, 12, 16, 19])
def test_in_place(chw, torch, m):
    x = W.normal_f32(m, 3, seed=m)
    got, _ = run_forward(chw, torch, x, m, "f32", "end", inplace=True)
    assert_bitwise(got, O.chw_cascade(x, m, np.float32, "end"), f"in place m={m}")


@pytest.mark.parametrize("m", [4, 10, 14, 16, 20])
def test_adjoint_is_reversed_cascade(chw, torch, m):
    x = W.normal_f32(m, 3, seed=700 + m)
    got, _ = run_forward(chw, torch, x, m, "f32", "per_level", adjoint=True)
    assert_bitwise(got, O.chw_reverse_cascade(x, m, np.float32, "per_level"), f"adjoint m={m}")
    if m <= 10:  # H^T y for each row y, from the dense matrix of eq. (1)
        assert O.rel_err_per_signal(got, x.astype(np.float64) @ O.hadamard_dyadic(m)).max() <= FP32_GATE


@pytest.mark.parametrize("m", [6, 12, 14, 15, 16, 19])
def test_diag_forward_and_adjoint(chw, torch, m):
    x = W.normal_f32(m, 4, seed=800 + m)
    d = W.diag_pm1(m, seed=6)
    got, _ = run_forward(chw, torch, x, m, "f32", "end", diag=d)
    ref = O.chw_cascade(x, m, np.float32, "end") * d.astype(np.float32)
    assert_bitwise(got, ref, f"D H x m={m}")
    got_a, _ = run_forward(chw, torch, x, m, "f32", "end", adjoint=True, diag=d)
    ref_a = O.chw_reverse_cascade(x * d.astype(np.float32), m, np.float32, "end")
    assert_bitwise(got_a, ref_a, f"H^T D y m={m}")


@pytest.mark.parametrize("m", [0, 1, 6, 14, 16, 17, 19])
@pytest.mark.parametrize("shift", [0, 1, 4])
def test_diag_at_any_byte_offset(chw, torch, m, shift):
    # D may start at any byte: an array on a 16-byte (4-byte) boundary is read 16 (4) bytes
    # at a time, others byte by byte -- the same signs either way, forward (D on the
    # outputs, also through the tiles' TMA store) and adjoint (D on the inputs)
    n = 1 << m
    batch = 3 if m >= 13 else max(3, (1 << (14 - m)) + 3)
    x = W.normal_f32(m, batch, seed=900 + m)
    d = W.diag_pm1(m, seed=7 + m)
    dev = torch.device("cuda:0")
    dbuf = torch.zeros(n + 32, dtype=torch.int8, device=dev)
    assert dbuf.data_ptr() % 16 == 0
    dd = dbuf[shift: shift + n]
    dd.copy_(torch.from_numpy(d))
    p = chw.chw_plan(m, batch, "f32", "end")
    xd = torch.from_numpy(x).to(dev)
    yf, ya = torch.empty_like(xd), torch.empty_like(xd)
    chw.chw_forward(p, xd, yf, diag=dd)
    chw.chw_adjoint(p, xd, ya, diag=dd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    assert_bitwise(yf.cpu().numpy(), O.chw_cascade(x, m, np.float32, "end") * d.astype(np.float32), f"D H x m={m}")
    ref_a = O.chw_reverse_cascade(x * d.astype(np.float32), m, np.float32, "end")
    assert_bitwise(ya.cpu().numpy(), ref_a, f"H^T D y m={m}")


def test_round_trip_identity(chw, torch):
    m = 16
    x = W.normal_f32(m, 8, seed=1)
    y, _ = run_forward(chw, torch, x, m, "f32", "per_level")
    back, _ = run_forward(chw, torch, y, m, "f32", "per_level", adjoint=True)
    assert O.rel_err_per_signal(back, x).max() <= FP32_GATE


# ---------------------------------------------------------------- boundary checks
def test_argument_errors(chw, torch):
    import ctypes

    from paper_1609_06641_gb300 import _lib

    lib = _lib.load()
    p = chw.chw_plan(10, 4, "f32", "end")
    buf = torch.zeros(4 * 1024 + 8, device="cuda:0")
    base = buf.data_ptr()
    st = lib.chw_forward(p.handle, ctypes.c_void_p(base + 4), ctypes.c_void_p(base), None, None, None, None)
    assert st == _lib.CHW_ERR_ALIGNMENT
    st = lib.chw_forward(p.handle, None, ctypes.c_void_p(base), None, None, None, None)
    assert st == _lib.CHW_ERR_INVALID_ARG
    e = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    st = lib.chw_forward(p.handle, ctypes.c_void_p(base), ctypes.c_void_p(base), ctypes.c_void_p(e.data_ptr()), None, None, None)
    assert st == _lib.CHW_ERR_INVALID_ARG
    with pytest.raises(chw.ChwError):
        chw.chw_plan(31, 1)
    with pytest.raises(chw.ChwError):
        chw.chw_plan(4, 1, "i32", "end")
    with pytest.raises(chw.ChwError):
        chw.chw_plan(14, 1, "bf16", "end")
    assert chw.chw_last_device_status(p) == 0


# ---------------------------------------------------------------- benchmark shapes
def test_config_m10_batch64(chw, torch):
    x = W.normal_f32(10, 64, seed=0)
    got, _ = run_forward(chw, torch, x, 10, "f32", "per_level")
    assert_bitwise(got, O.chw_cascade(x, 10, np.float32, "per_level"), "m=10 b=64")
    for ref in (O.wht_dense(x.astype(np.float64), 10), O.wht_fast_dyadic(x.astype(np.float64), 10)):
        assert O.rel_err_per_signal(got, ref).max() <= FP32_GATE


@pytest.mark.parametrize("norm", ["end", "per_level"])
def test_config_m16_batch4096_f32_sampled(chw, torch, norm):
    m, batch = 16, 4096
    x = W.normal_f32(m, batch, seed=2)
    got, info = run_forward(chw, torch, x, m, "f32", norm)
    assert info.tier == 7
    rows = np.random.default_rng(0).choice(batch, 6, replace=False)
    rows = np.concatenate([rows, [0, batch - 1]])
    assert_bitwise(got[rows], O.chw_cascade(x[rows], m, np.float32, norm), "m=16 sampled rows")
    assert O.rel_err_per_signal(got[rows], O.wht_fast_dyadic(x[rows].astype(np.float64), m)).max() <= FP32_GATE
    # every row: Parseval (H orthogonal) within fp32 rounding
    ratio = np.linalg.norm(got.astype(np.float64), axis=1) / np.linalg.norm(x.astype(np.float64), axis=1)
    assert np.abs(ratio - 1).max() < 1e-6


def test_config_m16_batch4096_i32_sampled(chw, torch):
    m, batch = 16, 4096
    x = W.uniform_int32(m, batch, seed=1)
    got, _ = run_forward(chw, torch, x, m, "i32", "none")
    rows = np.concatenate([np.random.default_rng(1).choice(batch, 6, replace=False), [0, batch - 1]])
    assert np.array_equal(got[rows], O.wht_fast_dyadic(x[rows].astype(np.int64), m, normalised=False))
    # every row: the unnormalised transform applied twice is n x (exact in int32 here)
    back, _ = run_forward(chw, torch, got, m, "i32", "none", adjoint=True)
    assert np.array_equal(back.astype(np.int64), x.astype(np.int64) << m)


def test_config_m26_batch4(chw, torch):
    m = 26
    x = W.uniform_pm1_f32(m, 4, seed=3)
    got, info = run_forward(chw, torch, x, m, "f32", "end")
    assert info.passes == 2
    assert_bitwise(got[1], O.chw_cascade(x[1:2], m, np.float32, "end")[0], "m=26 signal 1")
    ks = np.random.default_rng(3).integers(0, 1 << m, 3)
    ref = O.wht_closed_form(x[3], m, ks)
    assert np.abs(got[3, ks] - ref).max() <= 1e-5 * np.abs(ref).max()
    back, _ = run_forward(chw, torch, got, m, "f32", "end", adjoint=True)
    assert O.rel_err_per_signal(back, x).max() <= FP32_GATE


def test_config_m28_batch1(chw, torch):
    m = 28
    x = W.uniform_pm1_f32(m, 1, seed=3)
    got, info = run_forward(chw, torch, x, m, "f32", "end")
    assert info.passes == 2
    ks = np.random.default_rng(4).integers(0, 1 << m, 2)
    ref = O.wht_closed_form(x[0], m, ks)
    assert np.abs(got[0, ks] - ref).max() <= 1e-5 * np.abs(ref).max()
    nx = np.linalg.norm(x.astype(np.float64))
    assert abs(np.linalg.norm(got.astype(np.float64)) / nx - 1) < 1e-6
    back, _ = run_forward(chw, torch, got, m, "f32", "end", adjoint=True)
    assert O.rel_err_per_signal(back, x).max() <= FP32_GATE
