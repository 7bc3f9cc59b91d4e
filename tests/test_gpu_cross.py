"""The tensor-memory tier for signals longer than one SM holds (m = 17 on a pair of SMs),
through the C ABI, against the oracle's fp32 cascade of Theorem 1 bit for bit (needs a
GB300).

Each SM of a cluster holds the labels of one value of the top label bits; the last label
bits pair values on different SMs and are exchanged over distributed shared memory.  The
cascade's order of butterflies per value is kept, so the results are the cascade's.
"""

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise, run_forward
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CROSS_TIER = 8
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


def _rows(batch, seed):
    """A few sampled signals plus the first and the last (the oracle is slow at m = 17)."""
    pick = np.random.default_rng(seed).choice(batch, min(batch, 4), replace=False)
    return np.array(sorted(set(pick.tolist()) | {0, batch - 1}))


@pytest.mark.parametrize("m", [17])
@pytest.mark.parametrize("norm", ["per_level", "end", "none"])
@pytest.mark.parametrize("batch", [1, 2, 83, 331])
def test_cross_f32(chw, torch, m, norm, batch):
    # 83 and 331 signals: more signals than clusters (CTAs walk several signals, the last
    # round leaves clusters idle); 1 and 2 leave most clusters without work
    x = W.normal_f32(m, batch, seed=1700 + batch)
    got, info = run_forward(chw, torch, x, m, "f32", norm)
    assert info.tier == CROSS_TIER and info.passes == 1 and info.cluster == 1 << (m - 16)
    rows = _rows(batch, batch)
    assert_bitwise(got[rows], O.chw_cascade(x[rows], m, np.float32, norm), f"m={m} {norm} batch={batch}")
    if norm != "none":
        ref = O.wht_fast_dyadic(x[rows].astype(np.float64), m)
        assert O.rel_err_per_signal(got[rows], ref).max() <= FP32_GATE
        # every signal: Parseval (H orthogonal) within fp32 rounding
        ratio = np.linalg.norm(got.astype(np.float64), axis=1) / np.linalg.norm(x.astype(np.float64), axis=1)
        assert np.abs(ratio - 1).max() < 1e-6


@pytest.mark.parametrize("m", [17])
def test_cross_i32_wrap(chw, torch, m):
    rng = np.random.default_rng(m)
    x = rng.integers(-(2**31), 2**31 - 1, size=(3, 1 << m), endpoint=True, dtype=np.int64).astype(np.int32)
    got, info = run_forward(chw, torch, x, m, "i32", "none")
    assert info.tier == CROSS_TIER
    assert_bitwise(got, O.chw_cascade(x, m, np.int32, "none"), "int32 wrap")
    xs = W.uniform_int32(m, 5, seed=1710, bound=2 ** (29 - m))
    got, _ = run_forward(chw, torch, xs, m, "i32", "none")
    assert np.array_equal(got, O.wht_fast_dyadic(xs.astype(np.int64), m, normalised=False).astype(np.int32))


@pytest.mark.parametrize("m", [17])
def test_cross_adjoint_diag_in_place(chw, torch, m):
    x = W.normal_f32(m, 3, seed=1720)
    d = W.diag_pm1(m, seed=6)
    got, _ = run_forward(chw, torch, x, m, "f32", "end", diag=d)
    assert_bitwise(got, O.chw_cascade(x, m, np.float32, "end") * d.astype(np.float32), "D H x")
    got_a, _ = run_forward(chw, torch, x, m, "f32", "per_level", adjoint=True, diag=d)
    ref_a = O.chw_reverse_cascade(x * d.astype(np.float32), m, np.float32, "per_level")
    assert_bitwise(got_a, ref_a, "H^T D y")
    got_i, _ = run_forward(chw, torch, x, m, "f32", "end", inplace=True)
    assert_bitwise(got_i, O.chw_cascade(x, m, np.float32, "end"), "in place")


@pytest.mark.parametrize("m", [17])
def test_cross_equals_two_pass(chw, torch, m):
    # the same signals through the two HBM passes of the split (a = 6): identical bits
    x = W.normal_f32(m, 40, seed=1730)
    got, info = run_forward(chw, torch, x, m, "f32", "per_level")
    assert info.tier == CROSS_TIER
    ref, rinfo = run_forward(chw, torch, x, m, "f32", "per_level", flags=chw.CHW_FLAG_FORCE_MULTIPASS)
    assert rinfo.passes == 2
    assert_bitwise(got, ref, "cross-SM vs two passes")


@pytest.mark.parametrize("m", [17])
def test_cross_checked_mode(chw, torch, m):
    x = W.normal_f32(m, 9, seed=1740)
    got, info = run_forward(chw, torch, x, m, "f32", "end", flags=chw.CHW_FLAG_CHECKED)
    assert info.tier == CROSS_TIER
    rows = _rows(9, 1)
    assert_bitwise(got[rows], O.chw_cascade(x[rows], m, np.float32, "end"), "checked mode")


@pytest.mark.parametrize("m", [17])
def test_cross_host_buffers(chw, torch, m):
    # chw_forward_host runs chunks of 64 MiB on three streams at once: each stream has its
    # own exchange scratch, so the chunks' kernels may overlap on the device
    batch = 1200  # 600 MiB: ten chunks, the last one partial
    x = W.normal_f32(m, batch, seed=1750)
    y = np.empty_like(x)
    p = chw.chw_plan(m, batch, "f32", "end")
    assert chw.chw_plan_get_info(p).tier == CROSS_TIER
    chw.chw_forward_host(p, x, y)
    assert chw.chw_last_device_status(p) == 0
    rows = np.array([0, 127, 128, 700, batch - 1])
    assert_bitwise(y[rows], O.chw_cascade(x[rows], m, np.float32, "end"), "host buffers")
    xd = torch.from_numpy(x[:256]).to("cuda:0")
    yd = torch.empty_like(xd)
    q = chw.chw_plan(m, 256, "f32", "end")
    chw.chw_forward(q, xd, yd)
    torch.cuda.synchronize()
    assert_bitwise(yd.cpu().numpy(), y[:256], "host buffers vs device buffers")
