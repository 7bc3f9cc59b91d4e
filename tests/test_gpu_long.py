"""Long single signals, m = 25..30: the two-pass split y = H_b X^T H_a with both passes on
the tensor-memory kernel (GPU).

For m >= 26 the column pass runs column blocks of 2^a rows x 2^c columns on one SM each
(a = m - 16; c = 5 for a <= 11, else 16 - a), which needs the first pass to write blocks of
that width.  Transforming such signals on the host takes minutes, so the outputs are
checked at sampled positions (2^20 random ones plus the first and last 4096) against the
oracle's closed form for a sparse input, exactly: the unnormalised int32 transform is an
integer sum, and with END normalisation every butterfly of a sparse integer input is exact
in fp32, so the result is that sum rounded once and multiplied by fp32(2^{-m/2}).  Dense
inputs are checked by the round trip H^T H x = x (two transforms: twice the fp32 gate)
and by Parseval.
"""

import numpy as np
import pytest

import oracle as O
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_GATE = 1e-6


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


@pytest.fixture(scope="module")
def torch(cuda_device):
    import torch

    return torch


def sparse_case(m, seed, count=8, bound=1000):
    rng = np.random.default_rng(seed)
    n = 1 << m
    js = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, count - 2)]))
    cs = rng.integers(-bound, bound + 1, len(js))
    ks = np.unique(np.concatenate([rng.integers(0, n, 1 << 20), np.arange(4096), np.arange(n - 4096, n)]))
    return js, cs, ks


def run_sparse(chw, torch, m, dtype, norm, js, cs, ks, diag=None):
    dev = torch.device("cuda:0")
    tdt = torch.int32 if dtype == "i32" else torch.float32
    x = torch.zeros(1, 1 << m, dtype=tdt, device=dev)
    x[0, torch.from_numpy(js).to(dev)] = torch.from_numpy(cs).to(tdt).to(dev)
    y = torch.empty_like(x)
    p = chw.chw_plan(m, 1, dtype, norm)
    info = chw.chw_plan_get_info(p)
    chw.chw_forward(p, x, y, diag=None if diag is None else torch.from_numpy(diag).to(dev))
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    got = y[0, torch.from_numpy(ks).to(dev)].cpu().numpy()
    del x, y
    p.close()
    return got, info


@pytest.mark.parametrize("m", [25, 26, 27, 28, 29, 30])
def test_sparse_int32_exact_at_sampled_outputs(chw, torch, m):
    js, cs, ks = sparse_case(m, 1000 + m)
    got, info = run_sparse(chw, torch, m, "i32", "none", js, cs, ks)
    assert info.tier == 3 and info.passes == 2 and info.row_bits == 16
    want = O.wht_sparse_closed_form(js, cs, m, ks, normalised=False)
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("m", [26, 27, 28, 29, 30])
def test_sparse_f32_end_bitwise_at_sampled_outputs(chw, torch, m):
    js, cs, ks = sparse_case(m, 2000 + m)
    got, _ = run_sparse(chw, torch, m, "f32", "end", js, cs, ks)
    sums = O.wht_sparse_closed_form(js, cs, m, ks, normalised=False)  # exact integers
    want = sums.astype(np.float32) * O.end_scale_f32(m)  # one fp32 multiply (eq. (1)'s scale)
    assert np.array_equal(got.view(np.uint32), want.astype(np.float32).view(np.uint32))


@pytest.mark.parametrize("m", [27, 28])
def test_sparse_int32_with_output_diagonal(chw, torch, m):
    js, cs, ks = sparse_case(m, 3000 + m)
    d = W.diag_pm1(m, seed=6)
    got, _ = run_sparse(chw, torch, m, "i32", "none", js, cs, ks, diag=d)
    want = O.wht_sparse_closed_form(js, cs, m, ks, normalised=False) * d[ks].astype(np.int64)
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("m,norm", [(27, "per_level"), (29, "end"), (30, "per_level")])
def test_dense_round_trip_and_parseval(chw, torch, m, norm):
    dev = torch.device("cuda:0")
    x = torch.from_numpy(W.uniform_pm1_f32(m, 1, seed=3)).to(dev)
    y = torch.empty_like(x)
    p = chw.chw_plan(m, 1, "f32", norm)
    chw.chw_forward(p, x, y)
    back = torch.empty_like(x)
    chw.chw_adjoint(p, y, back)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    x64 = x.double()
    # H^T H x chains two transforms, each within the fp32 gate, so their errors add (m = 30
    # in per-level normalisation passes 60 rounded levels: measured 1.05e-6)
    assert float((back.double() - x64).norm() / x64.norm()) <= 2 * FP32_GATE
    assert abs(float(y.double().norm() / x64.norm()) - 1) < 1e-6

