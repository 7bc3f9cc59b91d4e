"""y = D H_m x under torch.autograd (GPU): backward through chw_adjoint."""

import numpy as np
import pytest

import oracle as O
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def layer_cls(cuda_device):
    from paper_1609_06641_gb300 import build

    build.build()
    from paper_1609_06641_gb300.autograd import DHLayer

    return DHLayer


def oracle_loss(x64, m, d, w):
    """FP64 loss sum(w * D H x) through the oracle."""
    return float(np.sum(w * (d * O.wht_fast_dyadic(x64, m))))


@pytest.mark.parametrize("m", [4, 5, 6, 7, 8])
def test_backward_vs_fp64_finite_differences(layer_cls, m):
    import torch

    rng = np.random.default_rng(m)
    batch = 2
    x64 = rng.standard_normal((batch, 1 << m))
    w = rng.standard_normal((batch, 1 << m))
    d = W.diag_pm1(m, 6).astype(np.float64)
    layer = layer_cls(m, torch.from_numpy(W.diag_pm1(m, 6)).cuda())
    x = torch.tensor(x64, dtype=torch.float32, device="cuda", requires_grad=True)
    y = layer(x)
    (y * torch.tensor(w, dtype=torch.float32, device="cuda")).sum().backward()
    g = x.grad.cpu().numpy().astype(np.float64)
    # central differences of the FP64 oracle loss on a sample of coordinates
    h = 1e-6
    fd = np.zeros_like(x64)
    idx = [(b, j) for b in range(batch) for j in rng.choice(1 << m, min(12, 1 << m), replace=False)]
    for b, j in idx:
        xp, xm = x64.copy(), x64.copy()
        xp[b, j] += h
        xm[b, j] -= h
        fd[b, j] = (oracle_loss(xp, m, d, w) - oracle_loss(xm, m, d, w)) / (2 * h)
    got = np.array([g[b, j] for b, j in idx])
    ref = np.array([fd[b, j] for b, j in idx])
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_sum_of_squares_gradient_is_2x(layer_cls):
    import torch

    m, batch = 14, 512
    x64 = np.random.default_rng(0).standard_normal((batch, 1 << m))
    layer = layer_cls(m, torch.from_numpy(W.diag_pm1(m, 6)).cuda())
    x = torch.tensor(x64, dtype=torch.float32, device="cuda", requires_grad=True)
    (layer(x) ** 2).sum().backward()
    g = x.grad.double()
    assert torch.allclose(g, 2 * x.double(), rtol=0, atol=1e-5 * float(x.abs().max()))


def test_gradient_matches_oracle_transpose(layer_cls):
    import torch

    m, batch = 14, 16
    rng = np.random.default_rng(1)
    x = torch.randn(batch, 1 << m, device="cuda", requires_grad=True)
    w = rng.standard_normal((batch, 1 << m)).astype(np.float32)
    d = W.diag_pm1(m, 6)
    layer = layer_cls(m, torch.from_numpy(d).cuda())
    (layer(x) * torch.from_numpy(w).cuda()).sum().backward()
    ref = O.chw_reverse_cascade(w * d.astype(np.float32), m, np.float32, "end")
    assert np.array_equal(x.grad.cpu().numpy().view(np.uint32), ref.view(np.uint32))
