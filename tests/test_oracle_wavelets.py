"""Pins of the oracle's Haar, inverse Haar and Haar-Walsh transforms (no GPU).

They are checked against the dense matrices of eq. (2) (Psi_m, itself pinned by the
hand-derived golden matrices) and eq. (4) (the block diagonal of Hadamard matrices),
against orthogonality, against the literal cascade of Theorem 1 (stage 0 followed by
stages 1..m-1 is the whole cascade, operation for operation), and against unit vectors
whose images are single columns of H_k.
"""

import numpy as np
import pytest

import oracle as O


def _haar_blocks(m):
    """(k, start, length) of the Haar scales: position 0, then blocks [2^k, 2^(k+1))."""
    return [(k, 1 << k, 1 << k) for k in range(m)]


def test_haar_levels_by_bit_length():
    for m in range(0, 11):
        lev = O.haar_levels(m)
        assert lev[0] == m
        for p in range(1, 1 << m):
            assert lev[p] == m - (p.bit_length() - 1)
        # block sizes: 2^(m-l) coefficients at level l, plus the approximation
        for l in range(1, m + 1):
            assert int((lev[1:] == l).sum()) == 1 << (m - l)


@pytest.mark.parametrize("m", range(0, 10))
def test_haar_forward_is_eq2_matrix(m):
    rng = np.random.default_rng(100 + m)
    x = rng.standard_normal((3, 1 << m))
    psi = O.haar_matrix(m)
    for norm in ("per_level", "end"):
        z = O.haar_forward(x, m, np.float64, norm)
        assert np.abs(z - x @ psi.T).max() < 1e-12, norm
    xi = rng.integers(-1000, 1000, (2, 1 << m))
    zi = O.haar_forward(xi, m, np.int64, "none")
    assert np.array_equal(zi, xi @ O.haar_matrix(m, normalised=False).T)


@pytest.mark.parametrize("m", range(0, 10))
def test_haar_inverse_is_transpose(m):
    rng = np.random.default_rng(200 + m)
    z = rng.standard_normal((3, 1 << m))
    psi = O.haar_matrix(m)
    for norm in ("per_level", "end"):
        x = O.haar_inverse(z, m, np.float64, norm)
        assert np.abs(x - z @ psi).max() < 1e-12, norm
        # orthogonality: Psi^T Psi = I
        assert np.abs(O.haar_inverse(O.haar_forward(x, m, np.float64, norm), m, np.float64, norm) - x).max() < 1e-12
    zi = rng.integers(-1000, 1000, (2, 1 << m))
    assert np.array_equal(O.haar_inverse(zi, m, np.int64, "none"), zi @ O.haar_matrix(m, normalised=False))


@pytest.mark.parametrize("m", range(0, 9))
def test_haar_walsh_is_eq4(m):
    rng = np.random.default_rng(300 + m)
    z = rng.standard_normal((3, 1 << m))
    blk = O.haar_walsh_blockdiag(m)
    for norm in ("per_level", "end"):
        y = O.haar_walsh(z, m, np.float64, norm)
        assert np.abs(y - z @ blk.T).max() < 1e-12, norm
        # and H_m Psi_m^T z through the definitions
        assert np.abs(y - z @ O.haar_matrix(m) @ O.hadamard_dyadic(m).T).max() < 1e-12


@pytest.mark.parametrize("m", range(0, 9))
def test_haar_walsh_unit_vectors_unnormalised(m):
    n = 1 << m
    eye = np.eye(n, dtype=np.int64)
    y = O.haar_walsh(eye, m, np.int64, "none")  # row p = image of e_p
    assert y[0, 0] == 1 and np.count_nonzero(y[0]) == 1
    for k, start, length in _haar_blocks(m):
        hk = O.hadamard_dyadic(k, normalised=False)
        for j in range(length):
            col = np.zeros(n, dtype=np.int64)
            col[start: start + length] = hk[:, j]
            assert np.array_equal(y[start + j], col), (k, j)


@pytest.mark.parametrize("m", [1, 2, 5, 8, 11, 12])
def test_haar_then_haar_walsh_is_the_cascade_bitwise(m):
    rng = np.random.default_rng(400 + m)
    x32 = rng.standard_normal((4, 1 << m)).astype(np.float32)
    for norm in ("per_level", "none"):
        z = O.haar_forward(x32, m, np.float32, norm)
        y = O.haar_walsh(z, m, np.float32, norm)
        ref = O.chw_cascade(x32, m, np.float32, norm)
        assert np.array_equal(y.view(np.uint32), ref.view(np.uint32)), norm
    xi = rng.integers(-(1 << 12), 1 << 12, (3, 1 << m)).astype(np.int32)
    zi = O.haar_forward(xi, m, np.int32, "none")
    assert np.array_equal(O.haar_walsh(zi, m, np.int32, "none"), O.chw_cascade(xi, m, np.int32, "none"))


def test_end_mode_scales_are_single_roundings():
    # END: one multiply by fp32(2^{-L/2}) per coefficient after unscaled butterflies
    rng = np.random.default_rng(7)
    m = 6
    x = rng.standard_normal((2, 1 << m)).astype(np.float32)
    z = O.haar_forward(x, m, np.float32, "end")
    raw = O.haar_forward(x, m, np.float32, "none")
    lev = O.haar_levels(m)
    for p in range(1 << m):
        s = np.float32(2.0 ** (-lev[p] / 2.0))
        assert np.array_equal(z[:, p].view(np.uint32), (raw[:, p] * s).astype(np.float32).view(np.uint32))
    w = O.haar_inverse(z, m, np.float32, "end")
    assert np.abs(w - x).max() < 1e-5


def test_eq4_mutation_is_caught():
    # a Haar-Walsh that forgot the last stage no longer matches eq. (4)
    m = 5
    z = np.eye(1 << m)
    y = O.haar_walsh(z, m, np.float64, "per_level")
    blk = O.haar_walsh_blockdiag(m)
    c = O.inv_sqrt2(np.float64)
    bad = np.array(z, copy=True)
    for r in range(1, m - 1):
        half = 1 << (m - r)
        v = bad.reshape(bad.shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., half:] = O.haar_analysis(v[..., half:], c)
        bad = v.reshape(bad.shape)
    assert np.abs(y - blk.T).max() < 1e-12
    assert np.abs(bad - blk.T).max() > 0.1
