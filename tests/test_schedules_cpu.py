"""The schedules the kernels use round exactly like the cascade of Theorem 1 (CPU).

The kernels do not run the cascade stage by stage.  They give every element a label (its
index in the input) and, for t = 0..m-1, apply one butterfly (a, b) -> ((a+b)c, (a-b)c) to
every pair of labels that differ in bit t, then store label L at dyadic position
bitrev_m(L).  The two-pass tier does the same in two sweeps: label bits 0..b-1 on the rows
of the 2^a x 2^b matrix X of a signal, then bits b..m-1 on the columns of X^T, giving
Y = H_b X^T H_a.  Every value meets bits 0, 1, ..., m-1 in that order, so each schedule
performs the same additions on the same operands as the stages of Theorem 1, and rounds
identically.  These tests check that claim against the oracle's stage-by-stage cascade,
bit for bit in fp32 (per-level scaling and unscaled) and int32, and check that the order
matters: the same butterflies in the reversed bit order give the same exact result but
different fp32 roundings.
"""

import numpy as np
import pytest

import oracle as O


def _bitrev(m):
    perm = np.zeros(1 << m, dtype=np.int64)
    for k in range(1 << m):
        r = 0
        for i in range(m):
            r |= ((k >> i) & 1) << (m - 1 - i)
        perm[k] = r
    return perm


def label_bit_schedule(x, m, dtype, c, bits=None):
    """Butterflies on label bits in the order `bits` (default 0..m-1) over the last axis,
    then the dyadic store y[..., bitrev_m(L)] = v[..., L]."""
    v = np.array(x, dtype=dtype, copy=True)
    lead = v.shape[:-1]
    for t in (range(m) if bits is None else bits):
        w = v.reshape(lead + (1 << (m - 1 - t), 2, 1 << t))
        a, b = w[..., 0, :].copy(), w[..., 1, :].copy()
        s, d = a + b, a - b
        if c is not None:
            s, d = s * c, d * c
        w[..., 0, :], w[..., 1, :] = s, d
        v = w.reshape(lead + (1 << m,))
    y = np.empty_like(v)
    y[..., _bitrev(m)] = v
    return y


def two_pass_split(x, m, a, dtype, c):
    """Y = H_b X^T H_a: label bits 0..b-1 on the rows of X (2^a x 2^b), then bits b..m-1 on
    the rows of the transposed intermediate; y is Y read row by row."""
    b = m - a
    lead = x.shape[:-1]
    rows = label_bit_schedule(np.asarray(x, dtype=dtype).reshape(lead + (1 << a, 1 << b)), b, dtype, c)
    cols = np.swapaxes(rows, -1, -2).copy()
    return label_bit_schedule(cols, a, dtype, c).reshape(lead + (1 << m,))


@pytest.mark.parametrize("m", list(range(1, 13)))
@pytest.mark.parametrize("norm", ["per_level", "none"])
def test_label_bit_schedule_rounds_like_the_cascade(m, norm):
    x = np.random.default_rng(100 + m).standard_normal((3, 1 << m)).astype(np.float32)
    c = O.inv_sqrt2(np.float32) if norm == "per_level" else None
    got = label_bit_schedule(x, m, np.float32, c)
    want = O.chw_cascade(x, m, np.float32, norm)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("m", [1, 5, 9, 12])
def test_label_bit_schedule_int32_wraps_like_the_cascade(m):
    x = np.random.default_rng(7 + m).integers(-(2**31), 2**31, size=(2, 1 << m), dtype=np.int64).astype(np.int32)
    with np.errstate(over="ignore"):
        got = label_bit_schedule(x, m, np.int32, None)
        want = O.chw_cascade(x, m, np.int32, "none")
    assert np.array_equal(got, want)


@pytest.mark.parametrize("m,a", [(2, 1), (7, 3), (10, 5), (12, 4), (12, 9), (13, 6)])
@pytest.mark.parametrize("norm", ["per_level", "none"])
def test_two_pass_split_rounds_like_the_cascade(m, a, norm):
    x = np.random.default_rng(200 + m + a).standard_normal((2, 1 << m)).astype(np.float32)
    c = O.inv_sqrt2(np.float32) if norm == "per_level" else None
    got = two_pass_split(x, m, a, np.float32, c)
    want = O.chw_cascade(x, m, np.float32, norm)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_the_bit_order_matters_in_fp32_only():
    m = 10
    x = np.random.default_rng(5).standard_normal((4, 1 << m))
    reverse = list(range(m - 1, -1, -1))
    # exact arithmetic (integers, unscaled): the butterflies of different bits commute
    xi = np.rint(x * 1000).astype(np.int64)
    assert np.array_equal(label_bit_schedule(xi, m, np.int64, None, reverse), label_bit_schedule(xi, m, np.int64, None))
    # fp32: the reversed order rounds differently from the cascade
    xf = x.astype(np.float32)
    c = O.inv_sqrt2(np.float32)
    rev = label_bit_schedule(xf, m, np.float32, c, reverse)
    want = O.chw_cascade(xf, m, np.float32, "per_level")
    assert not np.array_equal(rev.view(np.uint32), want.view(np.uint32))
    assert np.max(np.abs(rev.astype(np.float64) - want)) < 1e-5 * np.max(np.abs(want))
