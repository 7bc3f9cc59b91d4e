"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case replaces one oracle function with a plausibly wrong variant (dropped
term, wrong sign, wrong index/half, transposed Kronecker operand, missing reorder)
and checks that the pin checks below fail for it.  The mistakes are planted in
the oracle, never in the CUDA path.
"""

import numpy as np
import pytest

import oracle.definitions as D
import oracle.transforms as T
from conftest import load_golden_matrices, load_golden_table


def pin_checks():
    """A compact run of the oracle pins; returns the names of the pins that fail."""
    failed = []
    h3 = load_golden_matrices("hadamard_unnormalised.txt")["H3"]
    psi3 = load_golden_matrices("haar_unnormalised.txt")["Psi3"]
    try:
        if not np.array_equal(D.hadamard_dyadic(3, normalised=False), h3):
            failed.append("golden H3")
        if not np.array_equal(D.haar_matrix(3, normalised=False), psi3):
            failed.append("golden Psi3")
        for m in range(1, 7):
            if not np.array_equal(D.cascade_product(m, normalised=False), D.hadamard_dyadic(m, normalised=False)):
                failed.append("Theorem 1")
                break
        n = 8
        eye = np.eye(n, dtype=np.int64)
        if not np.array_equal(T.chw_cascade(eye, 3, np.int64, "none"), h3.T):
            failed.append("cascade vs golden H3")
        if not np.array_equal(T.wht_fast_dyadic(eye, 3, normalised=False), h3.T):
            failed.append("fast WHT vs golden H3")
        rng = np.random.default_rng(0)
        x = rng.standard_normal((2, 1 << 6))
        if np.abs(T.wht_fast_dyadic(x, 6) - T.chw_cascade(x, 6)).max() > 1e-12:
            failed.append("O2 vs O4")
        for m, haar_ops, chw_ops in load_golden_table("op_counts.txt")[:6]:
            c = T.OpCounter()
            T.chw_cascade(np.zeros(1 << m), int(m), counter=c)
            if c.adds != chw_ops:
                failed.append("Theorem 2 count")
                break
        y = rng.standard_normal((2, 1 << 5))
        if np.abs(T.chw_reverse_cascade(y, 5) - y @ D.hadamard_dyadic(5)).max() > 1e-12:
            failed.append("reverse cascade transpose")
    except Exception as e:  # a crash counts as a caught mistake
        failed.append(f"raised {type(e).__name__}")
    return failed


def test_unmutated_oracle_passes():
    assert pin_checks() == []


def _haar_wrong_sign(v, c=None, counter=None):
    out = np.array(v, copy=True)
    seg = out.shape[-1]
    while seg > 1:
        a = out[..., 0:seg:2].copy()
        b = out[..., 1:seg:2].copy()
        s, d = a + b, b - a  # planted: difference sign flipped
        if c is not None:
            s, d = s * c, d * c
        out[..., : seg // 2], out[..., seg // 2: seg] = s, d
        seg //= 2
    return out


def _haar_one_level_only(v, c=None, counter=None):
    out = np.array(v, copy=True)
    seg = out.shape[-1]
    if seg > 1:  # planted: the recursion on the sums is dropped
        a, b = out[..., 0::2].copy(), out[..., 1::2].copy()
        out[..., : seg // 2], out[..., seg // 2:] = a + b, a - b
    return out


def _cascade_first_halves(x, m, dtype=np.float64, norm="per_level", counter=None):
    dt = np.dtype(dtype)
    y = np.array(x, dtype=dt, copy=True)
    c = T.inv_sqrt2(dt) if norm == "per_level" else None
    if m == 0:
        return y
    y = T.haar_analysis(y, c, counter)
    shape = y.shape
    for r in range(1, m):
        half = 1 << (m - r)
        v = y.reshape(shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., :half] = T.haar_analysis(v[..., :half], c, counter)  # planted: wrong half
        y = v.reshape(shape)
    return y


def _cascade_reversed_stages(x, m, dtype=np.float64, norm="per_level", counter=None):
    dt = np.dtype(dtype)
    y = np.array(x, dtype=dt, copy=True)
    c = T.inv_sqrt2(dt) if norm == "per_level" else None
    if m == 0:
        return y
    y = T.haar_analysis(y, c, counter)
    shape = y.shape
    for r in range(m - 1, 0, -1):  # planted: stage order reversed
        half = 1 << (m - r)
        v = y.reshape(shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., half:] = T.haar_analysis(v[..., half:], c, counter)
        y = v.reshape(shape)
    return y


def _cascade_drop_last_stage(x, m, dtype=np.float64, norm="per_level", counter=None):
    dt = np.dtype(dtype)
    y = np.array(x, dtype=dt, copy=True)
    c = T.inv_sqrt2(dt) if norm == "per_level" else None
    if m == 0:
        return y
    y = T.haar_analysis(y, c, counter)
    shape = y.shape
    for r in range(1, m - 1):  # planted: stage m-1 dropped
        half = 1 << (m - r)
        v = y.reshape(shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., half:] = T.haar_analysis(v[..., half:], c, counter)
        y = v.reshape(shape)
    return y


def _fast_no_reorder(x, m, normalised=True):
    n = 1 << m
    z = np.array(x, dtype=np.float64 if normalised else np.int64).reshape(-1, n)
    h = 1
    while h < n:
        v = z.reshape(z.shape[0], n // (2 * h), 2, h)
        lo, hi = v[:, :, 0, :].copy(), v[:, :, 1, :].copy()
        v[:, :, 0, :], v[:, :, 1, :] = lo + hi, lo - hi
        h *= 2
    return z * (2.0 ** (-m / 2)) if normalised else z  # planted: natural order kept


def _hadamard_transposed_kron(m, normalised=True):
    h = np.ones((1, 1), dtype=np.int64)
    for _ in range(m):  # planted: operands of the Kronecker product swapped
        h = np.vstack([np.kron([[1, 1]], h), np.kron([[1, -1]], h)])
    return h * 2.0 ** (-m / 2) if normalised else h


def _haar_detail_sum(m, normalised=True):
    p = np.ones((1, 1), dtype=np.int64)
    for k in range(m):  # planted: (1 1) instead of (1 -1) in the detail rows
        p = np.vstack([np.kron(p, [[1, 1]]), np.kron(np.eye(2**k, dtype=np.int64), [[1, 1]])])
    return p * 1.0 if normalised else p


def _synthesis_transposed(w, c=None, counter=None):
    out = np.array(w, copy=True)
    n = out.shape[-1]
    seg = 2
    while seg <= n:
        u, d = out[..., : seg // 2].copy(), out[..., seg // 2: seg].copy()
        even, odd = u + d, d - u  # planted: operands of the difference swapped
        if c is not None:
            even, odd = even * c, odd * c
        out[..., 0:seg:2], out[..., 1:seg:2] = even, odd
        seg *= 2
    return out


MUTANTS = [
    ("transforms", "haar_analysis", _haar_wrong_sign),
    ("transforms", "haar_analysis", _haar_one_level_only),
    ("transforms", "chw_cascade", _cascade_first_halves),
    ("transforms", "chw_cascade", _cascade_reversed_stages),
    ("transforms", "chw_cascade", _cascade_drop_last_stage),
    ("transforms", "wht_fast_dyadic", _fast_no_reorder),
    ("definitions", "hadamard_dyadic", _hadamard_transposed_kron),
    ("definitions", "haar_matrix", _haar_detail_sum),
    ("transforms", "haar_synthesis", _synthesis_transposed),
]


@pytest.mark.parametrize("module,name,fn", MUTANTS, ids=[f.__name__ for _, _, f in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, module, name, fn):
    mod = {"transforms": T, "definitions": D}[module]
    monkeypatch.setattr(mod, name, fn)
    if module == "definitions" and name == "hadamard_dyadic":
        monkeypatch.setattr(T, "hadamard_dyadic", fn)
    failed = pin_checks()
    assert failed, f"planted mistake in {module}.{name} ({fn.__name__}) was not caught"
