"""Pins of the oracle's error norm, oracle.rel_err_per_signal (CPU only).

Every floating-point gate of the GPU tests, the smoke check and the benchmark's error
fields goes through this function: the per-signal normwise relative error
||y - y_ref||_2 / ||y_ref||_2 in FP64, with the absolute norm ||y|| where the reference is
zero.  The expected values below are worked out by hand from that definition (Pythagorean
triples and quadruples, so every norm is an exact integer), not by calling the function.
The planted mistakes at the end (a dropped square root, the wrong denominator, another
norm, a lost row, a zero result) each fail at least one of these pins.
"""

import numpy as np
import pytest

import oracle.errors as E

# (y, y_ref, expected) worked by hand
CASES = [
    # ||(3,4) - 0|| = 5 with a zero reference: the absolute norm
    ([3.0, 4.0], [0.0, 0.0], 5.0),
    # diff (0, 1), ||ref|| = 1
    ([1.0, 1.0], [1.0, 0.0], 1.0),
    # diff (3, 4) -> 5, ||(6, 8)|| = 10; no sqrt would give 25/100, ||y|| = 15 would give 1/3
    ([9.0, 12.0], [6.0, 8.0], 0.5),
    # diff (1, 2, 2) -> 3, ||(2, 3, 6)|| = 7; max norm would give 2/6, 1-norm 5/11
    ([3.0, 5.0, 8.0], [2.0, 3.0, 6.0], 3.0 / 7.0),
    # equal vectors
    ([-1.5, 2.25, 0.0, 7.0], [-1.5, 2.25, 0.0, 7.0], 0.0),
    # both zero
    ([0.0, 0.0], [0.0, 0.0], 0.0),
    # y = -y_ref: diff = 2 y_ref, ratio exactly 2
    ([-2.0, -3.0, -6.0], [2.0, 3.0, 6.0], 2.0),
]


@pytest.mark.parametrize("y,ref,expected", CASES)
def test_hand_values(y, ref, expected):
    got = E.rel_err_per_signal(np.array(y), np.array(ref))
    assert got.shape == (1,)
    assert got[0] == pytest.approx(expected, rel=1e-15, abs=0)


def test_rows_are_independent_and_leading_axes_flatten():
    y = np.array([[9.0, 12.0], [3.0, 4.0], [1.0, 1.0]])
    ref = np.array([[6.0, 8.0], [0.0, 0.0], [1.0, 0.0]])
    got = E.rel_err_per_signal(y, ref)
    assert got.tolist() == [0.5, 5.0, 1.0]
    # any leading shape is a batch of signals along the last axis
    got3 = E.rel_err_per_signal(y.reshape(3, 1, 2), ref.reshape(3, 1, 2))
    assert got3.tolist() == [0.5, 5.0, 1.0]


def test_fp64_accumulation_of_fp32_inputs():
    # 2^13 entries of 1 against 2^13 entries of 1 + 2^-12: a float32 sum of squares of the
    # differences would still be exact here, but the reference norm of (1 + 2^-12) over
    # 2^13 entries needs more than fp32's 24 bits; the result must equal the FP64 value.
    n = 1 << 13
    y = np.ones(n, dtype=np.float32)
    ref = np.full(n, 1.0 + 2.0**-12, dtype=np.float32)
    want = 2.0**-12 / (1.0 + 2.0**-12)  # ||d|| = sqrt(n) 2^-12, ||ref|| = sqrt(n) (1 + 2^-12)
    assert E.rel_err_per_signal(y, ref)[0] == pytest.approx(want, rel=1e-13)


def test_scale_invariance_by_powers_of_two():
    rng = np.random.default_rng(3)
    y, ref = rng.standard_normal((4, 64)), rng.standard_normal((4, 64))
    base = E.rel_err_per_signal(y, ref)
    for k in (-40, -3, 5, 60):
        assert np.array_equal(E.rel_err_per_signal(y * 2.0**k, ref * 2.0**k), base)


def error_pin_failures():
    """The pins above as one check; returns the names of those that fail (for mutations)."""
    failed = []
    try:
        for i, (y, ref, expected) in enumerate(CASES):
            got = E.rel_err_per_signal(np.array(y), np.array(ref))
            if got.shape != (1,) or abs(float(got[0]) - expected) > 1e-15 * max(1.0, expected):
                failed.append(f"hand value {i}")
        got = E.rel_err_per_signal(np.array([[9.0, 12.0], [3.0, 4.0]]), np.array([[6.0, 8.0], [0.0, 0.0]]))
        if np.asarray(got).tolist() != [0.5, 5.0]:
            failed.append("per-row")
    except Exception as e:  # a crash counts as a caught mistake
        failed.append(f"raised {type(e).__name__}")
    return failed


def _no_sqrt(y, y_ref):
    a = np.asarray(y, dtype=np.float64).reshape(-1, np.shape(y)[-1])
    b = np.asarray(y_ref, dtype=np.float64).reshape(-1, np.shape(y_ref)[-1])
    num, den = np.sum((a - b) ** 2, axis=1), np.sum(b**2, axis=1)  # planted: squares
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def _wrong_denominator(y, y_ref):
    a = np.asarray(y, dtype=np.float64).reshape(-1, np.shape(y)[-1])
    b = np.asarray(y_ref, dtype=np.float64).reshape(-1, np.shape(y_ref)[-1])
    num, den = np.linalg.norm(a - b, axis=1), np.linalg.norm(a, axis=1)  # planted: ||y||
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def _max_norm(y, y_ref):
    a = np.asarray(y, dtype=np.float64).reshape(-1, np.shape(y)[-1])
    b = np.asarray(y_ref, dtype=np.float64).reshape(-1, np.shape(y_ref)[-1])
    num, den = np.abs(a - b).max(axis=1), np.abs(b).max(axis=1)  # planted: infinity norm
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def _pooled(y, y_ref):
    a = np.asarray(y, dtype=np.float64).reshape(-1, np.shape(y)[-1])
    b = np.asarray(y_ref, dtype=np.float64).reshape(-1, np.shape(y_ref)[-1])
    r = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)  # planted: one number for the batch
    return np.full(a.shape[0], r)


def _zero_ref_gives_zero(y, y_ref):
    a = np.asarray(y, dtype=np.float64).reshape(-1, np.shape(y)[-1])
    b = np.asarray(y_ref, dtype=np.float64).reshape(-1, np.shape(y_ref)[-1])
    num, den = np.linalg.norm(a - b, axis=1), np.linalg.norm(b, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)  # planted: hides ||y||


def _always_zero(y, y_ref):
    return np.zeros(np.asarray(y).reshape(-1, np.shape(y)[-1]).shape[0])  # planted


ERROR_MUTANTS = [_no_sqrt, _wrong_denominator, _max_norm, _pooled, _zero_ref_gives_zero, _always_zero]


def test_unmutated_error_norm_passes():
    assert error_pin_failures() == []


@pytest.mark.parametrize("fn", ERROR_MUTANTS, ids=[f.__name__ for f in ERROR_MUTANTS])
def test_planted_error_norm_mistake_is_caught(monkeypatch, fn):
    monkeypatch.setattr(E, "rel_err_per_signal", fn)
    assert error_pin_failures(), f"planted mistake {fn.__name__} in the error norm was not caught"
