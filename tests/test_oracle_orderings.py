"""Pins of the oracle's output orderings (no GPU).

Natural order is pinned to the Sylvester recursion, sequency order to its definition (rows
sorted by sign changes, each count 0..n-1 appearing once), and both permutations to
those dense matrices; the ordered matrices are symmetric (so their adjoints are
themselves).
"""

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("m", range(0, 10))
def test_natural_matrix_is_row_permuted_dyadic(m):
    nat = O.hadamard_natural(m)
    dy = O.hadamard_dyadic(m)
    perm = O.order_permutation(m, "natural")
    assert np.abs(nat - dy[perm]).max() < 1e-13
    assert np.array_equal(O.hadamard_natural(m, False), O.hadamard_dyadic(m, False)[perm])
    assert np.array_equal(nat, nat.T)
    n = 1 << m
    assert np.abs(nat @ nat - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("m", range(0, 10))
def test_sequency_matrix_definition(m):
    seq = O.walsh_sequency_matrix(m, normalised=False)
    counts = [O.sign_changes(r) for r in seq]
    assert counts == list(range(1 << m))  # each number of sign changes exactly once
    perm = O.order_permutation(m, "sequency")
    assert np.array_equal(seq, O.hadamard_dyadic(m, False)[perm])
    assert np.array_equal(seq, seq.T)


@pytest.mark.parametrize("m", [0, 1, 5, 11])
def test_natural_permutation_is_bitrev(m):
    perm = O.order_permutation(m, "natural")
    assert [int(v) for v in perm] == [O.bitrev(k, m) for k in range(1 << m)]


def test_small_cases_by_hand():
    # m = 2: dyadic rows [1,1,1,1], [1,1,-1,-1], [1,-1,1,-1], [1,-1,-1,1] (eq. (1));
    # natural swaps the middle two, sequency orders by 0,1,2,3 sign changes
    assert O.order_permutation(2, "natural").tolist() == [0, 2, 1, 3]
    assert O.order_permutation(2, "sequency").tolist() == [0, 1, 3, 2]
    assert O.hadamard_natural(2, False).tolist() == [[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]]


@pytest.mark.parametrize("m", [1, 3, 6, 9])
@pytest.mark.parametrize("order", ["natural", "sequency"])
def test_wht_ordered_against_dense(m, order):
    rng = np.random.default_rng(500 + m)
    x = rng.standard_normal((3, 1 << m))
    mat = O.hadamard_natural(m) if order == "natural" else O.walsh_sequency_matrix(m)
    for norm in ("per_level", "end"):
        y = O.wht_ordered(x, m, order, np.float64, norm)
        assert np.abs(y - x @ mat.T).max() < 1e-12
    xi = rng.integers(-100, 100, (2, 1 << m))
    mati = O.hadamard_natural(m, False) if order == "natural" else O.walsh_sequency_matrix(m, False)
    assert np.array_equal(O.wht_ordered(xi, m, order, np.int64, "none"), xi @ mati.T)
