"""Natural (Hadamard) and sequency (Walsh) orderings of the transform (test infrastructure only).

The paper's H_m lists the Walsh functions in dyadic (Paley) order (eq. (1)); the same
functions are also commonly listed in natural order (the Sylvester recursion) and in
sequency order (by number of sign changes).  The CHW computation is the same in every
order -- only the position each result is stored at changes -- so the ordered outputs
are the cascade's outputs permuted.

``hadamard_natural``       the Sylvester matrix: S_0 = 1, S_{k+1} = [S_k S_k; S_k -S_k]
                           (times 2^{-1/2} per level when normalised).
``walsh_sequency_matrix``  the rows of the natural matrix sorted by their number of sign
                           changes (the definition of sequency order; row s has s changes).
``order_permutation``      perm with y_order[k] = y_dyadic[perm[k]]: identity (dyadic),
                           bitrev_m(k) (natural), k ^ (k >> 1) (sequency, the Gray code).
``wht_ordered``            the CHW cascade (any dtype and normalisation) stored in an order.

Parity pinned for: all (tests/test_oracle_orderings.py: the permutations against the dense
matrices built from their definitions, the sign-change count, symmetry).
"""

import numpy as np

from .transforms import chw_cascade

ORDERS = ("dyadic", "natural", "sequency")


def hadamard_natural(m, normalised=True):
    """The 2^m x 2^m Sylvester-Hadamard matrix (natural order), FP64 or int64."""
    s = np.ones((1, 1), dtype=np.float64 if normalised else np.int64)
    c = 1.0 / np.sqrt(2.0)
    for _ in range(m):
        s = np.block([[s, s], [s, -s]])
        if normalised:
            s = s * c
    return s


def sign_changes(row):
    """Number of sign changes between consecutive entries of a +-1 (scaled) row."""
    r = np.sign(np.asarray(row))
    return int(np.count_nonzero(r[1:] != r[:-1]))


def walsh_sequency_matrix(m, normalised=True):
    """Rows of the natural matrix reordered by increasing number of sign changes."""
    nat = hadamard_natural(m, normalised)
    counts = [sign_changes(r) for r in nat]
    order = np.argsort(counts, kind="stable")
    return nat[order]


def order_permutation(m, order):
    """perm (int64, length 2^m) with y_order[k] = y_dyadic[perm[k]]."""
    if order not in ORDERS:
        raise ValueError(f"order must be one of {ORDERS}")
    k = np.arange(1 << m, dtype=np.int64)
    if order == "dyadic":
        return k
    if order == "natural":
        # bitrev_m for every k at once: bit b of k moves to bit m-1-b
        r = np.zeros_like(k)
        for b in range(m):
            r |= ((k >> b) & 1) << (m - 1 - b)
        return r
    return k ^ (k >> 1)


def wht_ordered(x, m, order, dtype=np.float64, norm="per_level"):
    """The CHW cascade's result (Theorem 1, in ``dtype`` with ``norm``) stored in ``order``."""
    y = chw_cascade(x, m, dtype, norm)
    return y[..., order_permutation(m, order)]
