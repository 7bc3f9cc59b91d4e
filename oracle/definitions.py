"""Matrix definitions of the paper, built literally (test infrastructure only).

Every function builds a dense matrix from the recursion the paper states, so a
reader can hold each line against the equation it cites.  Dense matrices are only
built for small m (m <= 10 or so); they exist to pin the fast oracles.
"""

import numpy as np

_ONE_ONE = np.array([[1, 1]], dtype=np.int64)
_ONE_MINUS_ONE = np.array([[1, -1]], dtype=np.int64)


def hadamard_dyadic(m, normalised=True):
    """H_m, the 2^m x 2^m Hadamard matrix in dyadic (Paley) order, eq. (1).

    H_0 = 1 and H_{m+1} = 2^{-1/2} [ H_m (x) (1 1) ; H_m (x) (1 -1) ], where (x) is
    the Kronecker product.  With ``normalised=False`` the factor 2^{-1/2} is dropped
    at every level, which leaves the +-1 integer matrix 2^{m/2} H_m (int64).
    """
    if m < 0:
        raise ValueError("m must be >= 0")
    if normalised:
        h = np.ones((1, 1), dtype=np.float64)
        scale = 1.0 / np.sqrt(2.0)
        for _ in range(m):
            h = scale * np.vstack([np.kron(h, _ONE_ONE), np.kron(h, _ONE_MINUS_ONE)])
        return h
    h = np.ones((1, 1), dtype=np.int64)
    for _ in range(m):
        h = np.vstack([np.kron(h, _ONE_ONE), np.kron(h, _ONE_MINUS_ONE)])
    return h


def haar_matrix(m, normalised=True):
    """Psi_m, the 2^m x 2^m Haar matrix, eq. (2).

    Psi_0 = 1 and Psi_{m+1} = 2^{-1/2} [ Psi_m (x) (1 1) ; I_m (x) (1 -1) ], where
    I_m is the 2^m x 2^m identity.  ``normalised=False`` drops every 2^{-1/2}
    (int64 result; its rows then have different norms).
    """
    if m < 0:
        raise ValueError("m must be >= 0")
    if normalised:
        p = np.ones((1, 1), dtype=np.float64)
        scale = 1.0 / np.sqrt(2.0)
        for k in range(m):
            eye = np.eye(2**k, dtype=np.float64)
            p = scale * np.vstack([np.kron(p, _ONE_ONE), np.kron(eye, _ONE_MINUS_ONE)])
        return p
    p = np.ones((1, 1), dtype=np.int64)
    for k in range(m):
        eye = np.eye(2**k, dtype=np.int64)
        p = np.vstack([np.kron(p, _ONE_ONE), np.kron(eye, _ONE_MINUS_ONE)])
    return p


def _blockdiag(a, b):
    out = np.zeros((a.shape[0] + b.shape[0], a.shape[1] + b.shape[1]), dtype=np.result_type(a, b))
    out[: a.shape[0], : a.shape[1]] = a
    out[a.shape[0]:, a.shape[1]:] = b
    return out


def cascade_stage_factor(m, r, normalised=True):
    """Stage r of Theorem 1: I_{r-1} (x) [ I_{m-r}  0 ; 0  Psi_{m-r} ], for 1 <= r <= m-1.

    It applies Psi_{m-r} to the second half of each of the 2^{r-1} consecutive blocks
    of length 2^{m-r+1} and leaves the first halves alone (the identity blocks the
    paper says need not be performed).
    """
    if not 1 <= r <= m - 1:
        raise ValueError("stage index r must satisfy 1 <= r <= m-1")
    dt = np.float64 if normalised else np.int64
    inner = _blockdiag(np.eye(2 ** (m - r), dtype=dt), haar_matrix(m - r, normalised))
    return np.kron(np.eye(2 ** (r - 1), dtype=dt), inner)


def cascade_product(m, normalised=True):
    """Right-hand side of Theorem 1 (eq. (3)): { prod_{r=1}^{m-1} F_r } Psi_m.

    The paper's product notation prod_{r=1}^{p} M_r = M_p ... M_2 M_1 puts F_1 next to
    Psi_m, so stage 1 acts first.  Valid for m >= 1.
    """
    if m < 1:
        raise ValueError("Theorem 1 is stated for m >= 1")
    acc = haar_matrix(m, normalised)
    if not normalised:
        # Integer entries stay below 2^m in magnitude, so FP64 products are exact;
        # they are used only because numpy has no fast int64 matmul.
        acc = acc.astype(np.float64)
    for r in range(1, m):
        acc = cascade_stage_factor(m, r, normalised) @ acc
    if not normalised:
        out = np.rint(acc).astype(np.int64)
        assert np.array_equal(out, acc)
        return out
    return acc


def haar_walsh_blockdiag(m):
    """Right-hand side of eq. (4): blockdiag(1, H_0, H_1, ..., H_{m-1}) in FP64.

    eq. (4) states H_m Psi_m^T equals this matrix (the Haar-Walsh transform).
    """
    blocks = [np.ones((1, 1))] + [hadamard_dyadic(k) for k in range(m)]
    out = blocks[0]
    for b in blocks[1:]:
        out = _blockdiag(out, b)
    return out


def bitrev(k, m):
    """Reverse the m low bits of the integer k (plain loop, m >= 0)."""
    out = 0
    for _ in range(m):
        out = (out << 1) | (k & 1)
        k >>= 1
    return out


def hadamard_entry_closed_form(m, k, j):
    """Entry (k, j) of H_m without the 2^{-m/2} factor: (-1)^popcount(bitrev_m(k) & j).

    Derived from eq. (1): the top half of H_{m+1} keeps the sign of H_m and the
    bottom half multiplies column 2j+1 by -1, so the most significant bit of the
    row index pairs with the least significant bit of the column index, and so on
    down the recursion.  Pinned against ``hadamard_dyadic`` for m <= 10.
    """
    return -1 if bin(bitrev(k, m) & j).count("1") & 1 else 1
