"""The transform y = H_m x, computed plainly on the CPU (test infrastructure only).

Four independent routes, none sharing code with the CUDA path:

O1 ``wht_dense``         dense H_m from eq. (1), then a matvec (FP64 or int64).
O2 ``wht_fast_dyadic``   textbook natural-order fast WHT (stride-doubling butterflies)
                         followed by the bit-reversal reorder that turns natural order
                         into dyadic order, then the 2^{-m/2} scale.
O3 ``wht_closed_form``   selected outputs one at a time from the closed form
                         H_m[k][j] = 2^{-m/2} (-1)^popcount(bitrev_m(k) & j).
O4 ``chw_cascade``       the CHW algorithm itself, Theorem 1 taken literally in stage
                         order: Psi_m (eq. (2)), then for r = 1..m-1 Psi_{m-r} on the
                         second half of every block of length 2^{m-r+1}.  Runs in any
                         numpy dtype (FP64, fp32, int32 with two's-complement wrap),
                         so its fp32 result shows what IEEE single precision gives for
                         this exact order of operations.  An ``OpCounter`` counts the
                         additions and subtractions (Lemma 1, Theorem 2).

``chw_reverse_cascade`` is the transpose of O4: the stages in reverse order, each
replaced by its inverse Haar transform Psi^T (the synthesis butterflies).

Normalisation modes (eq. (1)-(2) put 2^{-1/2} in every recursion level; the paper
counts additions only and does not place the scalings):
  "per_level"  every butterfly output is multiplied by c = 1/sqrt2 rounded to the
               working precision: (a+b)*c and (a-b)*c;
  "end"        unscaled butterflies, then one multiply by 2^{-m/2} rounded to the
               working precision;
  "none"       unscaled butterflies: the result is 2^{m/2} H_m x (exact for ints).
"""

import numpy as np

from .definitions import hadamard_dyadic

NORMS = ("per_level", "end", "none")


class OpCounter:
    """Counts scalar additions/subtractions performed by the Haar butterflies."""

    def __init__(self):
        self.adds = 0
        self.per_call = []

    def add(self, k):
        self.adds += k


def inv_sqrt2(dtype):
    """1/sqrt2 rounded to ``dtype`` (round to nearest even, via the FP64 value)."""
    return np.dtype(dtype).type(1.0 / np.sqrt(2.0))


def end_scale_f32(m):
    """2^{-m/2} rounded once to fp32 from its FP64 value."""
    return np.float32(2.0 ** (-m / 2.0))


def _end_scale(m, dtype):
    return np.dtype(dtype).type(2.0 ** (-m / 2.0))


def _as_batch(x, m):
    a = np.asarray(x)
    n = 1 << m
    if a.shape[-1] != n:
        raise ValueError(f"last axis must have length 2^m = {n}, got {a.shape[-1]}")
    return a


# ---------------------------------------------------------------- O1, O2, O3
def wht_dense(x, m, normalised=True):
    """O1: y = H_m x with the dense matrix of eq. (1).  x has shape (..., 2^m)."""
    a = _as_batch(x, m)
    if normalised:
        h = hadamard_dyadic(m, normalised=True)
        return np.asarray(a, dtype=np.float64) @ h.T
    h = hadamard_dyadic(m, normalised=False)
    return np.asarray(a, dtype=np.int64) @ h.T


def bitrev_permutation(m):
    """perm[k] = bitrev_m(k) for k = 0..2^m-1, built bit by bit."""
    idx = np.arange(1 << m, dtype=np.int64)
    rev = np.zeros_like(idx)
    for b in range(m):
        rev |= ((idx >> b) & 1) << (m - 1 - b)
    return rev


def wht_fast_dyadic(x, m, normalised=True):
    """O2: textbook natural-order fast WHT, then reorder natural -> dyadic.

    The natural-order transform z[k] = sum_j (-1)^popcount(k & j) x[j] is computed
    by the classic in-place butterflies (a, b) -> (a+b, a-b) on pairs at distance
    h = 1, 2, 4, ... .  Dyadic order is y[k] = z[bitrev_m(k)] (the closed form of
    eq. (1)).  FP64 when ``normalised`` (times 2^{-m/2}), else exact int64.
    """
    a = _as_batch(x, m)
    n = 1 << m
    lead = a.shape[:-1]
    z = np.array(a, dtype=np.float64 if normalised else np.int64).reshape(-1, n)
    rows = z.shape[0]
    h = 1
    while h < n:
        v = z.reshape(rows, n // (2 * h), 2, h)
        lo = v[:, :, 0, :].copy()
        hi = v[:, :, 1, :].copy()
        v[:, :, 0, :] = lo + hi
        v[:, :, 1, :] = lo - hi
        h *= 2
    y = z[:, bitrev_permutation(m)]
    if normalised:
        y = y * (2.0 ** (-m / 2.0))
    return y.reshape(lead + (n,))


def wht_closed_form(x, m, ks, normalised=True):
    """O3: outputs y[k] for the indices ``ks`` from the closed form, one at a time.

    x has shape (2^m,) (one signal).  Each output is an O(n) signed sum.
    """
    a = _as_batch(x, m)
    if a.ndim != 1:
        raise ValueError("wht_closed_form takes one signal")
    n = 1 << m
    j = np.arange(n, dtype=np.uint64)
    perm_bits = bitrev_permutation(m)
    xs = np.asarray(a, dtype=np.float64 if normalised else np.int64)
    out = []
    for k in ks:
        rk = np.uint64(perm_bits[k])
        signs = 1 - 2 * (np.bitwise_count(j & rk).astype(np.int64) & 1)
        s = np.dot(signs, xs)
        out.append(s * (2.0 ** (-m / 2.0)) if normalised else s)
    return np.array(out)


def wht_sparse_closed_form(js, cs, m, ks, normalised=True):
    """O3 for a sparse input: outputs y[k], k in ``ks``, of y = H_m x where x has the value
    cs[i] at position js[i] and zeros elsewhere, from the closed form of eq. (1)'s entries,
    H_m[k][j] = 2^{-m/2} (-1)^popcount(bitrev_m(k) & j), vectorised over the outputs.

    With integer ``cs`` and normalised=False the result is the exact int64 sum
    sum_i cs[i] (-1)^popcount(bitrev_m(k) & js[i]) (the unnormalised transform).  Cost is
    O(len(js) * len(ks)), so very long signals can be checked at sampled outputs.
    """
    k = np.asarray(ks, dtype=np.uint64)
    rk = np.zeros_like(k)
    for b in range(m):  # bitrev_m(k), bit by bit
        rk |= ((k >> np.uint64(b)) & np.uint64(1)) << np.uint64(m - 1 - b)
    out = np.zeros(k.shape, dtype=np.int64 if not normalised else np.float64)
    for j, c in zip(js, cs):
        sign = 1 - 2 * (np.bitwise_count(rk & np.uint64(j)).astype(np.int64) & 1)
        out += sign * (c if not normalised else float(c))
    return out * (2.0 ** (-m / 2.0)) if normalised else out


# ---------------------------------------------------------------- O4: the CHW cascade
def haar_analysis(v, c=None, counter=None):
    """Psi_L v along the last axis (eq. (2)); length 2^L.

    Psi_{L} = c [ Psi_{L-1} (x) (1 1) ; I (x) (1 -1) ]: one level forms the pair sums
    s_i = (v_{2i} + v_{2i+1}) c and differences d_i = (v_{2i} - v_{2i+1}) c of the
    current approximation segment, keeps the differences in the segment's second
    half and recurses on the sums in its first half.  ``c=None`` leaves the
    butterflies unscaled.
    """
    out = np.array(v, copy=True)
    seg = out.shape[-1]
    while seg > 1:
        a = out[..., 0:seg:2].copy()
        b = out[..., 1:seg:2].copy()
        s = a + b
        d = a - b
        if c is not None:
            s = s * c
            d = d * c
        out[..., : seg // 2] = s
        out[..., seg // 2: seg] = d
        if counter is not None:
            counter.add(seg * int(np.prod(out.shape[:-1], dtype=np.int64)))
        seg //= 2
    return out


def haar_synthesis(w, c=None, counter=None):
    """Psi_L^T w along the last axis: the inverse Haar transform, coarse to fine.

    Transposing one level of eq. (2) gives v_{2i} = (u_i + d_i) c and
    v_{2i+1} = (u_i - d_i) c, where u is the already-synthesised approximation of
    half the length and d the details stored in the segment's second half.
    """
    out = np.array(w, copy=True)
    n = out.shape[-1]
    seg = 2
    while seg <= n:
        u = out[..., : seg // 2].copy()
        d = out[..., seg // 2: seg].copy()
        even = u + d
        odd = u - d
        if c is not None:
            even = even * c
            odd = odd * c
        out[..., 0:seg:2] = even
        out[..., 1:seg:2] = odd
        if counter is not None:
            counter.add(seg * int(np.prod(out.shape[:-1], dtype=np.int64)))
        seg *= 2
    return out


def _check_mode(dtype, norm):
    if norm not in NORMS:
        raise ValueError(f"norm must be one of {NORMS}")
    if np.issubdtype(np.dtype(dtype), np.integer) and norm != "none":
        raise ValueError("integer cascades are unnormalised (norm='none')")


def chw_cascade(x, m, dtype=np.float64, norm="per_level", counter=None):
    """O4: the CHW algorithm of Theorem 1 in stage order, in ``dtype``.

    Stage 0 is the full Haar transform Psi_m.  Stage r (r = 1..m-1) is
    I_{r-1} (x) diag(I_{m-r}, Psi_{m-r}): Psi_{m-r} on the second half of each of the
    2^{r-1} blocks of length 2^{m-r+1}; first halves are left alone.  The product
    notation of Theorem 1 applies stage 1 first.  m = 0 is the identity (H_0 = 1).
    """
    _check_mode(dtype, norm)
    a = _as_batch(x, m)
    dt = np.dtype(dtype)
    y = np.array(a, dtype=dt, copy=True)
    c = inv_sqrt2(dt) if norm == "per_level" else None
    if m == 0:
        return y
    y = haar_analysis(y, c, counter)
    shape = y.shape
    for r in range(1, m):
        half = 1 << (m - r)
        v = y.reshape(shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., half:] = haar_analysis(v[..., half:], c, counter)
        y = v.reshape(shape)
    if norm == "end":
        y = y * _end_scale(m, dt)
    return y


def chw_reverse_cascade(y, m, dtype=np.float64, norm="per_level", counter=None):
    """Transpose of ``chw_cascade``: H_m^T y = Psi_m^T F_1^T ... F_{m-1}^T y.

    Stage m-1 is undone first: Psi_{m-r}^T on the second half of each block, for
    r = m-1 down to 1, then the full inverse Haar transform Psi_m^T.  In "end" mode
    the single 2^{-m/2} multiply is applied last, as in the forward cascade.
    """
    _check_mode(dtype, norm)
    a = _as_batch(y, m)
    dt = np.dtype(dtype)
    x = np.array(a, dtype=dt, copy=True)
    c = inv_sqrt2(dt) if norm == "per_level" else None
    if m == 0:
        return x
    shape = x.shape
    for r in range(m - 1, 0, -1):
        half = 1 << (m - r)
        v = x.reshape(shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., half:] = haar_synthesis(v[..., half:], c, counter)
        x = v.reshape(shape)
    x = haar_synthesis(x, c, counter)
    if norm == "end":
        x = x * _end_scale(m, dt)
    return x
