"""The Haar wavelet transform and the Haar-Walsh transform (test infrastructure only).

Three operators around the CHW factorisation, each computed plainly on the CPU:

``haar_forward``   z = Psi_m x, the orthonormal Haar wavelet transform of eq. (2),
                   with its output in the layout eq. (2) produces:
                   z = [a, d_m, d_{m-1} (2 values), ..., d_1 (2^{m-1} values)], where
                   d_l holds the level-l details (2^{m-l} values at positions
                   [2^{m-l}, 2^{m-l+1})) and a the final approximation.
``haar_inverse``   x = Psi_m^T z, the synthesis butterflies from coarse to fine.
``haar_walsh``     y = H_m Psi_m^T z: stages r = 1..m-1 of Theorem 1 applied to Haar
                   coefficients z.  By eq. (4) this is block diagonal,
                   diag(1, H_0, H_1, ..., H_{m-1}), acting on the Haar scales.

Normalisation modes (the same names as the Walsh-Hadamard cascade):
  "per_level"  every butterfly output times c = 1/sqrt2 in the working precision;
  "none"       unscaled butterflies (unnormalised Psi', exact for integers);
  "end"        unscaled butterflies with a single multiply per element by 2^{-L/2}
               rounded to the working precision, where L is the number of butterfly
               levels that give the element its scale:
                 haar_forward: after the butterflies, coefficient p is multiplied by
                   2^{-L(p)/2}, L(p) = the level of its detail (m for a);
                 haar_inverse: before the butterflies, coefficient p is multiplied by
                   2^{-L(p)/2} (the transpose applies the same diagonal first);
                 haar_walsh: after the unscaled stages, the block of scale k (positions
                   [2^k, 2^{k+1})) is multiplied by 2^{-k/2}; positions 0 and 1 keep
                   their value (H_0 = 1).
Nothing here imports or is imported by the CUDA path.

Parity pinned for: all three (tests/test_oracle_wavelets.py: the dense matrices of eq. (2)
and eq. (4) in FP64, orthogonality, bitwise agreement of haar_walsh o haar_forward with
the literal cascade, and unit-vector columns).
"""

import numpy as np

from .transforms import NORMS, haar_analysis, haar_synthesis, inv_sqrt2


def _check(dtype, norm):
    if norm not in NORMS:
        raise ValueError(f"norm must be one of {NORMS}")
    if np.issubdtype(np.dtype(dtype), np.integer) and norm != "none":
        raise ValueError("integer transforms are unnormalised (norm='none')")


def _last_axis(x, m):
    a = np.asarray(x)
    if a.shape[-1] != (1 << m):
        raise ValueError(f"last axis must have length 2^m = {1 << m}, got {a.shape[-1]}")
    return a


def haar_levels(m):
    """L[p]: the number of Haar butterfly levels behind coefficient p of Psi_m x.

    Position 0 (the approximation a) passed all m levels; position p >= 1 lies in the
    detail block [2^{m-l}, 2^{m-l+1}) of level l = m - floor(log2 p).
    """
    n = 1 << m
    lev = np.empty(n, dtype=np.int64)
    lev[0] = m
    # frexp(p) = (f, e) with p = f 2^e, 1/2 <= f < 1, so floor(log2 p) = e - 1 (exact)
    _, e = np.frexp(np.arange(1, n, dtype=np.float64))
    lev[1:] = m - (e.astype(np.int64) - 1)
    return lev


def _level_scales(m, dtype):
    """2^{-L/2} per coefficient, each rounded once to ``dtype`` from its FP64 value."""
    table = np.array([2.0 ** (-L / 2.0) for L in range(m + 1)], dtype=np.float64).astype(dtype)
    return table[haar_levels(m)]


def haar_forward(x, m, dtype=np.float64, norm="per_level"):
    """z = Psi_m x along the last axis (eq. (2)), in ``dtype`` with ``norm``."""
    _check(dtype, norm)
    dt = np.dtype(dtype)
    v = np.array(_last_axis(x, m), dtype=dt, copy=True)
    if m == 0:
        return v
    c = inv_sqrt2(dt) if norm == "per_level" else None
    z = haar_analysis(v, c)
    if norm == "end":
        z = z * _level_scales(m, dt)
    return z


def haar_inverse(z, m, dtype=np.float64, norm="per_level"):
    """x = Psi_m^T z along the last axis (the transpose of eq. (2)), in ``dtype``."""
    _check(dtype, norm)
    dt = np.dtype(dtype)
    w = np.array(_last_axis(z, m), dtype=dt, copy=True)
    if m == 0:
        return w
    c = inv_sqrt2(dt) if norm == "per_level" else None
    if norm == "end":
        w = w * _level_scales(m, dt)
    return haar_synthesis(w, c)


def haar_walsh(z, m, dtype=np.float64, norm="per_level"):
    """y = H_m Psi_m^T z: stages r = 1..m-1 of Theorem 1 on Haar coefficients z.

    Stage r applies Psi_{m-r} to the second half of each of the 2^{r-1} blocks of
    length 2^{m-r+1}; first halves are left alone (the same loop as the cascade of
    Theorem 1 after its stage 0).
    """
    _check(dtype, norm)
    dt = np.dtype(dtype)
    y = np.array(_last_axis(z, m), dtype=dt, copy=True)
    if m == 0:
        return y
    c = inv_sqrt2(dt) if norm == "per_level" else None
    shape = y.shape
    for r in range(1, m):
        half = 1 << (m - r)
        v = y.reshape(shape[:-1] + (1 << (r - 1), 2 * half))
        v[..., half:] = haar_analysis(v[..., half:], c)
        y = v.reshape(shape)
    if norm == "end":
        for k in range(1, m):
            y[..., 1 << k: 2 << k] = y[..., 1 << k: 2 << k] * dt.type(2.0 ** (-k / 2.0))
    return y
