"""bf16 / fp16 storage form with per-signal power-of-two exponents (test infrastructure only).

Storage convention: a signal is a pair (q, e) meaning x = 2^e * q, with q stored in
bf16 or fp16 and e an int32 per signal.  The transform is accumulated in fp32.
The paper fixes no precision; this form and its rules are the library's:

  1. u = CHW(q) in fp32 (``chw_cascade`` in fp32, "end" or "per_level" mode), so
     that H_m x ~= 2^{e_in} u.
  2. M = max_j |u_j| (exact in fp32).  If M == 0: e_out = e_in and q_out = 0.
  3. E = floor(log2 M), read exactly from M's binary exponent.
  4. e_out = e_in + E - K and q_out = round_fmt(u * 2^{K-E}), the multiply done in
     fp32 (split into two power-of-two multiplies if 2^{K-E} is outside fp32's
     normal range), rounded to nearest even into the storage format.
     K = 0 for bf16 (|q_out| < 2) and K = 14 for fp16 (|q_out| < 2^15 < 65504).

Because the exponent and the codes are integers decided by floating point, they
are decided here in fp32 on the fp32 values of the cascade: the same precision the
kernels decide them in, so the codes can be compared exactly.
"""

import numpy as np

from .transforms import chw_cascade

TOP_BINADE = {"bf16": 0, "f16": 14}


def round_to_bf16(v):
    """Round fp32 values to bf16 (nearest, ties to even); returns the uint16 patterns."""
    f = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    rounded = (u + 0x7FFF + lsb) >> 16
    nan = np.isnan(f)
    out = rounded.astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def bf16_bits_to_f32(bits):
    """Widen bf16 bit patterns to fp32 values (exact)."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32)


def round_to_f16(v):
    """Round fp32 values to fp16 (IEEE nearest-even); returns the uint16 patterns."""
    return np.asarray(v, dtype=np.float32).astype(np.float16).view(np.uint16)


def f16_bits_to_f32(bits):
    return np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float32)


def codes_to_f32(bits, fmt):
    return bf16_bits_to_f32(bits) if fmt == "bf16" else f16_bits_to_f32(bits)


def dequantise(bits, e, fmt):
    """FP64 values 2^e * q of stored (q, e) pairs; ``bits`` has shape (batch, n)."""
    q = codes_to_f32(bits, fmt).astype(np.float64)
    return np.ldexp(q, np.asarray(e, dtype=np.int64)[:, None])


def _pow2_f32(k):
    return np.float32(np.ldexp(1.0, int(k)))


def _scale_pow2_f32(u, k):
    """u * 2^k in fp32; two multiplies when 2^k is outside fp32's normal range."""
    if -126 <= k <= 127:
        return u * _pow2_f32(k)
    h = int(k / 2)
    return (u * _pow2_f32(h)) * _pow2_f32(k - h)


def lowp_forward_reference(bits, e_in, m, fmt, norm="end"):
    """Reference (q_out bits, e_out) for stored input (bits, e_in), per the rules above.

    ``bits``: uint16 array (batch, 2^m); ``e_in``: int array (batch,).
    Returns (uint16 array (batch, 2^m), int64 array (batch,)).
    """
    if fmt not in TOP_BINADE:
        raise ValueError("fmt must be 'bf16' or 'f16'")
    K = TOP_BINADE[fmt]
    q = codes_to_f32(bits, fmt)
    u = chw_cascade(q, m, np.float32, norm)
    out_bits = np.zeros(u.shape, dtype=np.uint16)
    e_out = np.zeros(u.shape[0], dtype=np.int64)
    for s in range(u.shape[0]):
        big = np.float32(np.max(np.abs(u[s])))
        if big == 0:
            e_out[s] = int(e_in[s])
            continue
        _, ex = np.frexp(np.float64(big))  # big = f * 2^ex with f in [0.5, 1)
        E = int(ex) - 1
        scaled = _scale_pow2_f32(u[s], K - E)
        out_bits[s] = round_to_bf16(scaled) if fmt == "bf16" else round_to_f16(scaled)
        e_out[s] = int(e_in[s]) + E - K
    return out_bits, e_out
