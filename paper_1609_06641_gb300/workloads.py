"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Nothing here computes any part of the transform: these are random draws (numpy PCG64,
``default_rng(seed)``), their casts to the storage dtypes, the per-signal power-of-two
input scaling of the bf16/fp16 form, and the packing of ragged batches.  Both the CPU
oracle and the CUDA path consume the same arrays.

The paper runs no experiments, so the workloads stand for the shapes named in the
library's benchmark configurations: batched N(0,1) fp32 signals, bounded uniform int32
signals (exactly representable results), long uniform(-1,1) signals, heavy-tailed
signals with a wide per-signal dynamic range for the 16-bit storage form, and ragged
batches of mixed lengths.  A smaller ``batch`` takes the first rows of the same stream.
"""

import numpy as np

# Per-signal top binade of the 16-bit codes: max|q| in [2^K, 2^(K+1)).
TOP_BINADE = {"bf16": 0, "f16": 14}


def normal_f32(m, batch, seed):
    """batch x 2^m i.i.d. N(0,1), drawn directly in fp32."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, 1 << m), dtype=np.float32)


def uniform_int32(m, batch, seed, bound=2**14):
    """batch x 2^m integers uniform on [-bound, bound] (int32)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-bound, bound, size=(batch, 1 << m), endpoint=True, dtype=np.int32)


def uniform_pm1_f32(m, batch, seed):
    """batch x 2^m i.i.d. Uniform(-1, 1) in fp32 (2r - 1 is exact for r = k 2^-24)."""
    rng = np.random.default_rng(seed)
    r = rng.random((batch, 1 << m), dtype=np.float32)
    return r * np.float32(2) - np.float32(1)


def heavy_tailed_f64(m, batch, seed):
    """Student-t (nu = 3) entries times a per-signal lognormal(0, sigma=2) scale, FP64."""
    rng = np.random.default_rng(seed)
    scale = rng.lognormal(0.0, 2.0, (batch, 1))
    return rng.standard_t(3, (batch, 1 << m)) * scale


def _bf16_bits(f32):
    u = np.ascontiguousarray(f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def quantise_pow2(x64, fmt):
    """Store FP64 signals as (codes, exponents): x = 2^e q with max|q| in [2^K, 2^(K+1)).

    Returns (uint16 code patterns (batch, n), int32 exponents (batch,)).  Codes are the
    FP64 value scaled by 2^-e, rounded to fp32 and then to bf16/fp16 (nearest even).
    All-zero signals get e = 0.
    """
    K = TOP_BINADE[fmt]
    big = np.abs(x64).max(axis=1)
    e = np.zeros(x64.shape[0], dtype=np.int64)
    nz = big > 0
    e[nz] = np.floor(np.log2(big[nz])).astype(np.int64) - K
    scaled = np.ldexp(x64, -e[:, None]).astype(np.float32)
    bits = _bf16_bits(scaled) if fmt == "bf16" else scaled.astype(np.float16).view(np.uint16)
    return bits, e.astype(np.int32)


def ragged_ms(count, seed, lo=6, hi=20):
    """Bit counts m_i uniform on [lo, hi] (the first draw of the ragged stream)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=count, endpoint=True).astype(np.uint8), rng


def ragged_offsets(ms):
    """Packing of a ragged batch (the library's): signal i starts at offsets[i], a multiple
    of 32 elements, or of 2^(m-8) for m = 15..17; the end is rounded up to 32."""
    off = np.zeros(len(ms) + 1, dtype=np.int64)
    o = 0
    for i, m in enumerate(ms):
        al = 1 << (int(m) - 8) if 15 <= int(m) <= 17 else 32
        o = (o + al - 1) // al * al
        off[i] = o
        o += 1 << int(m)
        o = (o + 31) // 32 * 32
    off[len(ms)] = o
    return off


def ragged_normal_f32(count, seed, lo=6, hi=20):
    """A ragged batch: ms from ``ragged_ms`` then N(0,1) fp32 values from the same stream,
    packed at ``ragged_offsets`` (padding entries are zero)."""
    ms, rng = ragged_ms(count, seed, lo, hi)
    off = ragged_offsets(ms)
    x = np.zeros(off[-1], dtype=np.float32)
    for i, m in enumerate(ms):
        x[off[i]: off[i] + (1 << int(m))] = rng.standard_normal(1 << int(m), dtype=np.float32)
    return ms, off, x


def diag_pm1(m, seed):
    """A random +-1 diagonal of length 2^m (int8)."""
    rng = np.random.default_rng(seed)
    return (1 - 2 * rng.integers(0, 2, size=1 << m)).astype(np.int8)
