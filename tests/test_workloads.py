"""Seeded input generators: determinism, shapes, prefix property, 16-bit scaling, packing (CPU)."""

import numpy as np

from paper_1609_06641_gb300 import workloads as W


def test_deterministic_and_prefix_consistent():
    a = W.normal_f32(10, 64, 0)
    b = W.normal_f32(10, 8, 0)
    assert a.dtype == np.float32 and a.shape == (64, 1024)
    assert np.array_equal(a[:8], b)
    assert np.array_equal(a, W.normal_f32(10, 64, 0))
    i = W.uniform_int32(12, 16, 1)
    assert i.dtype == np.int32 and i.min() >= -(2**14) and i.max() <= 2**14
    assert np.array_equal(i[:4], W.uniform_int32(12, 4, 1))
    u = W.uniform_pm1_f32(12, 4, 3)
    assert u.min() >= -1 and u.max() < 1


def test_quantise_pow2_top_binade():
    x = W.heavy_tailed_f64(8, 32, 4)
    for fmt, K in (("bf16", 0), ("f16", 14)):
        bits, e = W.quantise_pow2(x, fmt)
        q = bits.view(np.float16).astype(np.float64) if fmt == "f16" else (bits.astype(np.uint32) << 16).view(np.float32)
        top = np.abs(q).max(axis=1)
        assert ((top >= 2.0**K) & (top <= 2.0 ** (K + 1))).all()
        back = np.ldexp(np.asarray(q, dtype=np.float64), e.astype(np.int64)[:, None])
        rel = np.linalg.norm(back - x, axis=1) / np.linalg.norm(x, axis=1)
        assert rel.max() < (1e-2 if fmt == "bf16" else 1e-3)


def test_ragged_packing():
    ms, off, x = W.ragged_normal_f32(50, 5, lo=0, hi=12)
    assert len(off) == 51 and off[0] == 0
    assert np.all(off % 32 == 0)
    sizes = np.diff(off)
    assert np.all(sizes >= (1 << ms.astype(np.int64)))
    assert x.shape == (off[-1],)
    ms2, _ = W.ragged_ms(50, 5, lo=0, hi=12)
    assert np.array_equal(ms, ms2)


def test_diag():
    d = W.diag_pm1(10, 6)
    assert d.dtype == np.int8 and set(np.unique(d)) == {-1, 1}


def test_ragged_packing_aligns_long_signals():
    # signals of 2^15..2^17 start on whole output runs of the tensor-memory kernels
    # (2^(m-8) elements), every other one on 32; signals never overlap

    ms, _ = W.ragged_ms(2000, 5, lo=6, hi=20)
    off = W.ragged_offsets(ms)
    for i, m in enumerate(ms):
        al = 1 << (int(m) - 8) if 15 <= int(m) <= 17 else 32
        assert off[i] % al == 0
        assert off[i] + (1 << int(m)) <= off[i + 1]
    assert off[-1] % 32 == 0
    # the padding stays small: under 0.1 % of the elements for this length mix
    assert off[-1] - sum(1 << int(m) for m in ms) < 1e-3 * off[-1]
    assert np.all(np.diff(off) > 0)
