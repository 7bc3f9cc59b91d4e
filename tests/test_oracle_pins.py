"""Pins of the CPU oracle to things other than itself (no GPU).

Each test checks the oracle against what the paper or the mathematics fixes:
hand-derived matrices from eq. (1)/(2) and the printed stage expansion
(tests/golden), Theorem 1 in exact integer arithmetic, eq. (4), the counts of
Lemma 1 and Theorem 2, orthogonality / symmetry / involution / Parseval,
special inputs with known transforms, brute force on tiny sizes, and exact
integer ring arithmetic.
"""

from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle.lowp import bf16_bits_to_f32, f16_bits_to_f32
from oracle.transforms import bitrev_permutation
from conftest import load_golden_matrices, load_golden_table


# ------------------------------------------------------------ golden, hand-derived
def test_golden_hadamard_h2_h3():
    g = load_golden_matrices("hadamard_unnormalised.txt")
    assert np.array_equal(O.hadamard_dyadic(2, normalised=False), g["H2"])
    assert np.array_equal(O.hadamard_dyadic(3, normalised=False), g["H3"])
    s = 2.0 ** -1.5
    assert np.allclose(O.hadamard_dyadic(3), s * g["H3"], rtol=0, atol=1e-15)


def test_golden_haar_psi():
    g = load_golden_matrices("haar_unnormalised.txt")
    for m in (1, 2, 3):
        assert np.array_equal(O.haar_matrix(m, normalised=False), g[f"Psi{m}"])


def test_golden_cascade_stages_m3():
    g = load_golden_matrices("cascade_stages_m3.txt")
    h = load_golden_matrices("hadamard_unnormalised.txt")["H3"]
    psi3 = load_golden_matrices("haar_unnormalised.txt")["Psi3"]
    # The typed-in fixtures alone satisfy Theorem 1 (no oracle code involved) ...
    assert np.array_equal(g["F2"] @ g["F1"] @ psi3, h)
    # ... and the oracle builds the same factors and the same product.
    assert np.array_equal(O.cascade_stage_factor(3, 1, normalised=False), g["F1"])
    assert np.array_equal(O.cascade_stage_factor(3, 2, normalised=False), g["F2"])
    assert np.array_equal(O.cascade_product(3, normalised=False), h)


def test_golden_op_counts():
    table = load_golden_table("op_counts.txt")
    for m, haar_ops, chw_ops in table:
        c = O.OpCounter()
        O.haar_analysis(np.zeros(1 << m), counter=c)
        assert c.adds == haar_ops, ("Lemma 1", m)
        c = O.OpCounter()
        O.chw_cascade(np.zeros(1 << m), m, counter=c)
        assert c.adds == chw_ops == m * (1 << m), ("Theorem 2", m)


def test_op_counts_per_stage():
    # Stage r applies 2^{r-1} Haar transforms of length 2^{m-r}; Lemma 1 prices each.
    m = 9
    c = O.OpCounter()
    x = np.zeros(1 << m)
    y = O.haar_analysis(x, counter=c)
    assert c.adds == 2 * (2**m - 1)
    for r in range(1, m):
        c = O.OpCounter()
        half = 1 << (m - r)
        v = y.reshape(1 << (r - 1), 2 * half)
        O.haar_analysis(v[:, half:], counter=c)
        assert c.adds == 2 ** (r - 1) * 2 * (2 ** (m - r) - 1)


# ------------------------------------------------------------ Theorem 1, eq. (4)
@pytest.mark.parametrize("m", range(1, 11))
def test_theorem1_exact_integers(m):
    assert np.array_equal(O.cascade_product(m, normalised=False), O.hadamard_dyadic(m, normalised=False))


@pytest.mark.parametrize("m", range(1, 9))
def test_theorem1_normalised(m):
    assert np.abs(O.cascade_product(m) - O.hadamard_dyadic(m)).max() < 1e-13


@pytest.mark.parametrize("m", range(1, 9))
def test_eq4_haar_walsh(m):
    lhs = O.hadamard_dyadic(m) @ O.haar_matrix(m).T
    assert np.abs(lhs - O.haar_walsh_blockdiag(m)).max() < 1e-13


# ------------------------------------------------------------ structure of H_m
@pytest.mark.parametrize("m", range(0, 10))
def test_orthogonal_symmetric_involution(m):
    h = O.hadamard_dyadic(m)
    n = 1 << m
    assert np.abs(h @ h.T - np.eye(n)).max() < 1e-12
    assert np.array_equal(h, h.T)
    assert np.abs(h @ h - np.eye(n)).max() < 1e-12
    hu = O.hadamard_dyadic(m, normalised=False)
    assert np.array_equal(hu @ hu, n * np.eye(n, dtype=np.int64))


@pytest.mark.parametrize("m", range(0, 11))
def test_closed_form_entries(m):
    hu = O.hadamard_dyadic(m, normalised=False)
    n = 1 << m
    ks = range(n) if m <= 6 else np.random.default_rng(m).integers(0, n, 64)
    for k in ks:
        row = [O.hadamard_entry_closed_form(m, int(k), j) for j in range(n)]
        assert np.array_equal(hu[k], row)


def test_haar_analysis_matches_matrix_and_synthesis_inverts():
    rng = np.random.default_rng(11)
    for m in range(0, 9):
        x = rng.standard_normal((3, 1 << m))
        c = O.inv_sqrt2(np.float64)
        y = O.haar_analysis(x, c)
        assert np.abs(y - x @ O.haar_matrix(m).T).max() < 1e-12
        assert np.abs(O.haar_synthesis(y, c) - x).max() < 1e-12
        xi = rng.integers(-50, 50, (2, 1 << m))
        assert np.array_equal(O.haar_analysis(xi), xi @ O.haar_matrix(m, normalised=False).T)


# ------------------------------------------------------------ agreement, brute force
@pytest.mark.parametrize("m", range(0, 5))
def test_brute_force_unit_vectors(m):
    n = 1 << m
    eye = np.eye(n)
    dense = O.hadamard_dyadic(m)
    assert np.abs(O.wht_fast_dyadic(eye, m) - dense.T).max() < 1e-14
    assert np.abs(O.chw_cascade(eye, m) - dense.T).max() < 1e-14
    assert np.abs(O.wht_dense(eye, m) - dense.T).max() < 1e-14
    for j in range(n):
        cf = O.wht_closed_form(eye[j], m, list(range(n)))
        assert np.abs(cf - dense[:, j]).max() < 1e-14
    ei = np.eye(n, dtype=np.int64)
    assert np.array_equal(O.wht_fast_dyadic(ei, m, normalised=False), O.hadamard_dyadic(m, False).T)
    assert np.array_equal(O.chw_cascade(ei, m, np.int64, "none"), O.hadamard_dyadic(m, False).T)


@pytest.mark.parametrize("m", [1, 2, 5, 8, 10, 12])
def test_random_agreement(m):
    rng = np.random.default_rng(100 + m)
    x = rng.standard_normal((4, 1 << m))
    y2 = O.wht_fast_dyadic(x, m)
    y4 = O.chw_cascade(x, m)
    assert np.abs(y2 - y4).max() < 1e-12
    if m <= 10:
        assert np.abs(O.wht_dense(x, m) - y2).max() < 1e-12
    ks = rng.integers(0, 1 << m, 16)
    assert np.abs(O.wht_closed_form(x[1], m, ks) - y2[1, ks]).max() < 1e-12


def test_bitrev_permutation():
    for m in range(0, 11):
        perm = bitrev_permutation(m)
        assert [O.bitrev(k, m) for k in range(1 << m)] == perm.tolist()
        assert np.array_equal(perm[perm], np.arange(1 << m))


# ------------------------------------------------------------ special inputs
@pytest.mark.parametrize("m", [0, 1, 3, 7, 12])
def test_special_inputs(m):
    n = 1 << m
    e0 = np.zeros(n)
    e0[0] = 1.0
    for f in (O.wht_fast_dyadic, O.chw_cascade):
        assert np.abs(f(e0, m) - 2.0 ** (-m / 2)).max() < 1e-14
        ones = np.ones(n)
        expect = np.zeros(n)
        expect[0] = 2.0 ** (m / 2)
        assert np.abs(f(ones, m) - expect).max() < 1e-9
    rng = np.random.default_rng(m)
    for k in rng.integers(0, n, 4):
        row = np.array([O.hadamard_entry_closed_form(m, int(k), j) for j in range(n)], dtype=np.float64)
        row *= 2.0 ** (-m / 2)
        y = O.chw_cascade(row, m)
        expect = np.zeros(n)
        expect[k] = 1.0
        assert np.abs(y - expect).max() < 1e-12


def test_parseval_and_involution_large():
    rng = np.random.default_rng(7)
    m = 16
    x = rng.standard_normal((2, 1 << m))
    y = O.wht_fast_dyadic(x, m)
    assert np.allclose(np.linalg.norm(y, axis=1), np.linalg.norm(x, axis=1), rtol=1e-13)
    assert np.abs(O.wht_fast_dyadic(y, m) - x).max() < 1e-11
    xi = rng.integers(-(2**14), 2**14, (2, 1 << m), endpoint=True)
    yi = O.wht_fast_dyadic(xi, m, normalised=False)
    assert np.array_equal(O.wht_fast_dyadic(yi, m, normalised=False), (1 << m) * xi)


# ------------------------------------------------------------ integer ring, fp32 form
def test_int32_cascade_is_int64_mod_2_32():
    rng = np.random.default_rng(3)
    for m in (4, 9, 13):
        x = rng.integers(-(2**31), 2**31 - 1, (3, 1 << m), endpoint=True, dtype=np.int64)
        y32 = O.chw_cascade(x.astype(np.int32), m, np.int32, "none")
        y64 = O.wht_fast_dyadic(x, m, normalised=False)
        wrapped = ((y64 + 2**31) % 2**32 - 2**31).astype(np.int32)
        assert np.array_equal(y32, wrapped)


def test_reverse_cascade_is_transpose():
    rng = np.random.default_rng(5)
    for m in range(1, 9):
        y = rng.standard_normal((2, 1 << m))
        assert np.abs(O.chw_reverse_cascade(y, m) - y @ O.hadamard_dyadic(m)).max() < 1e-12
        yi = rng.integers(-100, 100, (2, 1 << m))
        assert np.array_equal(
            O.chw_reverse_cascade(yi, m, np.int64, "none"), yi @ O.hadamard_dyadic(m, normalised=False)
        )


def test_fp32_reverse_cascade_rounds_like_forward():
    # Each butterfly matrix is symmetric and the dyadic reorder is an involution, so
    # the transposed cascade is the forward cascade's graph with inputs and outputs
    # relabelled: the fp32 results agree bit for bit.
    rng = np.random.default_rng(9)
    for m in range(1, 14):
        x = rng.standard_normal((3, 1 << m)).astype(np.float32)
        for norm in ("per_level", "end", "none"):
            a = O.chw_cascade(x, m, np.float32, norm)
            b = O.chw_reverse_cascade(x, m, np.float32, norm)
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def _nearest_f32_to(value_decimal):
    """The fp32 nearest to an exact decimal value, by checking the neighbours exactly."""
    f = np.float32(float(value_decimal))
    best = None
    for cand in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - Fraction(value_decimal))
        if best is None or d < best[0]:
            best = (d, cand)
    return best[1]


def test_constants_are_correctly_rounded():
    getcontext().prec = 60
    s = Decimal(1) / Decimal(2).sqrt()
    assert O.inv_sqrt2(np.float32) == _nearest_f32_to(s)
    assert O.inv_sqrt2(np.float32).view(np.uint32) == 0x3F3504F3
    for m in range(0, 31):
        exact = Decimal(2) ** (-(m // 2)) * (s if m % 2 else Decimal(1))
        assert O.end_scale_f32(m) == _nearest_f32_to(exact)


@pytest.mark.parametrize("m", [4, 10, 16])
def test_fp32_cascade_error_bound(m):
    # Each of the m levels adds at most one rounding (two with the 1/sqrt2 multiply)
    # of relative size u = 2^-24 per value; with c rounded too the normwise error
    # stays below (2m + 1) u (orthogonal stages do not amplify errors).
    rng = np.random.default_rng(m)
    x = rng.standard_normal((4, 1 << m)).astype(np.float32)
    ref = O.wht_fast_dyadic(x.astype(np.float64), m)
    u = 2.0**-24
    for norm in ("per_level", "end"):
        y = O.chw_cascade(x, m, np.float32, norm)
        assert O.rel_err_per_signal(y, ref).max() <= (2 * m + 1) * u


# ------------------------------------------------------------ low precision form
def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5, 0.0, 3.0e38, 1e-40], dtype=np.float32)
    bits = O.round_to_bf16(vals)
    # 1+2^-8 is a tie between 1 and 1+2^-7: even mantissa (1.0) wins; 1+3*2^-8 -> 1+2^-6.
    assert bits[0] == 0x3F80 and bits[1] == 0x3F80 and bits[2] == 0x3F82
    assert bits[3] == 0xC020 and bits[4] == 0
    assert np.isfinite(bf16_bits_to_f32(bits[:5])).all()
    f16 = O.round_to_f16(np.array([1.0, 65504.0, 2.0**-24], dtype=np.float32))
    assert f16.tolist() == [0x3C00, 0x7BFF, 0x0001]
    assert f16_bits_to_f32(f16).tolist() == [1.0, 65504.0, 2.0**-24]


@pytest.mark.parametrize("fmt,gate", [("bf16", 1e-2), ("f16", 2e-3)])
def test_lowp_reference_properties(fmt, gate):
    m = 8
    rng = np.random.default_rng(4)
    x = rng.standard_t(3, (6, 1 << m)) * rng.lognormal(0, 2, (6, 1))
    K = 0 if fmt == "bf16" else 14
    e_in = np.floor(np.log2(np.abs(x).max(axis=1))).astype(np.int64) - K
    scaled = np.ldexp(x, -e_in[:, None]).astype(np.float32)
    bits = O.round_to_bf16(scaled) if fmt == "bf16" else O.round_to_f16(scaled)
    bits[5] = 0  # an all-zero signal
    qb, e_out = O.lowp_forward_reference(bits, e_in, m, fmt)
    q = bf16_bits_to_f32(qb) if fmt == "bf16" else f16_bits_to_f32(qb)
    top = np.abs(q[:5]).max(axis=1)
    assert ((top >= 2.0**K) & (top < 2.0 ** (K + 1))).all()
    assert np.all(q[5] == 0) and e_out[5] == e_in[5]
    ref = O.wht_fast_dyadic(O.dequantise(bits, e_in, fmt), m)
    err = O.rel_err_per_signal(O.dequantise(qb, e_out, fmt)[:5], ref[:5])
    assert err.max() < gate


# ---------------------------------------------------------------- O3 on sparse inputs
@pytest.mark.parametrize("m", [0, 1, 3, 6, 10])
def test_sparse_closed_form_matches_dense_matrix(m):
    rng = np.random.default_rng(90 + m)
    n = 1 << m
    js = rng.choice(n, size=min(n, 5), replace=False)
    cs = rng.integers(-7, 8, size=len(js))
    x = np.zeros(n, dtype=np.int64)
    x[js] = cs
    h = O.hadamard_dyadic(m, normalised=False)  # integer rows of eq. (1)
    ks = np.arange(n)
    assert np.array_equal(O.wht_sparse_closed_form(js, cs, m, ks, normalised=False), h @ x)
    got = O.wht_sparse_closed_form(js, cs, m, ks)
    assert np.allclose(got, O.hadamard_dyadic(m) @ x, rtol=0, atol=1e-12)


def test_sparse_closed_form_sampled_outputs_agree_with_fast_wht():
    m = 14
    rng = np.random.default_rng(7)
    js = rng.choice(1 << m, size=6, replace=False)
    cs = rng.integers(-100, 101, size=6)
    x = np.zeros((1, 1 << m), dtype=np.int64)
    x[0, js] = cs
    full = O.wht_fast_dyadic(x, m, normalised=False)[0]
    ks = rng.integers(0, 1 << m, 500)
    assert np.array_equal(O.wht_sparse_closed_form(js, cs, m, ks, normalised=False), full[ks])
