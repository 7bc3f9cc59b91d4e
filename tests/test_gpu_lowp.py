"""bf16/fp16 storage with fp32 accumulation and per-signal power-of-two exponents (GPU).

The output exponent and the 16-bit codes are integers decided by floating point, so the
oracle decides them the same way, in fp32 on the fp32 values of the cascade
(oracle.lowp): exponents and codes must match exactly.  The error of the dequantised
result against the FP64 transform of the dequantised input is gated per signal (max and
p99): bf16 <= 1e-2, fp16 <= 2e-3.
"""

import numpy as np
import pytest

import oracle as O
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GATES = {"bf16": 1e-2, "f16": 2e-3}


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


def run_lowp(chw, bits, e_in, m, fmt, norm="end", adjoint=False, diag=None):
    import torch

    tdt = torch.bfloat16 if fmt == "bf16" else torch.float16
    batch = bits.shape[0]
    p = chw.chw_plan(m, batch, fmt, norm)
    x = torch.from_numpy(bits.view(np.int16)).cuda().view(tdt)
    y = torch.empty_like(x)
    ei = torch.from_numpy(e_in.astype(np.int32)).cuda()
    eo = torch.empty_like(ei)
    dd = None if diag is None else torch.from_numpy(diag).cuda()
    (chw.chw_adjoint if adjoint else chw.chw_forward)(p, x, y, ei, eo, diag=dd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    return y.view(torch.int16).cpu().numpy().view(np.uint16), eo.cpu().numpy()


def check(chw, m, batch, fmt, norm, seed):
    x64 = W.heavy_tailed_f64(m, batch, seed)
    bits, e_in = W.quantise_pow2(x64, fmt)
    qb, e_out = run_lowp(chw, bits, e_in, m, fmt, norm)
    rb, re = O.lowp_forward_reference(bits, e_in, m, fmt, norm)
    assert np.array_equal(e_out, re), "exponents differ"
    assert np.array_equal(qb, rb), f"{np.count_nonzero(qb != rb)} codes differ"
    ref = O.wht_fast_dyadic(O.dequantise(bits, e_in, fmt), m)
    err = O.rel_err_per_signal(O.dequantise(qb, e_out, fmt), ref)
    assert err.max() <= GATES[fmt] and np.percentile(err, 99) <= GATES[fmt]
    return err


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("m", [3, 6, 9, 11, 12, 13])
def test_lowp_every_tier_size(chw, fmt, m):
    check(chw, m, 24, fmt, "end", seed=40 + m)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("m", [11, 12])
def test_lowp_fused_tier_and_adjoint(chw, fmt, m):
    import paper_1609_06641_gb300 as mod

    p = mod.chw_plan(m, 4, fmt, "end")
    assert mod.chw_plan_get_info(p).tier == 5
    x64 = W.heavy_tailed_f64(m, 40, 60 + m)
    bits, e_in = W.quantise_pow2(x64, fmt)
    qb, e_out = run_lowp(chw, bits, e_in, m, fmt, adjoint=True)
    rb, re = O.lowp_forward_reference(bits, e_in, m, fmt)  # H^T = H, same rounding
    assert np.array_equal(e_out, re) and np.array_equal(qb, rb)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("m", [11, 12])
def test_lowp_per_level(chw, fmt, m):
    check(chw, m, 16, fmt, "per_level", seed=3 + m)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("m", [11, 12])
def test_lowp_adjoint_with_input_diagonal(chw, fmt, m):
    # H^T D y: D flips the signs of the input codes, then the same transform and rounding
    x64 = W.heavy_tailed_f64(m, 12, 70 + m)
    bits, e_in = W.quantise_pow2(x64, fmt)
    d = W.diag_pm1(m, 8)
    qb, e_out = run_lowp(chw, bits, e_in, m, fmt, adjoint=True, diag=d)
    flipped = bits ^ np.where(d < 0, np.uint16(0x8000), np.uint16(0))[None, :]
    rb, re = O.lowp_forward_reference(flipped, e_in, m, fmt)
    assert np.array_equal(e_out, re) and np.array_equal(qb, rb)


@pytest.mark.parametrize("m", [11, 12])
def test_lowp_bf16_subnormal_codes(chw, m):
    # bf16 codes of magnitude below 2^-126 (subnormal): max|u| < 2^-120, so the output
    # scaling 2^(K - E) lies outside fp32's normal range and takes two multiplies; the
    # arithmetic keeps subnormals (no flush to zero), as the oracle's fp32 does
    rng = np.random.default_rng(11 + m)
    mag = rng.integers(1, 0x80, size=(6, 1 << m), dtype=np.uint16)  # bf16 subnormal patterns
    bits = mag | np.where(rng.random((6, 1 << m)) < 0.5, np.uint16(0x8000), np.uint16(0))
    bits[1, :] = 0x0001  # one all-equal signal: its transform is a single nonzero entry
    e_in = rng.integers(-5, 5, 6).astype(np.int32)
    qb, e_out = run_lowp(chw, bits, e_in, m, "bf16")
    rb, re = O.lowp_forward_reference(bits, e_in, m, "bf16")
    assert np.array_equal(e_out, re) and np.array_equal(qb, rb)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_lowp_config_m12_batch16384(chw, fmt):
    # the full configuration; the exact-code check runs on a sample of signals
    m, batch = 12, 16384
    x64 = W.heavy_tailed_f64(m, batch, 4)
    bits, e_in = W.quantise_pow2(x64, fmt)
    qb, e_out = run_lowp(chw, bits, e_in, m, fmt)
    rows = np.random.default_rng(1).choice(batch, 256, replace=False)
    rb, re = O.lowp_forward_reference(bits[rows], e_in[rows], m, fmt)
    assert np.array_equal(e_out[rows], re)
    assert np.array_equal(qb[rows], rb)
    ref = O.wht_fast_dyadic(O.dequantise(bits, e_in, fmt), m)
    err = O.rel_err_per_signal(O.dequantise(qb, e_out, fmt), ref)
    assert err.max() <= GATES[fmt], err.max()
    assert np.percentile(err, 99) <= GATES[fmt]
    # against the original FP64 draw (input quantisation included): reported, loosely gated
    err_draw = O.rel_err_per_signal(O.dequantise(qb, e_out, fmt), O.wht_fast_dyadic(x64, m))
    assert err_draw.max() <= 2 * GATES[fmt]


@pytest.mark.parametrize("m", [10, 11, 12])
def test_lowp_zero_signal_and_diag(chw, m):
    x64 = W.heavy_tailed_f64(m, 4, 9)
    x64[2] = 0
    bits, e_in = W.quantise_pow2(x64, "f16")
    e_in[2] = 17
    d = W.diag_pm1(m, 6)
    qb, e_out = run_lowp(chw, bits, e_in, m, "f16", diag=d)
    # D H 0 = 0: codes are +0 or -0 (a -1 entry of D flips the sign of a zero)
    assert np.all(O.codes_to_f32(qb[2], "f16") == 0) and e_out[2] == 17
    rb, re = O.lowp_forward_reference(bits, e_in, m, "f16")
    assert np.array_equal(e_out, re)
    signed = O.codes_to_f32(rb, "f16") * d.astype(np.float32)
    assert np.array_equal(O.codes_to_f32(qb, "f16"), signed)
