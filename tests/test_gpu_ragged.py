"""Ragged batches: one persistent, graph-replayed launch over signals of uneven length (GPU)."""

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


def run(chw, ms, x, dtype="f32", norm="end", inplace=False, repeats=1):
    import torch

    p = chw.chw_plan_ragged(ms, dtype, norm)
    off = chw.chw_ragged_offsets(p)
    assert np.array_equal(off, W.ragged_offsets(ms))
    xd = torch.from_numpy(x).cuda()
    yd = xd if inplace else torch.empty_like(xd)
    for _ in range(repeats):
        if inplace:
            xd.copy_(torch.from_numpy(x))
        chw.chw_forward_ragged(p, xd, yd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    return yd.cpu().numpy(), off, p


def per_signal_ref(ms, off, x, dtype, norm):
    outs = []
    for i, m in enumerate(ms):
        seg = x[off[i]: off[i] + (1 << int(m))][None, :]
        outs.append(O.chw_cascade(seg, int(m), dtype, norm)[0])
    return outs


@pytest.mark.parametrize("norm", ["end", "per_level"])
def test_ragged_mixed_lengths(chw, norm):
    # every length 0..20 appears, in a shuffled order, with repeats
    rng = np.random.default_rng(11)
    ms = np.concatenate([np.arange(0, 21), rng.integers(0, 21, 40)]).astype(np.uint8)
    rng.shuffle(ms)
    off = W.ragged_offsets(ms)
    x = np.zeros(off[-1], dtype=np.float32)
    for i, m in enumerate(ms):
        x[off[i]: off[i] + (1 << int(m))] = rng.standard_normal(1 << int(m), dtype=np.float32)
    got, _, p = run(chw, ms, x, "f32", norm, repeats=2)
    info = chw.chw_plan_get_info(p)
    assert info.tier == 4 and info.kernels_per_call >= 1  # one graph launch replays them
    for i, ref in enumerate(per_signal_ref(ms, off, x, np.float32, norm)):
        assert_bitwise(got[off[i]: off[i] + ref.size], ref, f"signal {i} m={ms[i]}")


def test_ragged_int32_and_in_place(chw):
    rng = np.random.default_rng(12)
    ms = rng.integers(0, 21, 30).astype(np.uint8)
    off = W.ragged_offsets(ms)
    x = np.zeros(off[-1], dtype=np.int32)
    for i, m in enumerate(ms):
        x[off[i]: off[i] + (1 << int(m))] = rng.integers(-(2**9), 2**9, 1 << int(m))
    got, _, _ = run(chw, ms, x, "i32", "none", inplace=True)
    for i, m in enumerate(ms):
        seg = x[off[i]: off[i] + (1 << int(m))].astype(np.int64)
        ref = O.wht_fast_dyadic(seg, int(m), normalised=False)
        assert np.array_equal(got[off[i]: off[i] + (1 << int(m))], ref.astype(np.int32)), (i, m)


def test_ragged_long_signals_in_several_scratch_chunks(chw):
    # 2^20-element signals go through the two-pass scratch 64 at a time: 70 of them take two
    # chunks; lengths 13..17 and a few short signals are mixed in, in a shuffled order
    rng = np.random.default_rng(13)
    ms = np.concatenate([np.full(70, 20), rng.integers(13, 18, 12), rng.integers(0, 13, 8)]).astype(np.uint8)
    rng.shuffle(ms)
    off = W.ragged_offsets(ms)
    x = rng.standard_normal(off[-1], dtype=np.float32)
    got, _, p = run(chw, ms, x, "f32", "end", repeats=2)
    info = chw.chw_plan_get_info(p)
    lengths = set(int(m) for m in ms)
    expect = int(any(m <= 12 for m in lengths)) + sum(1 for m in lengths if 13 <= m <= 17)
    expect += sum(2 * -(-int((ms == m).sum()) // (1 << (26 - m))) for m in lengths if m >= 18)
    assert info.passes == 2 and info.kernels_per_call == expect == 1 + 4 + 4  # m = 20: 2 chunks x 2 passes
    long_ids = [i for i in range(len(ms)) if ms[i] == 20]
    picks = list(rng.choice(len(ms), 8, replace=False)) + [long_ids[0], long_ids[63], long_ids[64], long_ids[-1]]
    for i in picks:
        ref = O.chw_cascade(x[off[i]: off[i] + (1 << int(ms[i]))][None, :], int(ms[i]), np.float32, "end")[0]
        assert_bitwise(got[off[i]: off[i] + ref.size], ref, f"signal {i} m={ms[i]}")


def test_ragged_config_10000_signals(chw):
    ms, off, x = W.ragged_normal_f32(10000, 5)
    got, _, p = run(chw, ms, x, "f32", "end")
    rng = np.random.default_rng(0)
    pick = list(rng.choice(len(ms), 12, replace=False)) + [int(np.argmax(ms)), int(np.argmin(ms))]
    for i in pick:
        seg = x[off[i]: off[i] + (1 << int(ms[i]))]
        ref = O.chw_cascade(seg[None, :], int(ms[i]), np.float32, "end")[0]
        assert_bitwise(got[off[i]: off[i] + ref.size], ref, f"signal {i} m={ms[i]}")
        err = O.rel_err_per_signal(got[off[i]: off[i] + ref.size], O.wht_fast_dyadic(seg.astype(np.float64), int(ms[i])))
        assert err.max() <= 1e-6


@pytest.mark.parametrize("shift", [0, 32])
def test_ragged_tensor_memory_groups_with_caller_offsets(chw, shift):
    # Signals of 2^15..2^17 run on the tensor-memory tiers (one SM, or a pair of SMs for
    # 2^17) when every offset of their length is a whole output run (2^(m-8) elements);
    # offsets moved by 32 elements are not, and those lengths fall back to clusters of
    # shared-memory tiles.  Both must give the cascade's bits, in every normalisation.
    import torch

    rng = np.random.default_rng(14 + shift)
    ms = np.concatenate([np.full(5, 15), np.full(5, 16), np.full(5, 17), rng.integers(6, 15, 10)]).astype(np.uint8)
    rng.shuffle(ms)
    base = W.ragged_offsets(ms)
    off = base[:-1] + shift
    total = int(base[-1]) + shift
    x = np.zeros(total, dtype=np.float32)
    for i, m in enumerate(ms):
        x[off[i]: off[i] + (1 << int(m))] = rng.standard_normal(1 << int(m), dtype=np.float32)
    for norm in ("end", "per_level"):
        p = chw.chw_plan_ragged(ms, "f32", norm, offsets=off, total=total)
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        chw.chw_forward_ragged(p, xd, yd)
        torch.cuda.synchronize()
        assert chw.chw_last_device_status(p) == 0
        got = yd.cpu().numpy()
        for i, m in enumerate(ms):
            ref = O.chw_cascade(x[off[i]: off[i] + (1 << int(m))][None, :], int(m), np.float32, norm)[0]
            assert_bitwise(got[off[i]: off[i] + ref.size], ref, f"shift {shift} signal {i} m={m} {norm}")
