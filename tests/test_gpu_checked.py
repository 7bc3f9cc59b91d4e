"""Checked mode (CHW_FLAG_CHECKED) and caller-chosen ragged layouts (GPU).

The checked mode stands in for a memory checker: the kernels that compute global indices
from offsets range-check every input tile and output address and latch
CHW_ERR_DEVICE_CHECK with the offending index instead of using it.  On valid inputs a
checked plan must give the same bits as an unchecked one and report CHW_OK.

The failure path is exercised by host-side corruption only: the test hook
CHW_FLAG_TEST_CORRUPT (accepted only together with CHW_FLAG_CHECKED) makes the plan
overwrite, on the host before upload, two signals' offsets with indices past the end of x
and y.  The buffers the test passes are allocated far larger than the plan's `total`, so
every corrupted range still lies inside memory the test owns: a missed check would write
into that guard region (which the test inspects), never outside an allocation.
"""

import numpy as np
import pytest

import oracle as O
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SENTINEL = np.float32(-12345.5)


@pytest.fixture(scope="module")
def chw(cuda_device):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    return chw


@pytest.fixture(scope="module")
def torch(cuda_device):
    import torch

    return torch


@pytest.mark.parametrize("m,batch,order", [(10, 64, "dyadic"), (14, 8, "dyadic"), (16, 6, "dyadic"), (16, 4, "sequency"),
                                           (15, 4, "natural"), (20, 2, "dyadic"), (26, 1, "dyadic")])
def test_checked_plan_is_bitwise_unchecked(chw, torch, m, batch, order):
    x = torch.from_numpy(W.normal_f32(m, batch, seed=900 + m)).cuda()
    outs = []
    for flags in (0, chw.CHW_FLAG_CHECKED):
        p = chw.chw_plan(m, batch, "f32", "end", flags, order=order)
        y = torch.empty_like(x)
        chw.chw_forward(p, x, y)
        torch.cuda.synchronize()
        assert chw.chw_last_device_status(p) == 0
        outs.append(y.cpu().numpy())
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


def custom_layout(seed, count=300):
    """Signals of 2^6..2^18 elements in shuffled order with gaps: long ones on 32-element
    rows, short ones at any offset."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(6, 19, count).astype(np.uint8)
    off = np.zeros(count, dtype=np.int64)
    o = 0
    for i in rng.permutation(count):
        o += int(rng.integers(0, 40))
        if ms[i] >= 13:
            o = (o + 31) // 32 * 32
        off[i] = o
        o += 1 << int(ms[i])
    return ms, off, o + int(rng.integers(0, 50))


def test_ragged_at_caller_layout_matches_oracle(chw, torch):
    ms, off, total = custom_layout(5)
    x = W.normal_f32(0, total, seed=6).reshape(-1)  # one value per element of the buffer
    xd = torch.from_numpy(x).cuda()
    yd = torch.full((total,), float(SENTINEL), device="cuda")
    p = chw.chw_plan_ragged(ms, "f32", "end", offsets=off, total=total)
    assert np.array_equal(chw.chw_ragged_offsets(p)[:-1], off)
    chw.chw_forward_ragged(p, xd, yd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    y = yd.cpu().numpy()
    covered = np.zeros(total, dtype=bool)
    for i in range(len(ms)):
        n = 1 << int(ms[i])
        seg = slice(off[i], off[i] + n)
        covered[seg] = True
        ref = O.chw_cascade(x[seg][None, :], int(ms[i]), np.float32, "end")[0]
        assert np.array_equal(y[seg].view(np.uint32), ref.view(np.uint32)), i
    assert np.all(y[~covered] == SENTINEL)  # the gaps are never written


def test_ragged_corrupted_offsets_are_caught(chw, torch):
    from paper_1609_06641_gb300 import _lib

    ms, off, total = custom_layout(8, count=120)
    guard = 1 << 23  # the corrupted ranges start 2^20 and 2^21 past total: all inside
    x = W.normal_f32(0, total + guard, seed=9).reshape(-1)
    xbuf = torch.from_numpy(x).cuda()
    ybuf = torch.full((total + guard,), float(SENTINEL), device="cuda")
    xd, yd = xbuf[:total], ybuf[:total]  # the plan's buffers; the guard region follows them
    # the plain checked plan first: every signal exact, CHW_OK
    flags = chw.CHW_FLAG_CHECKED
    p = chw.chw_plan_ragged(ms, "f32", "end", flags, offsets=off, total=total)
    chw.chw_forward_ragged(p, xd, yd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    good = ybuf.cpu().numpy().copy()
    p.close()
    # the corrupted plan: two offsets moved past the end of the buffers on the host
    ybuf.fill_(float(SENTINEL))
    pc = chw.chw_plan_ragged(ms, "f32", "end", flags | chw.CHW_FLAG_TEST_CORRUPT, offsets=off, total=total)
    bad_off = chw.chw_ragged_offsets(pc)[:-1]
    bad = np.nonzero(bad_off != off)[0]
    assert len(bad) == 2 and np.all(bad_off[bad] >= total)
    assert ms[bad[0]] >= 13 or ms[bad[1]] >= 13
    chw.chw_forward_ragged(pc, xd, yd)
    torch.cuda.synchronize()
    st = chw.chw_last_device_status(pc)
    assert st == _lib.CHW_ERR_DEVICE_CHECK
    msg = _lib.load().chw_last_error_message().decode()
    index = int(msg.split("element index ")[1].split()[0])
    assert index >= total, msg
    y = ybuf.cpu().numpy()
    assert np.all(y[total:] == SENTINEL), "a write escaped the checks into the guard region"
    for i in range(len(ms)):
        seg = slice(off[i], off[i] + (1 << int(ms[i])))
        if i in bad:
            assert np.all(y[seg] == SENTINEL), f"signal {i}: written although its offset was corrupted"
        else:
            assert np.array_equal(y[seg].view(np.uint32), good[seg].view(np.uint32)), i
    assert chw.chw_last_device_status(pc) == 0  # the read cleared the latch
