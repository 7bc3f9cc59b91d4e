"""Autotuned plans (GPU): the tuner times every candidate, keeps one, caches it, and the
plan it makes computes the same bits as the oracle's cascade."""

import os

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_bitwise
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORACLE_DT = {"f32": np.float32, "i32": np.int32}


@pytest.fixture(scope="module")
def chw(cuda_device, tmp_path_factory):
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    # read once per process, on the first autotuned plan
    os.environ["CHW_TUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "cache.txt")
    chw.chw_tune_cache_clear()
    return chw


def _x(m, batch, dtype, seed):
    if dtype == "i32":
        return W.uniform_int32(m, batch, seed, bound=1 << max(1, 29 - m))
    return W.normal_f32(m, batch, seed)


def _forward(chw, p, x):
    import torch

    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    chw.chw_forward(p, xd, yd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    return yd.cpu().numpy()


CASES = [
    (14, 40, "f32", "end", "dyadic"),
    (18, 5, "f32", "end", "dyadic"),
    (20, 3, "i32", "none", "sequency"),
    (17, 6, "f32", "per_level", "dyadic"),
    (17, 4, "f32", "end", "natural"),
    (19, 3, "i32", "none", "dyadic"),
    (21, 2, "f32", "end", "sequency"),
]


@pytest.mark.parametrize("m,batch,dtype,norm,order", CASES)
def test_autotuned_plan_is_bit_exact_and_cached(chw, m, batch, dtype, norm, order):
    cands = chw.chw_tune_candidates(m, dtype, norm, order=order)
    assert len(cands) >= 2
    p = chw.chw_plan(m, batch, dtype, norm, chw.CHW_FLAG_AUTOTUNE, order=order)
    info = chw.chw_plan_get_info(p)
    assert info.tuned == 1 and info.tune_us > 0
    assert (info.tier, info.row_bits, info.tile_bits) in cands
    assert info.passes == (2 if info.tier == 3 else 1)
    x = _x(m, batch, dtype, 9000 + m)
    y = _forward(chw, p, x)
    assert_bitwise(y, O.wht_ordered(x, m, order, ORACLE_DT[dtype], norm), f"tuned m={m} {order} {info.tier}")
    # the same key again: the cached choice, no timing
    p2 = chw.chw_plan(m, batch, dtype, norm, chw.CHW_FLAG_AUTOTUNE, order=order)
    i2 = chw.chw_plan_get_info(p2)
    assert i2.tuned == 2 and (i2.tier, i2.row_bits, i2.tile_bits) == (info.tier, info.row_bits, info.tile_bits)
    text = open(os.environ["CHW_TUNE_CACHE"]).read()
    assert f":m{m}:" in text


def test_every_candidate_is_bit_exact(chw):
    # the tuner may pick any candidate, so each must compute the cascade exactly: apply each
    # one through the cache and run it
    import torch

    m, batch = 17, 3
    x = W.normal_f32(m, batch, 9100)
    ref = O.chw_cascade(x, m, np.float32, "end")
    dev = torch.cuda.get_device_name(0)
    for cand in chw.chw_tune_candidates(m, "f32", "end"):
        chw.chw_tune_cache_put(dev, m, batch, "f32", "end", cand, 1.0)
        p = chw.chw_plan(m, batch, "f32", "end", chw.CHW_FLAG_AUTOTUNE)
        info = chw.chw_plan_get_info(p)
        assert info.tuned == 2 and (info.tier, info.row_bits, info.tile_bits) == cand
        assert_bitwise(_forward(chw, p, x), ref, f"candidate {cand}")


def test_single_configuration_is_not_timed(chw):
    p = chw.chw_plan(12, 8, "f32", "end", chw.CHW_FLAG_AUTOTUNE)
    assert chw.chw_plan_get_info(p).tuned == 0
    # m = 16: the tensor-memory kernel is the only candidate
    p16 = chw.chw_plan(16, 8, "f32", "end", chw.CHW_FLAG_AUTOTUNE)
    i16 = chw.chw_plan_get_info(p16)
    assert i16.tuned == 0 and i16.tier == 7


def test_tuned_ragged_plan_is_bit_exact(chw):
    import torch

    rng = np.random.default_rng(21)
    ms = np.concatenate([np.full(6, 15), np.full(5, 16), np.full(4, 17), np.full(3, 18), np.full(2, 20),
                         rng.integers(0, 15, 20)]).astype(np.uint8)
    rng.shuffle(ms)
    p = chw.chw_plan_ragged(ms, "f32", "end", chw.CHW_FLAG_AUTOTUNE)
    assert chw.chw_plan_get_info(p).tuned == 1
    off = chw.chw_ragged_offsets(p)
    x = rng.standard_normal(int(off[-1])).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    chw.chw_forward_ragged(p, xd, yd)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    y = yd.cpu().numpy()
    for i, m in enumerate(ms):
        seg = x[off[i]: off[i] + (1 << int(m))][None, :]
        assert_bitwise(y[off[i]: off[i] + seg.size], O.chw_cascade(seg, int(m), np.float32, "end")[0], f"signal {i} m={m}")


@pytest.mark.parametrize("m,b", [(21, 15), (22, 16), (24, 15), (24, 16), (25, 16)])
@pytest.mark.parametrize("dtype,norm", [("f32", "end"), ("f32", "per_level"), ("i32", "none")])
def test_two_pass_with_tensor_memory_rows(chw, m, b, dtype, norm):
    # the first pass on rows of 2^15 or 2^16 words runs on the tensor-memory kernel
    # (column-blocked output); forced through the cache so each split is exercised
    import torch

    batch = 2
    choice = (3, b, 14)
    assert choice in chw.chw_tune_candidates(m, dtype, norm)
    chw.chw_tune_cache_put(torch.cuda.get_device_name(0), m, batch, dtype, norm, choice, 1.0)
    p = chw.chw_plan(m, batch, dtype, norm, chw.CHW_FLAG_AUTOTUNE)
    info = chw.chw_plan_get_info(p)
    assert info.tuned == 2 and info.row_bits == b and info.cluster == 1
    x = _x(m, batch, dtype, 9200 + m)
    y = _forward(chw, p, x)
    assert_bitwise(y[1:], O.chw_cascade(x[1:], m, ORACLE_DT[dtype], norm), f"m={m} b={b} {dtype} {norm}")


@pytest.mark.parametrize("m", [28, 29])
def test_dense_narrow_column_blocks_equal_cluster_rows(chw, m):
    # The default split writes blocks of 2^(16 - a) columns (m = 28: 16, m = 29: 8) by TMA
    # tensor stores; every split rounds identically, so the split with 2^17-word cluster
    # rows in the first pass (its own store path, 32-column blocks), forced through the
    # cache, must give the same bits on a dense signal.
    import torch

    dev = torch.device("cuda:0")
    x = torch.from_numpy(W.uniform_pm1_f32(m, 1, seed=5)).to(dev)
    y = torch.empty_like(x)
    p = chw.chw_plan(m, 1, "f32", "per_level")
    assert chw.chw_plan_get_info(p).row_bits == 16
    chw.chw_forward(p, x, y)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(p) == 0
    p.close()
    choice = (3, 17, 14)  # two passes, b = 17 (8-CTA cluster rows), 2^14-word tiles
    assert choice in chw.chw_tune_candidates(m, "f32", "per_level")
    chw.chw_tune_cache_put(torch.cuda.get_device_name(0), m, 1, "f32", "per_level", choice, 1.0)
    q = chw.chw_plan(m, 1, "f32", "per_level", chw.CHW_FLAG_AUTOTUNE)
    info = chw.chw_plan_get_info(q)
    assert (info.tier, info.row_bits, info.tile_bits) == choice and info.tuned == 2
    y2 = torch.empty_like(x)
    chw.chw_forward(q, x, y2)
    torch.cuda.synchronize()
    assert chw.chw_last_device_status(q) == 0
    assert torch.equal(y.view(torch.int32), y2.view(torch.int32))
