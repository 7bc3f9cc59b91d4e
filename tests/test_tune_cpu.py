"""Autotuner host logic (no GPU): candidate enumeration and the choice cache.

The candidates are the configurations a plan of a given shape can run; every one of them
is a compiled kernel combination (the enumeration looks each one up), so the tuner only
ever times runnable configurations.  The cache maps (device, m, floor(log2 batch), dtype,
norm, order) to a choice and survives a save/load round trip through its text file.
"""

import pytest

TIER_FUSED, TIER_CLUSTER, TIER_TWO_PASS, TIER_ROWSTACK, TIER_TMEM, TIER_TMEM_CROSS = 1, 2, 3, 6, 7, 8


@pytest.fixture(scope="module")
def chw():
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import build

    build.build()
    chw._lib.load()
    return chw


@pytest.mark.parametrize("m", [0, 5, 10, 13])
def test_single_configuration_shapes_have_no_candidates(chw, m):
    for order in ("dyadic", "natural", "sequency"):
        assert chw.chw_tune_candidates(m, "f32", "end", order=order) == []


def test_fixed_tier_flags_and_16bit_have_no_candidates(chw):
    for fl in (chw.CHW_FLAG_FORCE_SIMPLE, chw.CHW_FLAG_FORCE_MULTIPASS, chw.CHW_FLAG_ROWSTACK,
               chw.CHW_FLAG_CLUSTER, chw.CHW_FLAG_TEST_STALL):
        assert chw.chw_tune_candidates(16, "f32", "end", flags=fl) == []
    assert chw.chw_tune_candidates(12, "bf16", "end") == []
    assert chw.chw_tune_candidates(30, "f32", "end") == []


@pytest.mark.parametrize("m", [15, 16])
def test_one_pass_shapes_are_not_tuned(chw, m):
    # the tensor-memory kernel is the only candidate (the cluster and row-stack tiers, far
    # slower, stay selectable by their flags): nothing to choose in any order
    for order in ("dyadic", "natural", "sequency"):
        assert chw.chw_tune_candidates(m, "f32", "end", order=order) == []
        assert chw.chw_tune_candidates(m, "i32", "none", order=order) == []


def test_m14_and_m17_one_pass_candidates(chw):
    assert (TIER_FUSED, 14, 14) in chw.chw_tune_candidates(14, "f32", "end")
    c17 = chw.chw_tune_candidates(17, "f32", "end")
    assert (TIER_CLUSTER, 17, 14) in c17 and all(t != TIER_ROWSTACK for t, _, _ in c17)
    # the pair of SMs holding the signal in tensor memory: dyadic order only
    assert (TIER_TMEM_CROSS, 17, 0) in c17
    assert (TIER_TMEM_CROSS, 17, 0) in chw.chw_tune_candidates(17, "i32", "none")
    for order in ("natural", "sequency"):
        assert all(t != TIER_TMEM_CROSS for t, _, _ in chw.chw_tune_candidates(17, "f32", "end", order=order))


@pytest.mark.parametrize("m", [17, 18, 20, 23, 24, 28, 29, 30])
@pytest.mark.parametrize("order", ["dyadic", "natural", "sequency"])
def test_two_pass_candidates_are_valid_splits(chw, m, order):
    c = chw.chw_tune_candidates(m, "f32", "per_level", order=order)
    if order == "natural" and m >= 23:
        assert c == []  # m = 23: a = 9, b = 14 is the only natural split compiled; beyond: none
        return
    if m == 30 or (m == 29 and order == "sequency"):
        # one configuration, nothing to choose: dyadic m = 30 has only the split a = 14,
        # b = 16; sequency order's column kernels take a <= 12 and its row kernels b <= 17
        # (m = 29: a = 12 only; m = 30: none)
        assert c == []
        return
    two = [x for x in c if x[0] == TIER_TWO_PASS]
    assert two, (m, order)
    for _, b, tb in two:
        a = m - b
        assert 6 <= a <= 14 and 5 <= b <= 17 and tb in (13, 14)
        if a > 12:  # only tensor-memory column tiles (narrow blocks) take a = 13, 14, after
            assert order == "dyadic" and b in (15, 16) and tb == 14  # a tensor-memory first pass
        if order == "natural":
            assert b <= 14 and a <= 9  # the natural-order kernels that exist
    if order == "dyadic" and m >= 26:
        assert (TIER_TWO_PASS, 16, 14) in c  # the built-in split a = m - 16
    assert len(set(c)) == len(c)
    if m == 17 and order != "natural":
        assert (TIER_CLUSTER, 17, 14) in c


def test_cache_put_get_bucket_and_keys(chw):
    chw.chw_tune_cache_clear()
    dev = "NVIDIA GB300 test"
    assert chw.chw_tune_cache_get(dev, 16, 4096, "f32", "end") is None
    chw.chw_tune_cache_put(dev, 16, 4096, "f32", "end", (TIER_TMEM, 16, 0), 350.5)
    got = chw.chw_tune_cache_get(dev, 16, 5000, "f32", "end")  # same bucket: floor(log2) = 12
    assert got is not None and got[0] == (TIER_TMEM, 16, 0) and abs(got[1] - 350.5) < 1e-3
    assert chw.chw_tune_cache_get(dev, 16, 8192, "f32", "end") is None  # next bucket
    assert chw.chw_tune_cache_get(dev, 16, 4096, "f32", "per_level") is None
    assert chw.chw_tune_cache_get(dev, 16, 4096, "f32", "end", order="natural") is None
    assert chw.chw_tune_cache_get("other device", 16, 4096, "f32", "end") is None
    chw.chw_tune_cache_clear()
    assert chw.chw_tune_cache_get(dev, 16, 4096, "f32", "end") is None


def test_cache_file_round_trip_and_malformed_lines(chw, tmp_path):
    chw.chw_tune_cache_clear()
    dev = "NVIDIA GB300"
    chw.chw_tune_cache_put(dev, 20, 256, "f32", "end", (TIER_TWO_PASS, 11, 14), 700.25)
    chw.chw_tune_cache_put(dev, 17, 2048, "i32", "none", (TIER_CLUSTER, 17, 14), 812.0, order="sequency")
    path = tmp_path / "tune.txt"
    chw.chw_tune_cache_save(str(path))
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and all(l.startswith("chw-tune-v1 ") for l in lines)
    chw.chw_tune_cache_clear()
    with open(path, "a") as f:
        f.write("garbage line\n")
        f.write("chw-tune-v1 k tier=3 row_bits=99 tile_bits=14 us=1.0\n")  # row_bits out of range
        f.write("chw-tune-v1 k2 tier=3 row_bits=9 tile_bits=12 us=1.0\n")  # tile bits neither 13 nor 14
    assert chw.chw_tune_cache_load(str(path)) == 2
    got = chw.chw_tune_cache_get(dev, 20, 300, "f32", "end")
    assert got is not None and got[0] == (TIER_TWO_PASS, 11, 14)
    got = chw.chw_tune_cache_get(dev, 17, 2048, "i32", "none", order="sequency")
    assert got is not None and got[0] == (TIER_CLUSTER, 17, 14)
    assert chw.chw_tune_cache_load(str(tmp_path / "missing.txt")) == -1
    chw.chw_tune_cache_clear()


def test_cache_argument_errors(chw):
    from paper_1609_06641_gb300 import _lib

    with pytest.raises(_lib.ChwError):
        chw.chw_tune_cache_put("dev", 16, 0, "f32", "end", (TIER_TMEM, 16, 0), 1.0)
    with pytest.raises(_lib.ChwError):
        chw.chw_tune_cache_save("/nonexistent-dir/x/tune.txt")
