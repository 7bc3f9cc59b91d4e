"""The C ABI library loads and exports every function include/chw.h declares (no GPU needed).

Only host-side argument validation runs here; it returns before any CUDA call, so the
results do not depend on a device being present.
"""

import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1609_06641_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_every_declared_function_is_exported(lib):
    from paper_1609_06641_gb300 import _lib

    names = _lib.header_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    assert set(names) == set(_lib._SIGNATURES), "the ctypes binding covers exactly the header"


def test_status_strings(lib):
    for code in range(8):
        s = lib.chw_status_string(code).decode()
        assert s.startswith("CHW_")
    assert "unknown" in lib.chw_status_string(99).decode()


@pytest.mark.parametrize(
    "m,batch,dtype,norm",
    [(-1, 1, 1, 1), (31, 1, 1, 1), (4, 0, 1, 1), (4, 1, 7, 1), (4, 1, 1, 9), (4, 1, 0, 1), (4, 1, 0, 2), (4, 1, 2, 0)],
)
def test_plan_argument_validation(lib, m, batch, dtype, norm):
    from paper_1609_06641_gb300 import _lib

    h = ctypes.c_void_p(123)
    st = lib.chw_plan(ctypes.byref(h), m, batch, dtype, norm, 0)
    assert st == _lib.CHW_ERR_INVALID_ARG
    assert h.value is None
    assert lib.chw_last_error_message().decode() != ""


def test_null_handles(lib):
    from paper_1609_06641_gb300 import _lib

    assert lib.chw_plan(None, 4, 1, 1, 1, 0) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward(None, None, None, None, None, None, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_adjoint(None, None, None, None, None, None, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward_ragged(None, None, None, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward_host(None, None, None, None, None, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_plan_get_info(None, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_last_device_status(None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_plan_destroy(None) == _lib.CHW_OK
    assert lib.chw_plan_ragged(None, None, 0, 1, 1, 0) == _lib.CHW_ERR_INVALID_ARG


def test_ragged_plan_validation(lib):
    import numpy as np

    from paper_1609_06641_gb300 import _lib

    h = ctypes.c_void_p()
    bad = np.array([3, 21], dtype=np.uint8)
    st = lib.chw_plan_ragged(ctypes.byref(h), bad.ctypes.data_as(ctypes.c_void_p), 2, 1, 1, 0)
    assert st == _lib.CHW_ERR_INVALID_ARG
    ok = np.array([3, 4], dtype=np.uint8)
    st = lib.chw_plan_ragged(ctypes.byref(h), ok.ctypes.data_as(ctypes.c_void_p), 2, 2, 2, 0)
    assert st == _lib.CHW_ERR_UNSUPPORTED  # ragged batches take int32 or fp32


def test_loader_raises_without_library(tmp_path, monkeypatch):
    from paper_1609_06641_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback implementation"):
        _lib.load(str(tmp_path / "missing.so"))


def test_noalloc_rejects_before_any_cuda_call(lib):
    """chw_forward_noalloc validates sizes on the host and reports the reason."""
    from paper_1609_06641_gb300 import _lib

    p = ctypes.c_void_p(4096)
    assert lib.chw_forward_noalloc(17, 1, _lib.CHW_F32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_UNSUPPORTED
    assert "18 <= m <= 22" in lib.chw_last_error_message().decode()
    assert lib.chw_forward_noalloc(20, 5, _lib.CHW_F32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_INVALID_ARG
    assert "2^22" in lib.chw_last_error_message().decode()
    assert lib.chw_forward_noalloc(20, 1, _lib.CHW_I32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward_noalloc(20, 1, _lib.CHW_F32, _lib.CHW_NORM_END, None, p, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward_noalloc(20, 1, _lib.CHW_F32, _lib.CHW_NORM_END, ctypes.c_void_p(4100), p, None) == _lib.CHW_ERR_ALIGNMENT


def test_ragged_at_validates_layout_on_the_host(lib):
    """chw_plan_ragged_at rejects signals outside [0, total), overlaps and TMA-misaligned
    long signals before anything is allocated or uploaded."""
    import numpy as np

    from paper_1609_06641_gb300 import _lib

    def plan_at(ms, off, total, flags=0):
        h = ctypes.c_void_p(7)
        ms = np.asarray(ms, dtype=np.uint8)
        off = np.asarray(off, dtype=np.int64)
        st = lib.chw_plan_ragged_at(ctypes.byref(h), ms.ctypes.data_as(ctypes.c_void_p),
                                    off.ctypes.data_as(ctypes.c_void_p), len(ms), total, _lib.CHW_F32,
                                    _lib.CHW_NORM_END, flags)
        assert h.value is None
        return st

    assert plan_at([6, 6], [0, 100], 150) == _lib.CHW_ERR_INVALID_ARG  # second ends at 164 > 150
    assert plan_at([6, 6], [0, -4], 1000) == _lib.CHW_ERR_INVALID_ARG
    assert plan_at([6, 7], [0, 40], 1000) == _lib.CHW_ERR_INVALID_ARG  # [0, 64) and [40, 168) overlap
    assert "overlap" in lib.chw_last_error_message().decode()
    assert plan_at([13], [16], 1 << 14) == _lib.CHW_ERR_ALIGNMENT  # a TMA signal off a 32-element row
    assert plan_at([6], [0], 0) == _lib.CHW_ERR_INVALID_ARG
    # the corruption hook runs only with the checked mode
    assert plan_at([13], [0], 1 << 13, _lib.CHW_FLAG_TEST_CORRUPT) == _lib.CHW_ERR_INVALID_ARG
    assert "CHW_FLAG_CHECKED" in lib.chw_last_error_message().decode()
    h = ctypes.c_void_p(7)
    ms = np.array([13], dtype=np.uint8)
    st = lib.chw_plan_ragged(ctypes.byref(h), ms.ctypes.data_as(ctypes.c_void_p), 1, _lib.CHW_F32,
                             _lib.CHW_NORM_END, _lib.CHW_FLAG_TEST_CORRUPT)
    assert st == _lib.CHW_ERR_INVALID_ARG and h.value is None
    st = lib.chw_plan(ctypes.byref(h), 10, 4, _lib.CHW_F32, _lib.CHW_NORM_END, _lib.CHW_FLAG_TEST_CORRUPT)
    assert st == _lib.CHW_ERR_INVALID_ARG and h.value is None
