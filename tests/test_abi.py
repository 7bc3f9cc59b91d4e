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
