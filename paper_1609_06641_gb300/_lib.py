"""ctypes binding of include/chw.h: the C ABI functions under their own names.

Argument marshalling only; every computation runs in libchw.so's CUDA kernels.  The
library is built in-tree (``paper_1609_06641_gb300/libchw.so``); if it is missing or fails
to load, ``load()`` raises -- there is no fallback implementation.
"""

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchw.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "chw.h")

# chw_status_t
CHW_OK = 0
CHW_ERR_INVALID_ARG = 1
CHW_ERR_UNSUPPORTED = 2
CHW_ERR_ALIGNMENT = 3
CHW_ERR_OOM = 4
CHW_ERR_CUDA = 5
CHW_ERR_TIMEOUT = 6
CHW_ERR_DEVICE_CHECK = 7
# chw_dtype_t
CHW_I32, CHW_F32, CHW_BF16, CHW_F16 = 0, 1, 2, 3
# chw_norm_t
CHW_NORM_NONE, CHW_NORM_PER_LEVEL, CHW_NORM_END = 0, 1, 2
CHW_MAX_M = 30
CHW_FLAG_NONE = 0
CHW_FLAG_FORCE_SIMPLE = 1
CHW_FLAG_FORCE_MULTIPASS = 2
CHW_FLAG_ROWSTACK = 4
CHW_FLAG_HAAR_WALSH = 8
CHW_FLAG_ORDER_NATURAL = 16
CHW_FLAG_ORDER_SEQUENCY = 32
CHW_FLAG_TEST_STALL = 64
CHW_FLAG_CLUSTER = 128
CHW_FLAG_AUTOTUNE = 256
CHW_FLAG_CHECKED = 512
CHW_FLAG_TEST_CORRUPT = 1024


class chw_plan_info_t(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int),
        ("batch", ctypes.c_int64),
        ("dtype", ctypes.c_int),
        ("norm", ctypes.c_int),
        ("tier", ctypes.c_int),
        ("passes", ctypes.c_int),
        ("row_bits", ctypes.c_int),
        ("cluster", ctypes.c_int),
        ("kernels_per_call", ctypes.c_int),
        ("workspace_bytes", ctypes.c_int64),
        ("total_elements", ctypes.c_int64),
        ("order", ctypes.c_int),
        ("tile_bits", ctypes.c_int),
        ("tuned", ctypes.c_int),
        ("tune_us", ctypes.c_float),
    ]


class chw_tune_choice_t(ctypes.Structure):
    _fields_ = [("tier", ctypes.c_int), ("row_bits", ctypes.c_int), ("tile_bits", ctypes.c_int)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "chw_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32]),
    "chw_plan_ragged": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32]),
    "chw_plan_ragged_at": (
        ctypes.c_int,
        [ctypes.POINTER(_P), _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32],
    ),
    "chw_ragged_offsets": (ctypes.c_int, [_P, _P]),
    "chw_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "chw_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "chw_forward_ragged": (ctypes.c_int, [_P, _P, _P, _P]),
    "chw_forward_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "chw_haar": (ctypes.c_int, [_P, _P, _P, _P]),
    "chw_haar_inverse": (ctypes.c_int, [_P, _P, _P, _P]),
    "chw_from_haar": (ctypes.c_int, [_P, _P, _P, _P]),
    "chw_forward_haar": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "chw_forward_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "chw_noalloc_device_status": (ctypes.c_int, []),
    "chw_plan_get_info": (ctypes.c_int, [_P, ctypes.POINTER(chw_plan_info_t)]),
    "chw_last_device_status": (ctypes.c_int, [_P]),
    "chw_plan_destroy": (ctypes.c_int, [_P]),
    "chw_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "chw_last_error_message": (ctypes.c_char_p, []),
    "chw_tune_candidates": (
        ctypes.c_int,
        [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(chw_tune_choice_t), ctypes.c_int],
    ),
    "chw_tune_cache_put": (
        ctypes.c_int,
        [ctypes.c_char_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
         ctypes.POINTER(chw_tune_choice_t), ctypes.c_float],
    ),
    "chw_tune_cache_get": (
        ctypes.c_int,
        [ctypes.c_char_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
         ctypes.POINTER(chw_tune_choice_t), ctypes.POINTER(ctypes.c_float)],
    ),
    "chw_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "chw_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "chw_tune_cache_clear": (None, []),
}

_lib = None


def header_functions():
    """Names of the functions declared in include/chw.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chw_[a-z_]+)\s*\(", text)))


def load(path=None):
    """Load libchw.so (once) and attach the C signatures; raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_1609_06641_gb300.build` "
            "(there is no fallback implementation)"
        )
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class ChwError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        self.status = status
        msg = lib.chw_last_error_message().decode()
        super().__init__(f"{where}: {lib.chw_status_string(status).decode()} ({msg})")


def check(status, where):
    if status != CHW_OK:
        raise ChwError(status, where)
