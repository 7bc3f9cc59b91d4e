"""GB300 (sm_103a) Cascading Haar Wavelet Walsh-Hadamard transform.

Python side of the C ABI in include/chw.h.  The functions keep the C names (``chw_plan``,
``chw_forward``, ``chw_adjoint``, ``chw_forward_ragged``, ``chw_haar``, ``chw_from_haar``, ...) and only marshal
arguments: tensors must already live on the GPU (PyTorch is used for device memory and
streams), and every step of the transform runs in the library's CUDA kernels.  There is
no CPU fallback; a missing library raises.

    import torch, paper_1609_06641_gb300 as chw
    p = chw.chw_plan(16, 4096, "f32", "end")
    y = torch.empty_like(x)
    chw.chw_forward(p, x, y)          # y = H_16 x for every row of x (dyadic order)
"""

import ctypes
import os

from . import _lib
from ._lib import (
    CHW_BF16,
    CHW_F16,
    CHW_F32,
    CHW_FLAG_AUTOTUNE,
    CHW_FLAG_CHECKED,
    CHW_FLAG_CLUSTER,
    CHW_FLAG_HAAR_WALSH,
    CHW_FLAG_ORDER_NATURAL,
    CHW_FLAG_ORDER_SEQUENCY,
    CHW_FLAG_ROWSTACK,
    CHW_FLAG_TEST_CORRUPT,
    CHW_FLAG_TEST_STALL,
    CHW_FLAG_FORCE_MULTIPASS,
    CHW_FLAG_FORCE_SIMPLE,
    CHW_FLAG_NONE,
    CHW_I32,
    CHW_MAX_M,
    CHW_NORM_END,
    CHW_NORM_NONE,
    CHW_NORM_PER_LEVEL,
    ChwError,
)

DTYPES = {"i32": CHW_I32, "f32": CHW_F32, "bf16": CHW_BF16, "f16": CHW_F16}
NORMS = {"none": CHW_NORM_NONE, "per_level": CHW_NORM_PER_LEVEL, "end": CHW_NORM_END}
ORDERS = {"dyadic": 0, "natural": CHW_FLAG_ORDER_NATURAL, "sequency": CHW_FLAG_ORDER_SEQUENCY}
TIERS = {
    0: "simple",
    1: "fused",
    2: "cluster",
    3: "two-pass",
    4: "ragged",
    5: "fused-16bit",
    6: "row-stack",
    7: "tensor-memory",
    8: "tensor-memory-pair",
}


def _torch_dtype(code):
    import torch

    return {CHW_I32: torch.int32, CHW_F32: torch.float32, CHW_BF16: torch.bfloat16, CHW_F16: torch.float16}[code]


class Plan:
    """Owns a chw_plan_t; released by ``close()`` or when garbage-collected."""

    def __init__(self, handle, m, batch, dtype, norm, ragged_ms=None):
        self.handle = handle
        self.m = m
        self.batch = batch
        self.dtype = dtype
        self.norm = norm
        self.ragged_ms = ragged_ms

    @property
    def torch_dtype(self):
        return _torch_dtype(self.dtype)

    def info(self):
        return chw_plan_get_info(self)

    def close(self):
        if self.handle:
            _lib.load().chw_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _code(v, table, what):
    if isinstance(v, str):
        if v not in table:
            raise ValueError(f"unknown {what} {v!r}; expected one of {sorted(table)}")
        return table[v]
    return int(v)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check_data(t, plan, name, numel):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype != plan.torch_dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, the plan computes {plan.torch_dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, the plan needs {numel}")


def chw_plan(m, batch, dtype="f32", norm="end", flags=CHW_FLAG_NONE, order="dyadic"):
    """Plan y = H_m x for ``batch`` signals of 2^m elements (see chw_plan in chw.h).

    ``order`` ("dyadic", "natural" or "sequency") adds the matching CHW_FLAG_ORDER_* flag.
    """
    lib = _lib.load()
    h = ctypes.c_void_p()
    d = _code(dtype, DTYPES, "dtype")
    nm = _code(norm, NORMS, "norm")
    flags = int(flags) | _code(order, ORDERS, "order")
    _lib.check(lib.chw_plan(ctypes.byref(h), int(m), int(batch), d, nm, flags), "chw_plan")
    return Plan(h, int(m), int(batch), d, nm)


def chw_plan_ragged(ms, dtype="f32", norm="end", flags=CHW_FLAG_NONE, offsets=None, total=None):
    """Plan one graph launch over signals of lengths 2^ms[i] (see chw_plan_ragged).

    With ``offsets`` (one element offset per signal) and ``total`` (elements of x and y) the
    signals sit where the caller put them (chw_plan_ragged_at); otherwise the library packs
    them (chw_ragged_offsets)."""
    import numpy as np

    lib = _lib.load()
    arr = np.ascontiguousarray(np.asarray(ms, dtype=np.uint8))
    h = ctypes.c_void_p()
    d = _code(dtype, DTYPES, "dtype")
    nm = _code(norm, NORMS, "norm")
    if offsets is None:
        _lib.check(
            lib.chw_plan_ragged(ctypes.byref(h), arr.ctypes.data_as(ctypes.c_void_p), arr.size, d, nm, int(flags)),
            "chw_plan_ragged",
        )
    else:
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        if off.size != arr.size or total is None:
            raise ValueError("offsets needs one entry per signal, and total")
        _lib.check(
            lib.chw_plan_ragged_at(ctypes.byref(h), arr.ctypes.data_as(ctypes.c_void_p),
                                   off.ctypes.data_as(ctypes.c_void_p), arr.size, int(total), d, nm, int(flags)),
            "chw_plan_ragged_at",
        )
    return Plan(h, -1, int(arr.size), d, nm, ragged_ms=arr)


def chw_ragged_offsets(plan):
    """Element offsets of a ragged plan's signals (count + 1 entries, numpy int64)."""
    import numpy as np

    out = np.zeros(plan.batch + 1, dtype=np.int64)
    _lib.check(_lib.load().chw_ragged_offsets(plan.handle, out.ctypes.data_as(ctypes.c_void_p)), "chw_ragged_offsets")
    return out


def _exp_args(plan, exp_in, exp_out):
    lowp = plan.dtype in (CHW_BF16, CHW_F16)
    if lowp:
        import torch

        for name, e in (("exp_in", exp_in), ("exp_out", exp_out)):
            if e is None or e.dtype != torch.int32 or not e.is_cuda or e.numel() != plan.batch or not e.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA int32 tensor of {plan.batch} exponents")
    return _ptr(exp_in), _ptr(exp_out)


def _diag_arg(plan, diag):
    if diag is None:
        return ctypes.c_void_p(0)
    import torch

    if diag.dtype != torch.int8 or not diag.is_cuda or diag.numel() != (1 << plan.m) or not diag.is_contiguous():
        raise ValueError("diag must be a contiguous CUDA int8 tensor of 2^m entries (+-1)")
    return _ptr(diag)


def chw_forward(plan, x, y, exp_in=None, exp_out=None, diag=None, stream=None):
    """y = D H_m x on the GPU (asynchronous on ``stream``, default: current stream)."""
    n = plan.batch << plan.m
    _check_data(x, plan, "x", n)
    _check_data(y, plan, "y", n)
    ei, eo = _exp_args(plan, exp_in, exp_out)
    st = _lib.load().chw_forward(plan.handle, _ptr(x), _ptr(y), ei, eo, _diag_arg(plan, diag), _stream(stream))
    _lib.check(st, "chw_forward")
    return y


def chw_adjoint(plan, y, x, exp_in=None, exp_out=None, diag=None, stream=None):
    """x = H_m^T D y on the GPU."""
    n = plan.batch << plan.m
    _check_data(y, plan, "y", n)
    _check_data(x, plan, "x", n)
    ei, eo = _exp_args(plan, exp_in, exp_out)
    st = _lib.load().chw_adjoint(plan.handle, _ptr(y), _ptr(x), ei, eo, _diag_arg(plan, diag), _stream(stream))
    _lib.check(st, "chw_adjoint")
    return x


def chw_forward_ragged(plan, x, y, stream=None):
    """Transform every signal of a ragged plan (packed at chw_ragged_offsets)."""
    total = int(chw_plan_get_info(plan).total_elements)
    _check_data(x, plan, "x", total)
    _check_data(y, plan, "y", total)
    _lib.check(_lib.load().chw_forward_ragged(plan.handle, _ptr(x), _ptr(y), _stream(stream)), "chw_forward_ragged")
    return y


def _check_batched(plan, where):
    if plan.m < 0:
        raise ValueError(f"{where} takes a batched plan, not a ragged one")


def chw_haar(plan, x, z, stream=None):
    """z = Psi_m x, the Haar transform of eq. (2) (layout in chw.h); x and z must not overlap."""
    _check_batched(plan, "chw_haar")
    n = plan.batch << plan.m
    _check_data(x, plan, "x", n)
    _check_data(z, plan, "z", n)
    _lib.check(_lib.load().chw_haar(plan.handle, _ptr(x), _ptr(z), _stream(stream)), "chw_haar")
    return z


def chw_haar_inverse(plan, z, x, stream=None):
    """x = Psi_m^T z; z and x must not overlap."""
    _check_batched(plan, "chw_haar_inverse")
    n = plan.batch << plan.m
    _check_data(z, plan, "z", n)
    _check_data(x, plan, "x", n)
    _lib.check(_lib.load().chw_haar_inverse(plan.handle, _ptr(z), _ptr(x), _stream(stream)), "chw_haar_inverse")
    return x


def chw_from_haar(plan, z, y, stream=None):
    """y = H_m Psi_m^T z, the Haar-Walsh transform of eq. (4) (plan needs CHW_FLAG_HAAR_WALSH)."""
    _check_batched(plan, "chw_from_haar")
    n = plan.batch << plan.m
    _check_data(z, plan, "z", n)
    _check_data(y, plan, "y", n)
    _lib.check(_lib.load().chw_from_haar(plan.handle, _ptr(z), _ptr(y), _stream(stream)), "chw_from_haar")
    return y


def chw_forward_haar(plan, x, y, z, stream=None):
    """y = H_m x with the Haar side output z = Psi_m x (plan needs CHW_FLAG_HAAR_WALSH)."""
    _check_batched(plan, "chw_forward_haar")
    n = plan.batch << plan.m
    for name, t in (("x", x), ("y", y), ("z", z)):
        _check_data(t, plan, name, n)
    _lib.check(_lib.load().chw_forward_haar(plan.handle, _ptr(x), _ptr(y), _ptr(z), _stream(stream)), "chw_forward_haar")
    return y


def chw_forward_host(plan, x_host, y_host, exp_in_host=None, exp_out_host=None, diag_host=None):
    """y_host = D H_m x_host for HOST tensors/arrays (copies and pipelining inside the call)."""

    def hp(a):
        if a is None:
            return ctypes.c_void_p(0)
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors")
            return ctypes.c_void_p(a.data_ptr())
        return a.ctypes.data_as(ctypes.c_void_p)

    st = _lib.load().chw_forward_host(plan.handle, hp(x_host), hp(y_host), hp(exp_in_host), hp(exp_out_host), hp(diag_host))
    _lib.check(st, "chw_forward_host")
    return y_host


def chw_plan_get_info(plan):
    info = _lib.chw_plan_info_t()
    _lib.check(_lib.load().chw_plan_get_info(plan.handle, ctypes.byref(info)), "chw_plan_get_info")
    return info


def chw_tune_candidates(m, dtype="f32", norm="end", flags=CHW_FLAG_NONE, order="dyadic"):
    """Configurations the autotuner times for this shape: a list of (tier, row_bits, tile_bits)."""
    lib = _lib.load()
    d = _code(dtype, DTYPES, "dtype")
    nm = _code(norm, NORMS, "norm")
    fl = int(flags) | _code(order, ORDERS, "order")
    n = lib.chw_tune_candidates(int(m), d, nm, fl, None, 0)
    arr = (_lib.chw_tune_choice_t * max(n, 1))()
    lib.chw_tune_candidates(int(m), d, nm, fl, arr, n)
    return [(c.tier, c.row_bits, c.tile_bits) for c in arr[:n]]


def chw_tune_cache_put(device, m, batch, dtype, norm, choice, us, flags=CHW_FLAG_NONE, order="dyadic"):
    """Set the autotuner's cache entry of a key; ``choice`` = (tier, row_bits, tile_bits)."""
    c = _lib.chw_tune_choice_t(*[int(v) for v in choice])
    fl = int(flags) | _code(order, ORDERS, "order")
    _lib.check(
        _lib.load().chw_tune_cache_put(device.encode(), int(m), int(batch), _code(dtype, DTYPES, "dtype"),
                                       _code(norm, NORMS, "norm"), fl, ctypes.byref(c), float(us)),
        "chw_tune_cache_put",
    )


def chw_tune_cache_get(device, m, batch, dtype, norm, flags=CHW_FLAG_NONE, order="dyadic"):
    """The cached (tier, row_bits, tile_bits) and time of a key, or None."""
    c = _lib.chw_tune_choice_t()
    us = ctypes.c_float()
    fl = int(flags) | _code(order, ORDERS, "order")
    st = _lib.load().chw_tune_cache_get(device.encode(), int(m), int(batch), _code(dtype, DTYPES, "dtype"),
                                        _code(norm, NORMS, "norm"), fl, ctypes.byref(c), ctypes.byref(us))
    if st == _lib.CHW_ERR_UNSUPPORTED:
        return None
    _lib.check(st, "chw_tune_cache_get")
    return (c.tier, c.row_bits, c.tile_bits), us.value


def chw_tune_cache_load(path):
    return _lib.load().chw_tune_cache_load(os.fsencode(path))


def chw_tune_cache_save(path):
    _lib.check(_lib.load().chw_tune_cache_save(os.fsencode(path)), "chw_tune_cache_save")


def chw_tune_cache_clear():
    _lib.load().chw_tune_cache_clear()


def chw_last_device_status(plan):
    """Synchronise and return the plan's latched device status (0 = CHW_OK)."""
    return _lib.load().chw_last_device_status(plan.handle)


def chw_plan_destroy(plan):
    plan.close()


def chw_status_string(status):
    return _lib.load().chw_status_string(int(status)).decode()


def chw_last_error_message():
    return _lib.load().chw_last_error_message().decode()
