"""chw_forward_noalloc: the transform for callers that cannot allocate device memory (GPU).

Some callers cannot let the library cudaMalloc a workspace: a process whose device memory
was handed in full to another allocator has none left to give, and latency-critical code
cannot take the device-wide synchronisation that cudaMalloc implies.  This entry point
keeps the two-pass intermediate in a fixed array inside the library instead.  It launches
what chw_forward launches for a two-pass plan of the same shape, so its results must equal
chw_forward's bit for bit (well within the fp32 tolerance of 1e-6 used everywhere else)
and the fp32 cascade of Theorem 1 computed by the CPU oracle, on two calls in a row that
reuse the array; after each call the array's status word must read CHW_OK.  This file
sorts last so that a run stopping at its first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_1609_06641_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(cuda_device):
    import torch

    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import _lib, build

    build.build()
    return chw, _lib, _lib.load(), torch


def noalloc(lib, torch, m, batch, dtype, norm, xd):
    yd = torch.empty_like(xd)
    st = lib.chw_forward_noalloc(m, batch, dtype, norm, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.chw_status_string(st).decode()
    return yd


@pytest.mark.parametrize(
    "m,batch,dtype,norm",
    [(18, 16, "f32", "end"), (19, 3, "f32", "none"), (20, 4, "f32", "per_level"), (21, 2, "f32", "end"),
     (22, 1, "f32", "per_level"), (22, 1, "i32", "none")],
)
def test_noalloc_matches_forward_and_oracle_on_two_calls(env, m, batch, dtype, norm):
    chw, _lib, lib, torch = env
    d = chw.DTYPES[dtype]
    nm = chw.NORMS[norm]
    for call in range(2):  # two calls in a row share the static array
        if dtype == "i32":
            x = W.uniform_int32(m, batch, seed=50 + call, bound=2 ** (29 - m))
        else:
            x = W.normal_f32(m, batch, seed=50 + call)
        xd = torch.from_numpy(x).cuda()
        got = noalloc(lib, torch, m, batch, d, nm, xd)
        assert lib.chw_noalloc_device_status() == _lib.CHW_OK, lib.chw_last_error_message().decode()
        p = chw.chw_plan(m, batch, dtype, norm)
        ref = torch.empty_like(xd)
        chw.chw_forward(p, xd, ref)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(g.view(np.uint32), r.view(np.uint32)), f"call {call}: differs from chw_forward"
        want = oracle.chw_cascade(x, m, np.int32 if dtype == "i32" else np.float32, norm)
        assert np.array_equal(g.view(np.uint32), want.view(np.uint32)), f"call {call}: differs from the cascade"
        if dtype == "f32":
            exact = oracle.wht_fast_dyadic(x.astype(np.float64), m)  # FP64 H_m x
            if norm == "none":
                exact = exact * 2.0 ** (m / 2)  # the unnormalised transform 2^{m/2} H_m x
            assert oracle.rel_err_per_signal(g, exact).max() <= 1e-6


def test_noalloc_rejects_what_it_cannot_hold(env):
    chw, _lib, lib, torch = env
    xd = torch.zeros(1 << 20, device="cuda")
    p = ctypes.c_void_p(xd.data_ptr())
    assert lib.chw_forward_noalloc(20, 8, _lib.CHW_F32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_INVALID_ARG
    assert lib.chw_forward_noalloc(23, 1, _lib.CHW_F32, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_UNSUPPORTED
    assert lib.chw_forward_noalloc(18, 1, _lib.CHW_BF16, _lib.CHW_NORM_END, p, p, None) == _lib.CHW_ERR_UNSUPPORTED
    assert lib.chw_forward_noalloc(18, 1, _lib.CHW_F32, _lib.CHW_NORM_END, ctypes.c_void_p(xd.data_ptr() + 4), p, None) == _lib.CHW_ERR_ALIGNMENT
    assert lib.chw_noalloc_device_status() == _lib.CHW_OK


def test_noalloc_call_replays_from_a_cuda_graph(env):
    """A call captured into a CUDA graph (after one warm-up call outside the capture, which
    does the per-kernel set-up) replays to chw_forward's bits and the fp32 cascade's, with
    the status word at CHW_OK: the call allocates nothing, so it may be captured."""
    chw, _lib, lib, torch = env
    m, batch = 20, 2
    d, nm = chw.DTYPES["f32"], chw.NORMS["end"]
    x = W.normal_f32(m, batch, seed=61)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    noalloc(lib, torch, m, batch, d, nm, xd)  # warm-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = lib.chw_forward_noalloc(m, batch, d, nm, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.CHW_OK, lib.chw_status_string(st).decode()
    for _ in range(2):
        yd.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert lib.chw_noalloc_device_status() == _lib.CHW_OK, lib.chw_last_error_message().decode()
        p = chw.chw_plan(m, batch, "f32", "end")
        ref = torch.empty_like(xd)
        chw.chw_forward(p, xd, ref)
        torch.cuda.synchronize()
        g, r = yd.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(g.view(np.uint32), r.view(np.uint32)), "graph replay differs from chw_forward"
        want = oracle.chw_cascade(x, m, np.float32, "end")
        assert np.array_equal(g.view(np.uint32), want.view(np.uint32)), "graph replay differs from the cascade"
