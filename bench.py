"""Benchmark of the CHW Walsh-Hadamard library on GB300: one JSON line on rank 0.

Headline workload: y = H_16 x for 4096 fp32 signals of 65536 elements (dyadic order,
normalised by one 2^-8 multiply), N(0,1) inputs.  One step is one chw_forward over the
whole batch; the metric is effective HBM bandwidth, 2 * n * 4 bytes per signal (read x
once, write y once) divided by the device time.  Inputs (1 GiB) exceed the 129 MB L2, so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-extra]

Under torchrun (N > 1) every rank transforms its own batch (independent signals, no
collective on the data path: weak scaling); the step time is the maximum over ranks.
``--impl reference`` times the CPU oracle (plain FP64 numpy) on bounded samples of the
same workload instead.
"""

import argparse
import ctypes
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "WHT effective HBM GB/s (% peak) at stated error; bf16/ragged vs plain fp32"
M, BATCH, SEED = 16, 4096, 2
FALLBACK_HBM_GBS = 6800.0


# ---------------------------------------------------------------- helpers
def gbs(nbytes, seconds):
    return nbytes / seconds / 1e9


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device=None):
    """Maximum of a float over all ranks (identity when world == 1)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


class ClockSampler:
    """Samples SM clock, max clock, power and clock-event reasons through NVML (ctypes)."""

    REASONS = {
        0x1: "gpu_idle",
        0x2: "applications_clocks_setting",
        0x4: "sw_power_cap",
        0x8: "hw_slowdown",
        0x10: "sync_boost",
        0x20: "sw_thermal_slowdown",
        0x40: "hw_thermal_slowdown",
        0x80: "hw_power_brake_slowdown",
        0x100: "display_clock_setting",
    }

    def __init__(self, index, period=0.001):
        self.samples = []
        self.period = period
        self.ok = False
        self.max_mhz = None
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.ok = True
        except OSError:
            self.ok = False

    def _read(self):
        clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk))
        self.nvml.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(pw))
        fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or getattr(
            self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons"
        )
        fn(self.h, ctypes.byref(rs))
        return clk.value, pw.value / 1000.0, rs.value

    def start(self):
        self.stop_flag = False
        if not self.ok:
            return

        def run():
            while not self.stop_flag:
                self.samples.append(self._read())
                time.sleep(self.period)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        if self.ok:
            self.thread.join()
            self.samples.append(self._read())

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["nvml unavailable"]}
        clk = np.array([s[0] for s in self.samples])
        bits = 0
        for s in self.samples:
            bits |= s[2]
        reasons = [name for b, name in self.REASONS.items() if bits & b]
        return {
            "sm_mhz": float(np.median(clk)),
            "sm_max_mhz": self.max_mhz,
            "reasons": reasons,
            "samples": len(self.samples),
            "power_w_max": float(max(s[1] for s in self.samples)),
        }


def time_device(fn, steps, warmup, world, stream, sampler=None):
    """W untimed calls, then K calls bracketed by barrier + synchronize, CUDA events on `stream`."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.stop()
    barrier(world)
    return start.elapsed_time(end) / steps  # ms per step


def traffic_from_profile(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it matches the compiled kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(kernel_key)
    if not ent:
        return None
    from paper_1609_06641_gb300 import build

    if ent.get("kernel_digest") != build.kernel_digest():
        return None
    return ent.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- CPU oracle leg
def oracle_rate(m, rows, seconds_budget=10.0):
    """Oracle (FP64 fast WHT + dyadic reorder) on `rows`; repeats until the budget; GB/s."""
    import oracle

    nbytes = 2 * rows.shape[0] * (1 << m) * 4
    reps, t0 = 0, time.perf_counter()
    ref = None
    while True:
        ref = oracle.wht_fast_dyadic(rows.astype(np.float64), m)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds_budget:
            break
    return gbs(nbytes * reps, el), ref, reps, el


def cpu_baseline_leg(x_rows, y_rows, budget):
    import oracle

    rate, ref, reps, el = oracle_rate(M, x_rows, budget)
    err = float(oracle.rel_err_per_signal(y_rows, ref).max())
    return (
        {
            "value": rate,
            "unit": "GB/s",
            "cores": 1,
            "kind": "oracle",
            "sample": f"{x_rows.shape[0]} of the {BATCH} signals (m={M}), FP64 numpy fast WHT + dyadic "
            f"reorder, repeated {reps}x over {el:.1f} s; GB/s counts 2*n*4 bytes per signal",
        },
        err,
    )


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    if rank != 0:
        return
    from paper_1609_06641_gb300 import workloads as W

    sample = 16
    rows = W.normal_f32(M, sample, SEED)
    import oracle

    for _ in range(args.warmup):
        oracle.wht_fast_dyadic(rows.astype(np.float64), M)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.wht_fast_dyadic(rows.astype(np.float64), M)
    el = time.perf_counter() - t0
    nbytes = 2 * sample * (1 << M) * 4
    value = gbs(nbytes * args.steps, el)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "GB/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic: N(0,1) fp32 signals, numpy PCG64 seed 2",
        "config": workload_config(),
        "cpu_baseline": {
            "value": value,
            "unit": "GB/s",
            "cores": 1,
            "kind": "oracle",
            "sample": f"each step: {sample} signals of m={M} through the FP64 oracle (plain numpy, one core)",
        },
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config():
    return {
        "workload": "y = H_16 x (dyadic order, CHW cascade), 4096 signals x 65536 fp32, normalised by one "
        "fp32(2^-8) multiply; inputs 1 GiB > 129 MB L2, no flush between steps",
        "m": M,
        "batch": BATCH,
        "norm": "end",
        "algorithmic_bytes_per_step": 2 * BATCH * (1 << M) * 4,
    }


# ---------------------------------------------------------------- extra configurations
def oracle_beside(fn, nbytes, budget=0.5):
    """The oracle as it stands, timed on a small host sample of a row's workload: repeats
    fn() until `budget` seconds have passed; returns GB/s counting `nbytes` per call."""
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget:
            return round(gbs(nbytes * reps, el), 4)


def extra_measurements(chw, torch, dev, steps, warmup, peak):
    """Device-timed throughput of the other benchmark shapes (inputs drawn on the device),
    each with the CPU oracle timed beside it on a small sample of the same workload
    ("cpu_oracle_GB/s", one host core, sample named in "cpu_oracle_sample")."""
    import oracle as O
    from paper_1609_06641_gb300 import workloads as W

    out = {}

    def rec(name, nbytes, ms, launches, oracle=None, **kw):
        v = gbs(nbytes, ms / 1e3)
        out[name] = {"GB/s": round(v, 1), "frac_of_peak": round(v / peak, 4), "ms_per_call": round(ms, 4),
                     "launches_per_call": launches, **kw}
        if oracle is not None:
            fn, sample_bytes, what = oracle
            out[name]["cpu_oracle_GB/s"] = oracle_beside(fn, sample_bytes)
            out[name]["cpu_oracle_sample"] = what

    h16 = W.normal_f32(M, 2, 11)  # two host signals of the headline shape for the oracle samples
    nb16 = 2 * h16.nbytes

    st = torch.cuda.current_stream()
    g = torch.Generator(device=dev).manual_seed(7)
    k = max(3, steps // 2)
    # the small configuration (m = 10, 64 signals, N(0,1) from seed 0, 256 KiB): a
    # launch-latency workload, so its row states the time per call -- device time of
    # back-to-back calls, and host wall time of one call plus a synchronize -- and its parity
    x10 = W.normal_f32(10, 64, 0)
    xd10 = torch.from_numpy(x10).to(dev)
    yd10 = torch.empty_like(xd10)
    p10 = chw.chw_plan(10, 64, "f32", "per_level")
    ms = time_device(lambda: chw.chw_forward(p10, xd10, yd10), k, warmup, 1, st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        chw.chw_forward(p10, xd10, yd10)
        torch.cuda.synchronize()
    call_us = (time.perf_counter() - t0) / k * 1e6
    # the device's own latency: the call captured once in a CUDA graph and replayed (no host
    # work between launches)
    graph_us = None
    try:
        cs = torch.cuda.Stream()
        cs.wait_stream(st)
        with torch.cuda.stream(cs):
            chw.chw_forward(p10, xd10, yd10)
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=cs):
                chw.chw_forward(p10, xd10, yd10)
        st.wait_stream(cs)
        torch.cuda.synchronize()
        graph_us = round(time_device(gr.replay, k, warmup, 1, st) * 1e3, 2)
    except RuntimeError:
        graph_us = None
    got10 = yd10.cpu().numpy()
    rec("m10_b64_f32_per_level", 2 * x10.nbytes, ms, 1,
        oracle=(lambda: O.wht_dense(x10.astype(np.float64), 10), 2 * x10.nbytes, "64 signals, FP64 dense H_10 (O1)"),
        device_us_per_call=round(ms * 1e3, 2), host_us_per_call_with_sync=round(call_us, 1),
        graph_replay_us_per_call=graph_us,
        bitwise_equal_to_fp32_cascade=bool(np.array_equal(
            got10.view(np.uint32), O.chw_cascade(x10, 10, np.float32, "per_level").view(np.uint32))),
        rel_err_vs_dense_fp64_max=float(O.rel_err_per_signal(got10, O.wht_dense(x10.astype(np.float64), 10)).max()),
        rel_err_vs_fast_fp64_max=float(O.rel_err_per_signal(got10, O.wht_fast_dyadic(x10.astype(np.float64), 10)).max()),
        error_gate=1e-6)
    del xd10, yd10
    # fp32 per-level normalisation and int32 on the headline shape
    x = torch.randn(BATCH, 1 << M, device=dev, generator=g)
    y = torch.empty_like(x)
    p = chw.chw_plan(M, BATCH, "f32", "per_level")
    ms = time_device(lambda: chw.chw_forward(p, x, y), k, warmup, 1, st)
    rec("m16_b4096_f32_per_level", 2 * x.numel() * 4, ms, 1,
        oracle=(lambda: O.chw_cascade(h16, M, np.float32, "per_level"), nb16, "2 signals, fp32 cascade (O4)"))
    xi = torch.randint(-(2**14), 2**14 + 1, (BATCH, 1 << M), device=dev, dtype=torch.int32, generator=g)
    yi = torch.empty_like(xi)
    pi = chw.chw_plan(M, BATCH, "i32", "none")
    ms = time_device(lambda: chw.chw_forward(pi, xi, yi), k, warmup, 1, st)
    hi = W.uniform_int32(M, 2, 12)
    rec("m16_b4096_i32", 2 * xi.numel() * 4, ms, 1,
        oracle=(lambda: O.wht_fast_dyadic(hi.astype(np.int64), M, normalised=False), 2 * hi.nbytes,
                "2 signals, int64 fast WHT (O2)"))
    del xi, yi
    # long signals (m = 26 x 4, m = 28 x 1, Uniform(-1,1) from seed 3): two HBM passes; the
    # round trip H^T H x against x on every signal (FP64 norms; the forward's bitwise parity
    # with the oracle's cascade at these sizes is a GPU test, too slow for the host here)
    for m, b in ((26, 4), (28, 1)):
        xh_l = W.uniform_pm1_f32(m, b, 3)
        xl = torch.from_numpy(xh_l).to(dev)
        yl = torch.empty_like(xl)
        pl = chw.chw_plan(m, b, "f32", "end")
        il = chw.chw_plan_get_info(pl)
        ms = time_device(lambda: chw.chw_forward(pl, xl, yl), k, warmup, 1, st)
        back = torch.empty_like(xl)
        chw.chw_adjoint(pl, yl, back)
        torch.cuda.synchronize()
        assert chw.chw_last_device_status(pl) == 0
        xd64 = xl.double()
        rt = float(((back.double() - xd64).norm(dim=1) / xd64.norm(dim=1)).max())
        del back, xd64
        kw = {"row_bits": int(il.row_bits), "roundtrip_rel_err_max": rt, "roundtrip_gate": 1e-6,
              "inputs": "Uniform(-1,1) fp32, numpy PCG64 seed 3"}
        rec(f"m{m}_b{b}_f32_two_pass", 2 * xl.numel() * 4, ms, il.kernels_per_call,
            dram_pass_frac=round(gbs(2 * il.passes * xl.numel() * 4, ms / 1e3) / peak, 4), **kw)
        del xl, yl, pl
    # autotuned plans (the tuner times every candidate configuration when the plan is made):
    # the built-in choice and the tuned one, side by side
    for m, b in ((17, 2048), (20, 256), (22, 64)):
        xa = torch.randn(b, 1 << m, device=dev, generator=g)
        ya = torch.empty_like(xa)
        for tag, fl in (("builtin", 0), ("autotuned", chw.CHW_FLAG_AUTOTUNE)):
            t0 = time.perf_counter()
            pa = chw.chw_plan(m, b, "f32", "end", fl)
            plan_s = time.perf_counter() - t0
            ia = chw.chw_plan_get_info(pa)
            ms = time_device(lambda: chw.chw_forward(pa, xa, ya), k, warmup, 1, st)
            rec(f"m{m}_b{b}_f32_{tag}", 2 * xa.numel() * 4, ms, ia.kernels_per_call, tier=int(ia.tier),
                row_bits=int(ia.row_bits), tile_bits=int(ia.tile_bits), plan_ms=round(plan_s * 1e3, 1))
            del pa
        del xa, ya
    # 16-bit storage, m = 12, batch 16384, on the precision workload: Student-t(3) x per-signal
    # lognormal(0, 2) from seed 4, stored as (codes, power-of-two exponent).  Errors per
    # signal on every 8th signal: the dequantised result against the FP64 oracle of the
    # dequantised input, and against the plain fp32 path on this GPU (same input values).
    x4 = W.heavy_tailed_f64(12, 16384, 4)
    sel = np.arange(0, 16384, 8)
    for fmt, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        codes, e_in = W.quantise_pow2(x4, fmt)
        xq = torch.from_numpy(codes.view(np.int16)).to(dev).view(tdt)
        yq = torch.empty_like(xq)
        ei = torch.from_numpy(e_in).to(dev)
        eo = torch.empty_like(ei)
        pq = chw.chw_plan(12, 16384, fmt, "end")
        ms = time_device(lambda: chw.chw_forward(pq, xq, yq, ei, eo), k, warmup, 1, st)
        torch.cuda.synchronize()
        assert chw.chw_last_device_status(pq) == 0
        q_out = yq.view(torch.int16).cpu().numpy().view(np.uint16)[sel]
        e_out = eo.cpu().numpy()[sel]
        # the plain fp32 path on the same (dequantised) input values
        t0 = time.perf_counter()
        deq_in = O.dequantise(codes[sel], e_in[sel], fmt)
        ref = O.wht_fast_dyadic(deq_in, 12)
        o_s = time.perf_counter() - t0
        x32 = torch.from_numpy(deq_in.astype(np.float32)).to(dev)
        y32 = torch.empty_like(x32)
        p32 = chw.chw_plan(12, len(sel), "f32", "end")
        chw.chw_forward(p32, x32, y32)
        got = O.dequantise(q_out, e_out, fmt)
        err = O.rel_err_per_signal(got, ref)
        err32 = O.rel_err_per_signal(got, y32.cpu().numpy())
        err_f32_path = O.rel_err_per_signal(y32.cpu().numpy(), ref)
        rec(f"m12_b16384_{fmt}", 2 * xq.numel() * 2, ms, 1,
            rel_err_vs_fp64_oracle={"max": float(err.max()), "p99": float(np.percentile(err, 99))},
            rel_err_vs_gpu_fp32_path={"max": float(err32.max()), "p99": float(np.percentile(err32, 99))},
            gpu_fp32_path_rel_err_vs_fp64={"max": float(err_f32_path.max())},
            error_gate={"bf16": 1e-2, "f16": 2e-3}[fmt],
            error_sample=f"every 8th signal ({len(sel)} of 16384)",
            inputs="Student-t(3) x lognormal(0,2) per signal, numpy PCG64 seed 4, (codes, 2^e) per signal",
            **{"cpu_oracle_GB/s": round(gbs(2 * len(sel) * 4096 * 2, o_s), 4),
               "cpu_oracle_sample": f"{len(sel)} signals, FP64 O2 of the dequantised input"})
        del xq, yq, x32, y32, p32
    del x4
    # D H_m layer, m = 14, batch 512: forward and adjoint
    xd = torch.randn(512, 1 << 14, device=dev, generator=g)
    yd = torch.empty_like(xd)
    d = (1 - 2 * torch.randint(0, 2, (1 << 14,), device=dev, generator=g)).to(torch.int8)
    pd = chw.chw_plan(14, 512, "f32", "end")
    ms = time_device(lambda: chw.chw_forward(pd, xd, yd, diag=d), k, warmup, 1, st)
    hd = W.normal_f32(14, 8, 13)
    dd = W.diag_pm1(14, 14)
    rec("m14_b512_DH_forward", 2 * xd.numel() * 4, ms, 1,
        oracle=(lambda: dd * O.wht_fast_dyadic(hd.astype(np.float64), 14), 2 * hd.nbytes, "8 signals, FP64 O2 then D"))
    ms = time_device(lambda: chw.chw_adjoint(pd, yd, xd, diag=d), k, warmup, 1, st)
    rec("m14_b512_DH_adjoint", 2 * xd.numel() * 4, ms, 1)
    del xd, yd
    # Haar transform (eq. (2)), its transpose, Haar-Walsh (eq. (4)) and the forward with its
    # Haar side output, on the headline shape
    xh = torch.randn(BATCH, 1 << M, device=dev, generator=g)
    zh = torch.empty_like(xh)
    yh = torch.empty_like(xh)
    ph = chw.chw_plan(M, BATCH, "f32", "per_level", chw.CHW_FLAG_HAAR_WALSH)
    nb = xh.numel() * 4
    ms = time_device(lambda: chw.chw_haar(ph, xh, zh), k, warmup, 1, st)
    rec("m16_b4096_f32_haar", 2 * nb, ms, 2,
        oracle=(lambda: O.haar_forward(h16, M, np.float32, "per_level"), nb16, "2 signals, fp32 Haar (eq. (2))"))
    ms = time_device(lambda: chw.chw_haar_inverse(ph, zh, yh), k, warmup, 1, st)
    rec("m16_b4096_f32_haar_inverse", 2 * nb, ms, 2,
        oracle=(lambda: O.haar_inverse(h16, M, np.float32, "per_level"), nb16, "2 signals, fp32 inverse Haar"))
    ms = time_device(lambda: chw.chw_from_haar(ph, zh, yh), k, warmup, 1, st)
    rec("m16_b4096_f32_haar_walsh", 2 * nb, ms, 3,
        oracle=(lambda: O.haar_walsh(h16, M, np.float32, "per_level"), nb16, "2 signals, fp32 stages 1..m-1"))
    ms = time_device(lambda: chw.chw_forward_haar(ph, xh, yh, zh), k, warmup, 1, st)
    rec("m16_b4096_f32_forward_with_haar_output", 3 * nb, ms, 1,
        bytes_counted="x read once, y and z written once (3 n 4 bytes per signal)",
        oracle=(lambda: (O.chw_cascade(h16, M, np.float32, "per_level"), O.haar_forward(h16, M, np.float32, "per_level")),
                3 * h16.nbytes, "2 signals, fp32 cascade and fp32 Haar"))
    # the same two calls with normalisation at the end (one scale per output instead of one
    # per level): the plans `--op haar_walsh` and `--op forward_haar` time
    try:
        pe = chw.chw_plan(M, BATCH, "f32", "end", chw.CHW_FLAG_HAAR_WALSH)
        ms = time_device(lambda: chw.chw_from_haar(pe, zh, yh), k, warmup, 1, st)
        rec("m16_b4096_f32_haar_walsh_end", 2 * nb, ms, 3)
        pf = chw.chw_plan(M, BATCH, "f32", "end")
        ms = time_device(lambda: chw.chw_forward_haar(pf, xh, yh, zh), k, warmup, 1, st)
        rec("m16_b4096_f32_forward_with_haar_output_end", 3 * nb, ms, 1,
            bytes_counted="x read once, y and z written once (3 n 4 bytes per signal)")
        del pe, pf
    except Exception as e:  # recorded; the other rows still run
        out["m16_b4096_f32_haar_end_rows"] = {"failed": repr(e)[:300]}
    del xh, zh, yh, ph
    # natural and sequency output orders on the headline shape and at m = 12
    for order in ("natural", "sequency"):
        for m, b in ((M, BATCH), (12, 65536)):
            xo = torch.randn(b, 1 << m, device=dev, generator=g)
            yo = torch.empty_like(xo)
            po = chw.chw_plan(m, b, "f32", "end", order=order)
            info = chw.chw_plan_get_info(po)
            ms = time_device(lambda: chw.chw_forward(po, xo, yo), k, warmup, 1, st)
            ho = W.normal_f32(m, 2, 15)
            rec(f"m{m}_b{b}_f32_{order}", 2 * xo.numel() * 4, ms, info.kernels_per_call, tier=int(info.tier),
                oracle=(lambda: O.wht_ordered(ho, m, order, np.float32, "end"), 2 * ho.nbytes,
                        "2 signals, fp32 cascade stored in order"))
            del xo, yo, po
    # further shapes with quoted rates: the single-CTA tiers at scale (m = 12, 14), m = 15 in
    # sequency order, and the longest signals (m = 29, 30: 8- and 4-column blocks between
    # the two passes); a failure is recorded in its row
    for m, b, order in ((12, 65536, "dyadic"), (14, 16384, "dyadic"), (15, 8192, "sequency"), (29, 1, "dyadic"),
                        (30, 1, "dyadic")):
        try:
            xo = torch.randn(b, 1 << m, device=dev, generator=g)
            yo = torch.empty_like(xo)
            po = chw.chw_plan(m, b, "f32", "end", order=order)
            info = chw.chw_plan_get_info(po)
            ms = time_device(lambda: chw.chw_forward(po, xo, yo), k, warmup, 1, st)
            rec(f"m{m}_b{b}_f32_{order}", 2 * xo.numel() * 4, ms, info.kernels_per_call, tier=int(info.tier),
                passes=int(info.passes))
            del xo, yo, po
        except Exception as e:
            out[f"m{m}_b{b}_f32_{order}"] = {"failed": repr(e)[:300]}
    # ragged: 10,000 signals with m uniform on 6..20 (seed 5), one graph launch
    from paper_1609_06641_gb300 import workloads as W

    ms_arr, _ = W.ragged_ms(10000, 5)
    pr = chw.chw_plan_ragged(ms_arr, "f32", "end")
    total = int(chw.chw_plan_get_info(pr).total_elements)
    xr = torch.randn(total, device=dev, generator=g)
    yr = torch.empty_like(xr)
    ms = time_device(lambda: chw.chw_forward_ragged(pr, xr, yr), k, warmup, 1, st)
    useful = int(sum(1 << int(m) for m in ms_arr))
    # the same signals as one batched launch per length (grouped by m, no ragged kernel)
    groups = []
    for mm in sorted(set(int(v) for v in ms_arr)):
        cnt = int((ms_arr == mm).sum())
        xg = torch.randn(cnt, 1 << mm, device=dev, generator=g)
        groups.append((chw.chw_plan(mm, cnt, "f32", "end"), xg, torch.empty_like(xg)))

    def per_m():
        for pg, xg, yg in groups:
            chw.chw_forward(pg, xg, yg)

    ms_pm = time_device(per_m, k, warmup, 1, st)
    rec("ragged_10000_as_per_m_launches", 2 * useful * 4, ms_pm, len(groups))
    del groups
    # errors on every 250th signal: against the FP64 oracle, and against the plain fp32 path
    # (a one-signal batched plan of the same length on this GPU, same input values)
    rsel = list(range(0, len(ms_arr), 250))
    roff = chw.chw_ragged_offsets(pr)
    hr, got_r, plain_r = [], [], []
    for i in rsel:
        mi, o = int(ms_arr[i]), int(roff[i])
        xi = xr[o: o + (1 << mi)].view(1, -1)
        yi = torch.empty_like(xi)
        chw.chw_forward(chw.chw_plan(mi, 1, "f32", "end"), xi, yi)
        hr.append(xi.cpu().numpy())
        got_r.append(yr[o: o + (1 << mi)].view(1, -1).cpu().numpy())
        plain_r.append(yi.cpu().numpy())
    t0 = time.perf_counter()
    refs_r = [O.wht_fast_dyadic(h.astype(np.float64), int(ms_arr[i])) for h, i in zip(hr, rsel)]
    o_s = time.perf_counter() - t0
    err_r = max(float(O.rel_err_per_signal(g, r).max()) for g, r in zip(got_r, refs_r))
    err_p = max(float(O.rel_err_per_signal(g, r).max()) for g, r in zip(got_r, plain_r))
    same = all(np.array_equal(g.view(np.uint32), r.view(np.uint32)) for g, r in zip(got_r, plain_r))
    rec("ragged_10000_m6to20_f32", 2 * useful * 4, ms, 1, elements=useful,
        kernels_in_graph=int(chw.chw_plan_get_info(pr).kernels_per_call),
        rel_err_vs_fp64_oracle_max=err_r, rel_err_vs_gpu_fp32_path_max=err_p, bitwise_equal_to_fp32_path=same,
        error_gate=1e-6, error_sample=f"every 250th signal ({len(rsel)} signals)",
        **{"cpu_oracle_GB/s": round(gbs(sum(2 * h.nbytes for h in hr), o_s), 4),
           "cpu_oracle_sample": "every 250th signal of the batch, FP64 O2"})
    # the same ragged batch with each length's configuration picked by the autotuner
    del pr
    t0 = time.perf_counter()
    pt = chw.chw_plan_ragged(ms_arr, "f32", "end", chw.CHW_FLAG_AUTOTUNE)
    plan_s = time.perf_counter() - t0
    ms_t = time_device(lambda: chw.chw_forward_ragged(pt, xr, yr), k, warmup, 1, st)
    it = chw.chw_plan_get_info(pt)
    rec("ragged_10000_m6to20_f32_autotuned", 2 * useful * 4, ms_t, 1, kernels_in_graph=int(it.kernels_per_call),
        tuned=int(it.tuned), plan_ms=round(plan_s * 1e3, 1))
    return out


def quick_other(args, chw, torch, dev, peak):
    """--quick with another storage type, normalisation or output order: one plan, device
    inputs, CUDA-event timing only (the profiling runs of the other kernels)."""
    m, batch = args.m, args.batch
    g = torch.Generator(device=dev).manual_seed(9)
    ebytes = 2 if args.dtype in ("bf16", "f16") else 4
    if args.dtype == "i32":
        x = torch.randint(-(2**14), 2**14 + 1, (batch, 1 << m), device=dev, dtype=torch.int32, generator=g)
    else:
        x = torch.randn(batch, 1 << m, device=dev, generator=g)
        if ebytes == 2:
            x = x.to(torch.bfloat16 if args.dtype == "bf16" else torch.float16)
    y = torch.empty_like(x)
    exps = ()
    if ebytes == 2:
        exps = (torch.zeros(batch, dtype=torch.int32, device=dev), torch.empty(batch, dtype=torch.int32, device=dev))
    norm = "none" if args.dtype == "i32" else args.norm
    plan = chw.chw_plan(m, batch, args.dtype, norm, args.flags, order=args.order)
    info = chw.chw_plan_get_info(plan)
    ms = time_device(lambda: chw.chw_forward(plan, x, y, *exps), args.steps, args.warmup, 1,
                     torch.cuda.current_stream())
    assert chw.chw_last_device_status(plan) == 0
    v = gbs(2 * batch * (1 << m) * ebytes, ms / 1e3)
    print(json.dumps({"op": "forward", "m": m, "batch": batch, "dtype": args.dtype, "norm": norm,
                      "order": args.order, "tier": int(info.tier), "ms_per_step": ms, "GB/s": v,
                      "frac": v / peak}), flush=True)


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="chw", choices=["chw", "reference"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--quick", action="store_true", help="device timing only (profiling runs)")
    ap.add_argument("--m", type=int, default=M, help="transform bits of the timed workload")
    ap.add_argument("--batch", type=int, default=BATCH, help="signals of the timed workload")
    ap.add_argument("--flags", type=int, default=0, help="chw_plan flags (e.g. 4: row-stack tier for m = 15..17)")
    ap.add_argument("--op", default="forward", choices=["forward", "haar", "haar_inverse", "haar_walsh", "forward_haar"],
                    help="with --quick: the call timed (profiling runs of the other kernels)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "i32", "bf16", "f16"],
                    help="with --quick: storage type of the timed forward (profiling runs)")
    ap.add_argument("--norm", default="end", choices=["end", "per_level", "none"],
                    help="with --quick: normalisation of the timed forward")
    ap.add_argument("--order", default="dyadic", choices=["dyadic", "natural", "sequency"],
                    help="with --quick: output order of the timed forward")
    args = ap.parse_args()
    world, rank, local = dist_env()

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1609_06641_gb300 as chw
    from paper_1609_06641_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    peak, peak_kind = load_peaks()

    m, batch = args.m, args.batch
    if args.quick and (args.dtype != "f32" or args.norm != "end" or args.order != "dyadic"):
        quick_other(args, chw, torch, dev, peak)
        return
    x_host = W.normal_f32(m, batch, SEED + rank)  # each rank its own signals
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    flags = args.flags | (chw.CHW_FLAG_HAAR_WALSH if args.op == "haar_walsh" else 0)
    plan = chw.chw_plan(m, batch, "f32", "end", flags)
    info = chw.chw_plan_get_info(plan)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    op = args.op if args.quick else "forward"
    if op == "forward_haar":  # y and the Haar side output z: x read once, y and z written
        z = torch.empty_like(x)
        call = lambda p, a, b: chw.chw_forward_haar(p, a, b, z)  # noqa: E731
    else:
        call = {"forward": chw.chw_forward, "haar": chw.chw_haar, "haar_inverse": chw.chw_haar_inverse,
                "haar_walsh": chw.chw_from_haar}[op]
    ms = time_device(lambda: call(plan, x, y), args.steps, args.warmup, world, stream, sampler)
    ms_max = max_over_ranks(ms, world, dev)
    step_bytes = (3 if op == "forward_haar" else 2) * batch * (1 << m) * 4
    value = world * gbs(step_bytes, ms_max / 1e3)
    assert chw.chw_last_device_status(plan) == 0
    if args.quick:
        if rank == 0:
            print(json.dumps({"op": args.op, "m": m, "batch": batch, "ms_per_step": ms_max, "GB/s": value,
                              "frac": value / world / peak, "clocks": sampler.summary()}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # end to end through the host-buffer entry point (pinned memory, copies inside)
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    chw.chw_forward_host(plan, xh, yh)
    barrier(world)
    reps = []
    for _ in range(3):  # the median of three runs of e2e_steps calls (the host link varies)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            chw.chw_forward_host(plan, xh, yh)
        reps.append((time.perf_counter() - t0) / e2e_steps)
    e2e_s = sorted(reps)[1]
    e2e_s = max_over_ranks(e2e_s, world, dev)
    if not torch.equal(yh, y.cpu()):
        raise RuntimeError("host-buffer path disagrees with the device path")
    # the host link alone, the bound of the e2e number: the same pipeline as chw_forward_host
    # (64 MiB chunks cycling over three streams, each copied in and back out) with no transform
    rows = max(1, (64 << 20) // (x.shape[1] * 4))
    bufs = [torch.empty(rows, x.shape[1], device=dev) for _ in range(3)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    torch.cuda.synchronize()
    reps = []
    for _ in range(3):
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for i, r0 in enumerate(range(0, x.shape[0], rows)):
                n_r = min(rows, x.shape[0] - r0)
                with torch.cuda.stream(streams[i % 3]):
                    bufs[i % 3][:n_r].copy_(xh[r0: r0 + n_r], non_blocking=True)
                    yh[r0: r0 + n_r].copy_(bufs[i % 3][:n_r], non_blocking=True)
            torch.cuda.synchronize()
        reps.append((time.perf_counter() - t0) / e2e_steps)
    link_s = sorted(reps)[1]
    del bufs

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    per_launch_ms = ms / info.kernels_per_call
    achieved = gbs(step_bytes / info.kernels_per_call, per_launch_ms / 1e3)
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: N(0,1) fp32 signals (numpy PCG64 seed 2 + rank), resident in HBM",
        "config": workload_config(),
        "pct_of_peak": round(100 * value / world / peak, 2),
        "signals_per_s": round(world * BATCH / (ms_max / 1e3), 1),
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": traffic_from_profile(f"m{m}_b{batch}_f32_end_tier{info.tier}"),
            "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else "fallback",
            "kernel": {2: "cluster_kernel<0,16,14,2> (4-CTA cluster per signal, DSMEM exchange)",
                       6: "rowstack_kernel<16> (one CTA per signal, rows through L2)",
                       7: "tmem_kernel<16> (one CTA per signal, rows via shared memory, signal in tensor memory)"}
            .get(info.tier, str(info.tier)),
        },
        "e2e": {
            "value": round(gbs(step_bytes, e2e_s) * world, 1),
            "unit": "GB/s",
            "h2d_bytes_per_step": BATCH * (1 << M) * 4,
            "d2h_bytes_per_step": BATCH * (1 << M) * 4,
            "ms_per_step": round(e2e_s * 1e3, 3),
            "api": "chw_forward_host (pinned host buffers, 64 MiB chunks over 3 streams)",
            "host_link_GB/s": round(gbs(step_bytes, link_s), 1),
            "host_link_note": "the same 64 MiB three-stream copy pipeline with no transform (pinned host buffers)",
        },
        "gpu_launches": args.steps * info.kernels_per_call,
        "clocks": sampler.summary(),
    }
    if world == 1:
        rows = np.random.default_rng(0).choice(BATCH, 16, replace=False)
        y_rows = y.cpu().numpy()[rows]
        cpu, err = cpu_baseline_leg(x_host[rows], y_rows, args.cpu_budget)
        line["cpu_baseline"] = cpu
        line["error"] = {"max_rel_err_vs_fp64_oracle": err, "signals_checked": len(rows), "gate": 1e-6}
        if not args.no_extra:
            try:
                line["extra"] = extra_measurements(chw, torch, dev, args.steps, args.warmup, peak)
            except Exception as e:  # the headline line is printed whatever happens to the extras
                line["extra"] = {"failed": repr(e)[:400]}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
