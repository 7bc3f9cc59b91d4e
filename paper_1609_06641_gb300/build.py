"""Build libchw.so (the CUDA library behind include/chw.h) in-tree for sm_103a.

The fused kernels are templates; this script writes one small translation unit per
kernel shape (explicit instantiations) plus the lookup table that maps a shape to its
launcher, so that nvcc can compile them in parallel.  Every translation unit compiles
with nvcc for sm_103a and the objects link into paper_1609_06641_gb300/libchw.so.
Sources are hashed so an unchanged tree is not rebuilt.  Run as
``python -m paper_1609_06641_gb300.build`` or call ``build()``.
"""

import concurrent.futures as cf
import hashlib
import os
import platform
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build", platform.machine())  # objects never cross architectures
LIB = os.path.join(HERE, "libchw.so")
STAMP = os.path.join(OBJ, "sources.sha256")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = [
    "-std=c++20",
    "--expt-relaxed-constexpr",
    "-O3",
    "-lineinfo",
    "-Xcompiler",
    "-fPIC",
    "-I" + os.path.join(ROOT, "include"),
    "-I" + CSRC,
]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CHW library needs the CUDA toolkit to build")
    return cand


GEN = os.path.join(OBJ, "gen")

# (TLO, M, TB, CB, OUTMODE, variants) of every fused kernel the host dispatch can ask for:
# one-pass rows (M <= 17), first pass of the two-pass split (column-blocked output), and
# second-pass column blocks (2^A rows x 32 columns).
ALL = ("kVarPerLevel", "kVarEnd", "kVarPlain", "kVarI32")
NO_END = ("kVarPerLevel", "kVarPlain", "kVarI32")
SHAPES = (
    [(0, m, 13, 0, 0, ALL) for m in range(0, 14)]
    + [(0, 14, 14, 0, 0, ALL), (0, 15, 14, 1, 0, ALL), (0, 16, 14, 2, 0, ALL), (0, 17, 14, 3, 0, ALL)]
    + [(0, b, 13 if b <= 13 else 14, max(0, b - 14), 1, NO_END) for b in (5, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17)]
    + [(5, a, 13 if a <= 8 else 14, max(0, a - 9), 0, ALL) for a in range(6, 13)]
    # 2^13-word tiles in 2-, 4- and 8-CTA clusters (three CTAs per SM)
    + [(0, m, 13, m - 13, 0, ALL) for m in (14, 15, 16)]
    + [(0, b, 13, b - 13, 1, NO_END) for b in (14, 15, 16)]
    + [(5, a, 13, a - 8, 0, ALL) for a in (9, 10, 11)]
    # natural order (mode 2: final output, mode 4: first pass of the natural two-pass split)
    + [(0, m, 13, 0, 2, ALL) for m in range(2, 14)]
    + [(0, 14, 14, 0, 2, ALL)]
    + [(0, b, 13 if b <= 13 else 14, 0, 4, NO_END) for b in range(5, 15)]
    + [(5, a, 13 if a <= 8 else 14, 0, 2, ALL) for a in (6, 7, 8, 9)]
    # the Haar-Walsh head (mode 6: per-scale transforms of a signal's first 2^m positions)
    + [(0, m, 13, 0, 6, NO_END) for m in range(0, 14)]
    + [(0, 14, 14, 0, 6, NO_END)]
    # sequency order (mode 3)
    + [(0, m, 13, 0, 3, ALL) for m in range(2, 14)]
    + [(0, 14, 14, 0, 3, ALL), (0, 15, 14, 1, 3, ALL), (0, 16, 14, 2, 3, ALL), (0, 17, 14, 3, 3, ALL)]
    + [(5, a, 13 if a <= 8 else 14, max(0, a - 9), 3, ALL) for a in range(6, 13)]
)
BF = {
    "kVarPerLevel": ("::chw::BfF32PerLevel", "false"),
    "kVarEnd": ("::chw::BfF32Plain", "true"),
    "kVarPlain": ("::chw::BfF32Plain", "false"),
    "kVarI32": ("::chw::BfI32", "false"),
}
SIG = "(const CUtensorMap*, const ::chw::FusedArgs&, int64_t, cudaStream_t)"


def _inst(shape, var, extern):
    tlo, m, tb, cb, om, _ = shape
    bf, sc = BF[var]
    kw = "extern template" if extern else "template"
    return f"{kw} cudaError_t chw::launch_fused<{tlo}, {m}, {tb}, {cb}, {bf}, {sc}, {om}>{SIG};\n"


# Single-CTA dyadic row kernels that also write the Haar side output (fused.cuh, HZ): one
# per m = 1..14, on the tile the plain kernel of that m uses.
HZ_SHAPES = [(m, 13 if m <= 13 else 14) for m in range(1, 15)]


def _inst_hz(m, tb, var, extern):
    bf, sc = BF[var]
    kw = "extern template" if extern else "template"
    return f"{kw} cudaError_t chw::launch_fused<0, {m}, {tb}, 0, {bf}, {sc}, 0, true>{SIG};\n"


def _generate():
    os.makedirs(GEN, exist_ok=True)
    files = {}
    for shape in SHAPES:
        tlo, m, tb, cb, om, vars_ = shape
        name = f"fused_{tlo}_{m}_{tb}_{cb}_{om}.cu"
        body = '#include "launch.cuh"\n' + "".join(_inst(shape, v, False) for v in vars_)
        files[name] = body
    for m, tb in HZ_SHAPES:
        files[f"fused_hz_{m}_{tb}.cu"] = '#include "launch.cuh"\n' + "".join(_inst_hz(m, tb, v, False) for v in ALL)
    lk = ['#include "launch.cuh"\n']
    for shape in SHAPES:
        lk += [_inst(shape, v, True) for v in shape[5]]
    for m, tb in HZ_SHAPES:
        lk += [_inst_hz(m, tb, v, True) for v in ALL]
    lk.append("namespace chw {\nFusedLaunchFn lookup_fused(int tlo, int m, int tb, int cb, int var, int om) {\n")
    for shape in SHAPES:
        tlo, m, tb, cb, om, vars_ = shape
        lk.append(f"  if (tlo == {tlo} && m == {m} && tb == {tb} && cb == {cb} && om == {om}) {{\n")
        for v in vars_:
            bf, sc = BF[v]
            lk.append(f"    if (var == {v}) return &launch_fused<{tlo}, {m}, {tb}, {cb}, {bf}, {sc}, {om}>;\n")
        lk.append("    return nullptr;\n  }\n")
    lk.append("  return nullptr;\n}\n")
    lk.append("FusedLaunchFn lookup_fused_hz(int m, int tb, int var) {\n")
    for m, tb in HZ_SHAPES:
        lk.append(f"  if (m == {m} && tb == {tb}) {{\n")
        for v in ALL:
            bf, sc = BF[v]
            lk.append(f"    if (var == {v}) return &launch_fused<0, {m}, {tb}, 0, {bf}, {sc}, 0, true>;\n")
        lk.append("    return nullptr;\n  }\n")
    lk.append("  return nullptr;\n}\n}  // namespace chw\n")
    files["fused_lookup.cu"] = "".join(lk)
    for v in ALL:
        files[f"ragged_{v}.cu"] = (
            '#include "ragged_kernel.cuh"\n'
            f"template cudaError_t chw::launch_ragged_small< ::chw::{v}>(const ::chw::RaggedArgs&, cudaStream_t);\n"
        )
    paths = []
    for name, body in files.items():
        path = os.path.join(GEN, name)
        old = open(path).read() if os.path.exists(path) else None
        if old != body:
            with open(path, "w") as f:
                f.write(body)
        paths.append(path)
    return paths


def _sources():
    fixed = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    return fixed + _generate()


def _digest():
    h = hashlib.sha256()
    files = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h")))
    files.append(os.path.join(ROOT, "include", "chw.h"))
    files.append(os.path.abspath(__file__))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


# Sources of the batched single-CTA, cluster and tensor-memory kernels (the kernels the
# benchmark's roofline record names); their digest (code only, comments removed) is
# recorded next to committed DRAM-traffic figures so that a figure is used only while the
# code it was measured on is unchanged.
KERNEL_SOURCES = ("ptx.cuh", "engine.cuh", "fused.cuh", "launch.cuh", "tmem.cuh", "tmem_launch.cuh", "tmem.cu")


def _code_only(text):
    """Source text without comments and blank lines (a comment edit leaves the code's digest)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_digest():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name)) as fh:
            h.update(name.encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def build(force=False, verbose=False, jobs=None):
    """Compile every csrc/*.cu for sm_103a and link libchw.so; returns the library path."""
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as f:
            if f.read().strip() == digest:
                return LIB
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()
    newest_header = max(
        os.path.getmtime(os.path.join(d, f))
        for d in (CSRC, os.path.join(ROOT, "include"))
        for f in os.listdir(d)
        if f.endswith((".cuh", ".h"))
    )
    if force:
        newest_header = float("inf")
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    # longest units first so the parallel build ends together
    srcs.sort(key=lambda p: (0 if "ragged_" in os.path.basename(p) else 1, -os.path.getsize(p)))

    def compile_one(src):
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        if os.path.exists(obj) and os.path.getmtime(obj) > max(os.path.getmtime(src), newest_header):
            return obj, ""
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-6000:]}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for obj, err in results:
            sys.stderr.write(f"--- {os.path.basename(obj)}\n{err}")
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
