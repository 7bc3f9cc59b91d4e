"""Staging layouts behind the kernels' TMA stores, checked on the CPU with the kernels' own
constexpr plans and the two-pass plan's column-blocked tensor view (csrc/colblock.h):
tests/native/layout_check.cu is compiled (host code only) and run."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_tma_store_staging_layouts(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "layout_check")
    cmd = [nvcc, "-std=c++20", "--expt-relaxed-constexpr", "-O2",
           "-I" + os.path.join(ROOT, "paper_1609_06641_gb300", "csrc"), "-I" + os.path.join(ROOT, "include"),
           "-gencode", "arch=compute_103a,code=sm_103a", os.path.join(HERE, "native", "layout_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "ALL OK" in out.stdout, out.stdout[-3000:]
