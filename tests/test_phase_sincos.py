"""The FP32 kernels' phase sine-cosine (xf_math.cuh, phase_sincos for
float): a Cody-Waite reduction by pi/2 of the float-float phase lam * dl and
Taylor polynomials on [-pi/4, pi/4], written from the mathematics in place of
the library's sincosf.  tests/xf_phase_check.cpp runs the same template on
the host over two million seeded phases from 1e-6 to 1.3e5 rad and at every
quadrant boundary up to 3100 rad, against the library's long-double sine and
cosine of the exact phase; the largest absolute error must stay within 1.25
FP32 ulps at 1 (1.5e-7): the error bound of the reduction (exact to 2^-60
below 2^14 rad) plus the polynomials' truncation (< 2e-9) and rounding."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        d = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


def test_fp32_phase_sincos_error_bound(tmp_path):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "xf_phase_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I" + inc,
                           "-I" + os.path.join(ROOT, "paper_1907_05560_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "xf_phase_check.cpp"), "-o", exe])
    out = subprocess.check_output([exe], text=True)
    r = {k: float(v) for k, v in (line.split() for line in out.splitlines())}
    assert r["samples"] > 2e6
    assert r["max_abs_err_sin"] < 1.5e-7, out
    assert r["max_abs_err_cos"] < 1.5e-7, out
