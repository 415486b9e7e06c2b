"""The float-float arithmetic of XF_FP32X2 (xf_ff.cuh), checked on the host.

tests/xf_ff_check.cpp runs the header's operations and the library's own
2x2 and 3x3 propagator templates (Eq. 3.10-3.12) instantiated on the
float-float type, against long double and against the same templates in
double, on seeded inputs.  Bounds: a sum, product or fused product-sum
within 3e-14 of the exact result relative to its operands' magnitudes (the
double-float unit roundoff is 2^-47 = 7.1e-15 for a correctly rounded
operation; these sloppy forms stay within a few units), the reciprocal
square root within 3e-14; one propagation within 1e-10 of the double
result for |T| <= 1 and phases up to 3e3 rad (a relative eigenvalue error
of a few 1e-15 times the phase); the phase sine-cosine (Cody-Waite reduction
by pi/2 and Taylor polynomials in float-float) within four units of the
float-float rounding of the phase itself."""
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


def test_float_float_arithmetic_and_propagators(tmp_path):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "xf_ff_check")
    # no contraction: the error-free transformations need their roundings
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + inc,
                           "-I" + os.path.join(ROOT, "paper_1907_05560_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "xf_ff_check.cpp"), "-o", exe])
    out = subprocess.check_output([exe], text=True)
    r = {k: float(v) for k, v in (line.split() for line in out.splitlines())}
    assert r["add_rel"] < 3e-14 and r["mul_rel"] < 3e-14 and r["fma_rel"] < 3e-14, out
    assert r["rsqrt_rel"] < 3e-14, out
    assert r["prop3_abs"] < 1e-10 and r["prop2_abs"] < 1e-10, out
    assert r["phase_over"] < 4.0, out
