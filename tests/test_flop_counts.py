"""The algorithmic work behind bench.py's roofline, regenerated from source.

tests/xf_flopcount.cpp runs the library's own per-bin templates (xf_math.cuh,
xf_psi.cuh) on the host with a counting number type, in the order in which
the kernels' per-pair loops call them, and prints the floating-point
operations per bin-step (per bin-attempt for the error-controlled step).
These tests build it, check that every constant bench.py uses is the
counter's figure, and measure the one data-dependent input of the count, the
Jacobi sweep number of the 3x3 eigensolver, on the Hamiltonians of the
workloads the bench times (built from the oracle's tables, moments and
matter potential, i.e. Eq. 3.5-3.7 and 3.13-3.15).
"""
import math
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


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


@pytest.fixture(scope="module")
def counter(tmp_path_factory):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("flops") / "xf_flopcount")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I" + inc,
                           "-I" + os.path.join(ROOT, "paper_1907_05560_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "xf_flopcount.cpp"), "-o", exe])
    return exe


def _run(exe, *args):
    out = subprocess.check_output([exe, *args], text=True)
    return {k: float(v) for k, v in (line.split() for line in out.splitlines())}


def test_bench_constants_are_the_counted_figures(counter):
    f = _run(counter)
    # the count is taken where the Jacobi solver takes two sweeps (matter-dominated)
    assert f["sweeps_matter"] == 2 and f["sweeps_vacuum"] == 3
    assert bench.FLOPS_PER_BIN_STEP == {("exph", 3): f["exph_3"], ("rk4", 3): f["rk4_3"],
                                        ("exph", 2): f["exph_2"], ("rk4", 2): f["rk4_2"]}
    assert bench.FLOPS_PER_BIN_STEP_PSI == {("exph", 3): f["psi_exph_3"], ("rk4", 3): f["psi_rk4_3"],
                                            ("exph", 2): f["psi_exph_2"], ("rk4", 2): f["psi_rk4_2"]}
    assert bench.FLOPS_PER_BIN_ATTEMPT_2SWEEPS == {3: f["attempt_3"], 2: f["attempt_2"]}
    assert bench.FLOPS_PER_EXTRA_SWEEP == f["eig3_extra_sweep"]
    assert bench.FLOPS_PER_BIN_STEP_AZIMUTH_2F == f["azimuth_exph_2"]
    assert bench.FLOPS_PER_BIN_STEP_CYLINDER_2F == f["cylinder_exph_2"]
    assert bench.PROP3_UNCOUNTED == {"sincos_pairs": f["prop3_sincos_pairs"], "rsqrt": f["prop3_rsqrt"],
                                     "flop": f["prop3"]}


def _hamiltonians(orc, p, r, rho, stride):
    """Traceless packed 3x3 Hamiltonians H_nu, H_nubar of every energy on
    every `stride`-th angle bin at radius r (bulb geometry: G = mu0 (M0 -
    c_u M1), c_u = sqrt(1 - (R/r)^2 u); Eq. 3.4-3.7, 3.13-3.15)."""
    E, u, phi, Hv = orc.tables(p)
    M0, M1 = orc.moments(p, rho, r)
    A = orc.matter_A(p, r)
    x2 = (p.R_nu / r) ** 2
    Pe = np.diag([1.0, 0.0, 0.0])
    Hvac = orc.unpack(Hv, 3)
    G0, G1 = orc.unpack(M0, 3)[0], orc.unpack(M1, 3)[0]
    out = []
    for j in range(0, p.n_u, stride):
        c = math.sqrt(1.0 - x2 * u[j])
        G = p.mu0 * (G0 - c * G1)
        for H in (Hvac + A * Pe + G, Hvac - A * Pe - np.conj(G)):
            H = H - np.trace(H, axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
            out.append(np.stack([H[:, 0, 0].real, H[:, 1, 1].real, H[:, 0, 1].real, H[:, 0, 1].imag,
                                 H[:, 0, 2].real, H[:, 0, 2].imag, H[:, 1, 2].real, H[:, 1, 2].imag], 1))
    return np.concatenate(out)


def _sweeps(counter, H, tmp_path):
    path = str(tmp_path / "h.bin")
    np.ascontiguousarray(H, dtype=np.float64).tofile(path)
    return _run(counter, "--sweeps", path)


def test_headline_workload_takes_two_jacobi_sweeps(counter, orc, tmp_path):
    """Over the bench's timed range of the three-flavor 1000 x 200 workload
    (about 25 -> 75 km) every Hamiltonian of the seeded state takes two
    sweeps, the sweep count at which the headline flop figure is taken."""
    p = I.bulb3f_1000x200()
    rho = orc.init_state(p)
    for r in (25.0, 50.0, 75.0):
        s = _sweeps(counter, _hamiltonians(orc, p, r, rho, 10), tmp_path)
        assert s["hamiltonians"] == 2 * 100 * p.n_E
        assert s["mean_sweeps"] == 2.0, (r, s)


def test_error_controlled_leg_sweep_count(counter, orc, tmp_path):
    """The error-controlled bench leg starts the same workload at 250 km;
    its flop figure is the two-sweep count plus FLOPS_PER_EXTRA_SWEEP for
    each sweep beyond two of its four eigendecompositions per bin-attempt,
    at the mean sweep count of the Hamiltonians there."""
    p = I.bulb3f_1000x200_from_250km()
    rho = orc.init_state(p)
    mean = np.mean([_sweeps(counter, _hamiltonians(orc, p, r, rho, 10), tmp_path)["mean_sweeps"]
                    for r in (250.0, 258.0)])
    assert abs(mean - bench.ADAPT_MEAN_SWEEPS) < 0.001, mean
    want = bench.FLOPS_PER_BIN_ATTEMPT_2SWEEPS[3] + 4 * (bench.ADAPT_MEAN_SWEEPS - 2) * bench.FLOPS_PER_EXTRA_SWEEP
    assert bench.flops_per_bin_attempt(3) == pytest.approx(want)
