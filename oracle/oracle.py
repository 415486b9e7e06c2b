"""ctypes wrapper for the FP64 CPU oracle (oracle/xf_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs are the only callers.  The CUDA library never
imports this module and this module never imports the CUDA library.

Packed state layout (shared interface, both sides write their own code for
it): doubles [s][u][E][n_f*n_f] with s = 0 nu, 1 nubar; per bin the n_f real
diagonal entries, then (Re, Im) of the upper triangle in row order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
# A prebuilt oracle library to load instead (tests/test_oracle_mutations.py
# points this at deliberately broken copies to show that the pins catch them).
_LIB_OVERRIDE = os.environ.get("XF_ORACLE_LIB")

_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n_E", ctypes.c_int32), ("n_u", ctypes.c_int32), ("n_f", ctypes.c_int32),
        ("stepper", ctypes.c_int32), ("geometry", ctypes.c_int32),
        ("hierarchy", ctypes.c_int32), ("matter", ctypes.c_int32),
        ("n_threads", ctypes.c_int32), ("renorm", ctypes.c_int32), ("n_phi", ctypes.c_int32),
        ("R_nu", ctypes.c_double), ("mu0", ctypes.c_double),
        ("E_min", ctypes.c_double), ("E_max", ctypes.c_double),
        ("dm2", ctypes.c_double * 2), ("theta", ctypes.c_double * 3),
        ("ne_ref", ctypes.c_double), ("r_ref", ctypes.c_double), ("ne_power", ctypes.c_double),
        ("nb0", ctypes.c_double), ("h_ns", ctypes.c_double), ("Ye", ctypes.c_double),
        ("T", ctypes.c_double * 4), ("eta", ctypes.c_double * 4), ("L", ctypes.c_double * 4),
        ("eps", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("eps0", ctypes.c_double), ("ksi", ctypes.c_double), ("dr_max", ctypes.c_double),
    ]


CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def compile_to(src: str, out: str) -> None:
    """gcc the oracle source `src` into the shared library `out`."""
    subprocess.check_call(["gcc", *CFLAGS, src, "-o", out + ".tmp", "-lm"])
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liborc.so with gcc (no CUDA)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_to(_SRC, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(OrcParams)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_tables.argtypes = [P, dp, dp, dp, dp]
        L.orc_init_state.argtypes = [P, dp]
        L.orc_evolve.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64)]
        L.orc_moments.argtypes = [P, dp, ctypes.c_double, dp, dp]
        L.orc_moments_ex.argtypes = [P, dp, ctypes.c_double, dp]
        L.orc_cyl_pair.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_init_psi.argtypes = [P, dp]
        L.orc_psi_to_rho.argtypes = [P, dp, dp]
        L.orc_evolve_psi.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64)]
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.orc_evolve_adaptive.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int64, dp, dp, i64p, i64p]
        L.orc_attempt_adaptive.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_expm.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
        L.orc_eigh.argtypes = [ctypes.c_int, dp, dp, dp]
        L.orc_fd_integral.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_fd_integral.restype = ctypes.c_double
        L.orc_vac_coeff.restype = ctypes.c_double
        L.orc_matter_coeff.restype = ctypes.c_double
        L.orc_matter_A.argtypes = [P, ctypes.c_double]
        L.orc_matter_A.restype = ctypes.c_double
        _lib = L
    return _lib


def params(p, n_threads: int = 0, renorm: bool = False) -> OrcParams:
    """Oracle parameter block from an inputs.Problem (renorm: restore each
    bin's entry tr(T^2) after every step)."""
    o = OrcParams()
    o.n_E, o.n_u, o.n_f = p.n_E, p.n_u, p.n_f
    o.stepper, o.geometry, o.hierarchy, o.matter = p.stepper, p.geometry, p.hierarchy, p.matter
    o.n_threads = n_threads
    o.renorm = 1 if renorm else 0
    o.n_phi = getattr(p, "n_phi", 1)
    o.R_nu, o.mu0, o.E_min, o.E_max = p.R_nu, p.mu0, p.E_min, p.E_max
    o.dm2[:] = list(p.dm2)
    o.theta[:] = list(p.theta)
    o.ne_ref, o.r_ref, o.ne_power = p.ne_ref, p.r_ref, p.ne_power
    o.nb0, o.h_ns, o.Ye = p.nb0, p.h_ns, p.Ye
    o.T[:] = list(p.T)
    o.eta[:] = list(p.eta)
    o.L[:] = list(p.L)
    o.eps, o.seed = p.eps, p.seed
    o.eps0, o.ksi, o.dr_max = p.eps0, p.ksi, p.dr_max
    return o


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def state_size(p) -> int:
    return 2 * p.n_u * getattr(p, "n_phi", 1) * p.n_E * p.n_f * p.n_f


def tables(p):
    o = params(p)
    E = np.zeros(p.n_E)
    u = np.zeros(p.n_u)
    phi = np.zeros((4, p.n_E))
    Hv = np.zeros((p.n_E, p.n_f * p.n_f))
    rc = lib().orc_tables(ctypes.byref(o), _dp(E), _dp(u), _dp(phi), _dp(Hv))
    if rc:
        raise ValueError(f"orc_tables: {rc}")
    return E, u, phi, Hv


def init_state(p) -> np.ndarray:
    o = params(p)
    rho = np.zeros(state_size(p))
    rc = lib().orc_init_state(ctypes.byref(o), _dp(rho))
    if rc:
        raise ValueError(f"orc_init_state: {rc}")
    return rho


def evolve(p, rho: np.ndarray, r0: float, h: float, n_steps: int, n_threads: int = 0, renorm: bool = False):
    """Returns (rho_out, status, steps_done); status 1 = non-finite stop."""
    o = params(p, n_threads, renorm)
    out = np.ascontiguousarray(rho, dtype=np.float64).copy()
    done = ctypes.c_int64(0)
    rc = lib().orc_evolve(ctypes.byref(o), _dp(out), r0, h, int(n_steps), ctypes.byref(done))
    if rc < 0:
        raise ValueError(f"orc_evolve: {rc}")
    return out, rc, done.value


def evolve_adaptive(p, rho: np.ndarray, r0: float, r_end: float, h0: float, max_iters: int = 1 << 40,
                    n_threads: int = 0):
    """Error-controlled evolution (eps0, ksi, dr_max from p).  Returns
    (rho_out, status, r, h_next, n_accepted, n_rejected); status 0 = reached
    r_end, 1 = non-finite, 2 = iteration budget spent, 3 = step underflow."""
    o = params(p, n_threads)
    out = np.ascontiguousarray(rho, dtype=np.float64).copy()
    r, h = ctypes.c_double(0.0), ctypes.c_double(0.0)
    na, nr = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib().orc_evolve_adaptive(ctypes.byref(o), _dp(out), r0, r_end, h0, int(max_iters), ctypes.byref(r),
                                   ctypes.byref(h), ctypes.byref(na), ctypes.byref(nr))
    if rc < 0:
        raise ValueError(f"orc_evolve_adaptive: {rc}")
    return out, rc, r.value, h.value, na.value, nr.value


def attempt_adaptive(p, rho: np.ndarray, r: float, h: float, n_threads: int = 0):
    """One attempt: returns (rho_coarse, rho_fine, err, status)."""
    o = params(p, n_threads)
    out = np.ascontiguousarray(rho, dtype=np.float64).copy()
    fine = np.zeros_like(out)
    err = ctypes.c_double(0.0)
    rc = lib().orc_attempt_adaptive(ctypes.byref(o), _dp(out), r, h, ctypes.byref(err), _dp(fine))
    if rc < 0:
        raise ValueError(f"orc_attempt_adaptive: {rc}")
    return out, fine, err.value, rc


def psi_size(p) -> int:
    return 2 * p.n_u * getattr(p, "n_phi", 1) * p.n_E * 2 * p.n_f * p.n_f


def init_psi(p) -> np.ndarray:
    """Seeded wavefunctions [s][t][E][a][i] (Re, Im): one per initial flavor."""
    o = params(p)
    psi = np.zeros(psi_size(p))
    rc = lib().orc_init_psi(ctypes.byref(o), _dp(psi))
    if rc:
        raise ValueError(f"orc_init_psi: {rc}")
    return psi


def psi_to_rho(p, psi: np.ndarray) -> np.ndarray:
    o = params(p)
    rho = np.zeros(state_size(p))
    rc = lib().orc_psi_to_rho(ctypes.byref(o), _dp(np.ascontiguousarray(psi, dtype=np.float64)), _dp(rho))
    if rc:
        raise ValueError(f"orc_psi_to_rho: {rc}")
    return rho


def evolve_psi(p, psi: np.ndarray, r0: float, h: float, n_steps: int, n_threads: int = 0):
    """Wavefunction form: returns (psi_out, status, steps_done)."""
    o = params(p, n_threads)
    out = np.ascontiguousarray(psi, dtype=np.float64).copy()
    done = ctypes.c_int64(0)
    rc = lib().orc_evolve_psi(ctypes.byref(o), _dp(out), r0, h, int(n_steps), ctypes.byref(done))
    if rc < 0:
        raise ValueError(f"orc_evolve_psi: {rc}")
    return out, rc, done.value


def cyl_pair(p, r: float, j: int, jp: int):
    """Cylinder model (Eq. 3.20): (Phi' - Phi, w_jp (1 - cos(alpha_j - alpha_jp)))."""
    o = params(p)
    sh, w = np.zeros(1), np.zeros(1)
    rc = lib().orc_cyl_pair(ctypes.byref(o), float(r), int(j), int(jp), _dp(sh), _dp(w))
    if rc != 0:
        raise ValueError(f"orc_cyl_pair: {rc}")
    return float(sh[0]), float(w[0])


def moments_ex(p, rho: np.ndarray, r: float) -> np.ndarray:
    """All four moments [4][n_f*n_f] packed (M2 = M3 = 0 without azimuth bins)."""
    o = params(p)
    M = np.zeros(4 * p.n_f * p.n_f)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    rc = lib().orc_moments_ex(ctypes.byref(o), _dp(rho), r, _dp(M))
    if rc:
        raise ValueError(f"orc_moments_ex: {rc}")
    return M.reshape(4, -1)


def moments(p, rho: np.ndarray, r: float):
    o = params(p)
    M0 = np.zeros(p.n_f * p.n_f)
    M1 = np.zeros(p.n_f * p.n_f)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    lib().orc_moments(ctypes.byref(o), _dp(rho), r, _dp(M0), _dp(M1))
    return M0, M1


def expm(H_packed: np.ndarray, t: float) -> np.ndarray:
    n = int(round(np.sqrt(H_packed.size)))
    U = np.zeros(2 * n * n)
    lib().orc_expm(n, _dp(np.ascontiguousarray(H_packed, dtype=np.float64)), t, _dp(U))
    return (U[0::2] + 1j * U[1::2]).reshape(n, n)


def eigh(H_packed: np.ndarray):
    n = int(round(np.sqrt(H_packed.size)))
    w = np.zeros(n)
    V = np.zeros(2 * n * n)
    lib().orc_eigh(n, _dp(np.ascontiguousarray(H_packed, dtype=np.float64)), _dp(w), _dp(V))
    return w, (V[0::2] + 1j * V[1::2]).reshape(n, n)


def fd_integral(k: int, eta: float) -> float:
    return lib().orc_fd_integral(k, eta)


def vac_coeff() -> float:
    return lib().orc_vac_coeff()


def matter_coeff() -> float:
    return lib().orc_matter_coeff()


def matter_A(p, r: float) -> float:
    o = params(p)
    return lib().orc_matter_A(ctypes.byref(o), r)


# ---- packed-layout helpers (plain numpy; interpretation of the layout) ----

def unpack(rho: np.ndarray, n_f: int) -> np.ndarray:
    """Packed [..., n_f*n_f] -> complex matrices [..., n_f, n_f]."""
    x = rho.reshape(-1, n_f * n_f)
    M = np.zeros((x.shape[0], n_f, n_f), dtype=complex)
    for i in range(n_f):
        M[:, i, i] = x[:, i]
    k = n_f
    for i in range(n_f):
        for j in range(i + 1, n_f):
            z = x[:, k] + 1j * x[:, k + 1]
            M[:, i, j] = z
            M[:, j, i] = np.conj(z)
            k += 2
    return M


def pack(M: np.ndarray) -> np.ndarray:
    n_f = M.shape[-1]
    M = M.reshape(-1, n_f, n_f)
    x = np.zeros((M.shape[0], n_f * n_f))
    for i in range(n_f):
        x[:, i] = M[:, i, i].real
    k = n_f
    for i in range(n_f):
        for j in range(i + 1, n_f):
            x[:, k] = M[:, i, j].real
            x[:, k + 1] = M[:, i, j].imag
            k += 2
    return x.reshape(-1)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
