"""Thin ctypes binding of libxf.so (include/xf.h): argument marshalling only.

Every step of the integration runs in the library's CUDA kernels.  PyTorch is
used only for device memory (its caching allocator, through the allocator
hook) and streams.  Loading fails loudly if libxf.so has not been built or no
GPU is usable: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxf.so")

XF_OK = 0
XF_PENDING = 1
STATUS = {0: "XF_OK", 1: "XF_PENDING", -1: "XF_E_ARG", -2: "XF_E_STATE", -3: "XF_E_NOMEM",
          -4: "XF_E_CUDA", -5: "XF_E_NONFINITE", -6: "XF_E_BARRIER_TIMEOUT", -7: "XF_E_UNSTABLE",
          -8: "XF_E_BUSY", -9: "XF_E_TOO_BIG", -10: "XF_E_NOTFOUND", -11: "XF_E_TIMEOUT",
          -12: "XF_E_UNSUPPORTED", -13: "XF_E_STEPSIZE", -14: "XF_E_BUDGET"}
STATUS_CODE = {v: k for k, v in STATUS.items()}


class XFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class XFParams(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32), ("version", ctypes.c_uint32),
        ("stepper", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("geometry", ctypes.c_int32), ("hierarchy", ctypes.c_int32),
        ("matter", ctypes.c_int32), ("n_phi", ctypes.c_int32), ("form", ctypes.c_int32),
        ("strict", ctypes.c_int32),
        ("R_nu_km", ctypes.c_double), ("mu0_per_km", ctypes.c_double),
        ("E_min_MeV", ctypes.c_double), ("E_max_MeV", ctypes.c_double),
        ("dm2_eV2", ctypes.c_double * 2), ("theta", ctypes.c_double * 3),
        ("ne_ref_cm3", ctypes.c_double), ("r_ref_km", ctypes.c_double), ("ne_power", ctypes.c_double),
        ("nb0_cm3", ctypes.c_double), ("h_ns_km", ctypes.c_double), ("Ye", ctypes.c_double),
        ("T_MeV", ctypes.c_double * 4), ("eta", ctypes.c_double * 4), ("L", ctypes.c_double * 4),
        ("eps_perturb", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("eps0", ctypes.c_double), ("ksi", ctypes.c_double), ("dr_max_km", ctypes.c_double),
    ]


class XFProblem(ctypes.Structure):
    _fields_ = [("n_E", ctypes.c_int32), ("n_u", ctypes.c_int32), ("n_flavor", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("params", XFParams)]


class XFServerCfg(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("max_jobs", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_int64),
                ("chunk_steps", ctypes.c_int64), ("queue_cap", ctypes.c_int32), ("stepper", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_flavor", ctypes.c_int32), ("tile_pairs", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class XFJob(ctypes.Structure):
    _fields_ = [("problem", XFProblem), ("r0_km", ctypes.c_double), ("dr_km", ctypes.c_double),
                ("n_steps", ctypes.c_int64), ("rho0", ctypes.POINTER(ctypes.c_double)),
                ("keep_state", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class XFJobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("steps_done", ctypes.c_int64),
                ("r_km", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class XFServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("resident", ctypes.c_int64), ("max_resident", ctypes.c_int64), ("epochs", ctypes.c_int64),
                ("bin_steps", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("mem_used_bytes", ctypes.c_int64), ("mem_peak_bytes", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class XFAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


# every symbol include/xf.h declares, with its ctypes signature
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "xf_params_default": (None, [ctypes.POINTER(XFParams)]),
    "xf_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(XFParams),
                                 ctypes.POINTER(_P)]),
    "xf_create_ex": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(XFParams),
                                    ctypes.POINTER(XFAllocator), ctypes.POINTER(_P)]),
    "xf_destroy": (ctypes.c_int, [_P]),
    "xf_set_stream": (ctypes.c_int, [_P, _P]),
    "xf_set_state": (ctypes.c_int, [_P, _D, ctypes.c_size_t, ctypes.c_double]),
    "xf_init_state": (ctypes.c_int, [_P, ctypes.c_double]),
    "xf_step": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double]),
    "xf_step_async": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double]),
    "xf_sync": (ctypes.c_int, [_P]),
    "xf_get_state": (ctypes.c_int, [_P, _D, ctypes.c_size_t, _D, ctypes.POINTER(ctypes.c_int64)]),
    "xf_moments": (ctypes.c_int, [_P, _D, _D, ctypes.c_size_t]),
    "xf_outputs": (ctypes.c_int, [_P, _D, _D, _D, ctypes.c_size_t]),
    "xf_tables": (ctypes.c_int, [_P, _D, _D]),
    "xf_launch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "xf_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    "xf_get_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "xf_create_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(XFProblem), ctypes.POINTER(XFAllocator),
                                       ctypes.POINTER(_P)]),
    "xf_batch_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "xf_batch_set_state": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_size_t, ctypes.c_double]),
    "xf_set_psi": (ctypes.c_int, [_P, _D, ctypes.c_size_t, ctypes.c_double]),
    "xf_get_psi": (ctypes.c_int, [_P, _D, ctypes.c_size_t, _D, ctypes.POINTER(ctypes.c_int64)]),
    "xf_batch_set_psi": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_size_t, ctypes.c_double]),
    "xf_batch_get_psi": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_size_t, _D,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "xf_batch_init_state": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "xf_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_size_t, _D,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "xf_batch_outputs": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D, ctypes.c_size_t]),
    "xf_batch_run_moments": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, ctypes.c_size_t]),
    "xf_evolve": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int64, ctypes.c_double]),
    "xf_moments_ex": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_size_t]),
    "xf_checkpoint_bytes": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "xf_checkpoint_save": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "xf_checkpoint_save_async": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "xf_checkpoint_wait": (ctypes.c_int, [_P]),
    "xf_checkpoint_load": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "xf_angle_average": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_size_t]),
    "xf_autotune": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), _D]),
    "xf_batch_evolve": (ctypes.c_int, [_P, _D, ctypes.c_int64, _D]),
    "xf_adapt_status": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D, _D,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _D]),
    "xf_batch_step": (ctypes.c_int, [_P, ctypes.c_int64, _D]),
    "xf_batch_status": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int64), _D]),
    "xf_server_create": (ctypes.c_int, [ctypes.POINTER(XFServerCfg), ctypes.POINTER(_P)]),
    "xf_submit": (ctypes.c_int, [_P, ctypes.POINTER(XFJob), ctypes.POINTER(ctypes.c_uint64)]),
    "xf_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(XFJobResult), _D, ctypes.c_size_t]),
    "xf_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
    "xf_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(XFServerStats)]),
    "xf_server_destroy": (ctypes.c_int, [_P]),
    "xf_peak": (ctypes.c_int, [ctypes.c_int, _D]),
    "xf_step_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(XFParams),
                                       _P, ctypes.c_double, ctypes.c_int64, ctypes.c_double, _P]),
    "xf_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "xf_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libxf.so and bind every entry point (no GPU needed to load)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(nvcc for sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def params_from(p: I.Problem) -> XFParams:
    L = load()
    x = XFParams()
    L.xf_params_default(ctypes.byref(x))
    x.stepper, x.precision, x.geometry = p.stepper, p.precision, p.geometry
    x.hierarchy, x.matter, x.strict = p.hierarchy, p.matter, p.strict
    x.n_phi, x.form = p.n_phi, p.form
    x.R_nu_km, x.mu0_per_km, x.E_min_MeV, x.E_max_MeV = p.R_nu, p.mu0, p.E_min, p.E_max
    x.dm2_eV2[:] = list(p.dm2)
    x.theta[:] = list(p.theta)
    x.ne_ref_cm3, x.r_ref_km, x.ne_power = p.ne_ref, p.r_ref, p.ne_power
    x.nb0_cm3, x.h_ns_km, x.Ye = p.nb0, p.h_ns, p.Ye
    x.T_MeV[:] = list(p.T)
    x.eta[:] = list(p.eta)
    x.L[:] = list(p.L)
    x.eps_perturb, x.seed = p.eps, p.seed
    x.eps0, x.ksi, x.dr_max_km = p.eps0, p.ksi, p.dr_max
    return x


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self._alloc = ALLOC_FN(self._a)
        self._free = FREE_FN(self._f)
        self.struct = XFAllocator(self._alloc, self._free, None)

    def _a(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.dev)
        except Exception:
            return None

    def _f(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


class Context:
    """One flavor-evolution problem resident on the GPU (xf_ctx)."""

    def __init__(self, problem: I.Problem, allocator: str = "torch", stream=None):
        self.L = load()
        self.problem = problem
        self.n_f = problem.n_f
        self.n_bins = problem.n_bins
        self.n_doubles = self.n_bins * self.n_f * self.n_f
        prm = params_from(problem)
        h = _P()
        self._allocator = None
        if allocator == "torch":
            self._allocator = _TorchAllocator()
            rc = self.L.xf_create_ex(problem.n_E, problem.n_u, problem.n_f, ctypes.byref(prm),
                                     ctypes.byref(self._allocator.struct), ctypes.byref(h))
        else:
            rc = self.L.xf_create(problem.n_E, problem.n_u, problem.n_f, ctypes.byref(prm),
                                  ctypes.byref(h))
        if rc != XF_OK:
            raise XFError(rc, self.L.xf_last_error(None).decode())
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    # -- helpers
    def _check(self, rc: int):
        if rc != XF_OK:
            raise XFError(rc, self.L.xf_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.xf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", 0))
        return self._check(self.L.xf_set_stream(self.h, _P(ptr)))

    def set_state(self, rho: np.ndarray, r_km: float):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        return self._check(self.L.xf_set_state(self.h, _dp(rho), rho.size, float(r_km)))

    def init_state(self, r_km: float):
        return self._check(self.L.xf_init_state(self.h, float(r_km)))

    def step(self, n_steps: int, dr_km: float):
        return self._check(self.L.xf_step(self.h, int(n_steps), float(dr_km)))

    def step_async(self, n_steps: int, dr_km: float):
        return self._check(self.L.xf_step_async(self.h, int(n_steps), float(dr_km)))

    def sync(self):
        return self._check(self.L.xf_sync(self.h))

    def get_state(self, out: np.ndarray | None = None):
        rho = out if out is not None else np.empty(self.n_doubles)
        r = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._check(self.L.xf_get_state(self.h, _dp(rho), rho.size, ctypes.byref(r), ctypes.byref(n)))
        return rho, r.value, n.value

    def set_psi(self, psi: np.ndarray, r_km: float, i: int = 0):
        """Wavefunction form: [s][u][phi][E][a][i] as (re, im) pairs."""
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        return self._check(self.L.xf_batch_set_psi(self.h, i, _dp(psi), psi.size, float(r_km)))

    def get_psi(self, i: int = 0, out: np.ndarray | None = None):
        p = getattr(self, "problems", [self.problem])[i]
        psi = out if out is not None else np.empty(p.n_bins * 2 * p.n_f * p.n_f)
        r = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._check(self.L.xf_batch_get_psi(self.h, i, _dp(psi), psi.size, ctypes.byref(r), ctypes.byref(n)))
        return psi, r.value, n.value

    def moments(self):
        m = self.n_f * self.n_f
        M0, M1 = np.empty(m), np.empty(m)
        self._check(self.L.xf_moments(self.h, _dp(M0), _dp(M1), m))
        return M0, M1

    def evolve(self, r_end_km: float, max_iters: int = 1 << 40, dr0_km: float = 0.0):
        """Error-controlled integration to r_end_km (XF_EXPH_ADAPTIVE)."""
        return self._check(self.L.xf_evolve(self.h, float(r_end_km), int(max_iters), float(dr0_km)))

    def checkpoint_bytes(self, i: int = 0) -> int:
        n = ctypes.c_size_t(0)
        self._check(self.L.xf_checkpoint_bytes(self.h, i, ctypes.byref(n)))
        return n.value

    def checkpoint_save(self, i: int = 0, buf: np.ndarray | None = None) -> np.ndarray:
        """Synchronous checkpoint of problem i into a uint8 array."""
        n = self.checkpoint_bytes(i)
        b = buf if buf is not None else np.empty(n, dtype=np.uint8)
        self._check(self.L.xf_checkpoint_save(self.h, i, ctypes.c_void_p(b.ctypes.data), n))
        return b

    def checkpoint_save_async(self, buf: np.ndarray, i: int = 0):
        """Start an asynchronous checkpoint into `buf` (kept alive by the
        caller until checkpoint_wait)."""
        self._check(self.L.xf_checkpoint_save_async(self.h, i, ctypes.c_void_p(buf.ctypes.data), buf.size))

    def checkpoint_wait(self):
        return self._check(self.L.xf_checkpoint_wait(self.h))

    def checkpoint_load(self, buf: np.ndarray, i: int = 0):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        return self._check(self.L.xf_checkpoint_load(self.h, i, ctypes.c_void_p(b.ctypes.data), b.size))

    def angle_average(self, i: int = 0) -> np.ndarray:
        """Dump mode 2: [2][n_u][n_f^2] energy-averaged density matrices."""
        p = self.problems[i] if hasattr(self, "problems") else self.problem
        out = np.empty(2 * p.n_u * p.n_phi * p.n_f * p.n_f)
        self._check(self.L.xf_angle_average(self.h, i, _dp(out), out.size))
        return out

    def autotune(self, n_probe: int, dr_km: float = 0.0, candidates=None):
        """Measured tile-size search (xf_autotune); returns (tile, ms per step)."""
        best, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        if candidates is None:
            arr, n = None, 0
        else:
            arr = (ctypes.c_int * len(candidates))(*candidates)
            n = len(candidates)
        self._check(self.L.xf_autotune(self.h, int(n_probe), float(dr_km), arr, n, ctypes.byref(best),
                                       ctypes.byref(ms)))
        return best.value, ms.value

    def adapt_status(self, i: int = 0):
        st, r, h, e = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        na, nr = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self.L.xf_adapt_status(self.h, i, ctypes.byref(st), ctypes.byref(r), ctypes.byref(h),
                                           ctypes.byref(na), ctypes.byref(nr), ctypes.byref(e)))
        return dict(status=STATUS.get(st.value, st.value), r=r.value, h_next=h.value, n_accepted=na.value,
                    n_rejected=nr.value, err=e.value)

    def moments_ex(self, i: int = 0):
        """M0..M3 [4][n_f^2] (FP64 sums of the current state)."""
        n_f = self.problems[i].n_f if hasattr(self, "problems") else self.n_f
        M = np.empty(4 * n_f * n_f)
        self._check(self.L.xf_moments_ex(self.h, i, _dp(M), M.size))
        return M.reshape(4, -1)

    def run_moments(self, i: int = 0):
        """Traceless M0, M1 of problem i's state as the integrator summed them."""
        n_f = self.problems[i].n_f if hasattr(self, "problems") else self.n_f
        M0, M1 = np.empty(n_f * n_f), np.empty(n_f * n_f)
        self._check(self.L.xf_batch_run_moments(self.h, i, _dp(M0), _dp(M1), n_f * n_f))
        return M0, M1

    def outputs(self):
        p, t, q = np.empty(self.n_bins), np.empty(self.n_bins), np.empty(self.n_bins)
        self._check(self.L.xf_outputs(self.h, _dp(p), _dp(t), _dp(q), self.n_bins))
        return p, t, q

    def tables(self):
        E = np.empty(self.problem.n_E)
        phi = np.empty(4 * self.problem.n_E)
        self._check(self.L.xf_tables(self.h, _dp(E), _dp(phi)))
        return E, phi.reshape(4, -1)

    def set_option(self, option: int, value: int):
        return self._check(self.L.xf_set_option(self.h, int(option), int(value)))

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64(0)
        self._check(self.L.xf_get_option(self.h, int(option), ctypes.byref(v)))
        return v.value

    def launch_info(self):
        g, t, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.L.xf_launch_info(self.h, ctypes.byref(g), ctypes.byref(t), ctypes.byref(b)))
        return g.value, t.value, b.value


OPT_GRID, OPT_BARRIER_TIMEOUT_NS, OPT_TEST_SKIP_ARRIVAL, OPT_TILE_PAIRS, OPT_GRAPH, OPT_DYNAMIC_TILES = 1, 2, 3, 4, 5, 6


class Batch(Context):
    """Several problems advanced together in one persistent launch (a batch
    xf_ctx).  Problems may differ in size, flavors and physics; stepper and
    precision are shared."""

    def __init__(self, problems, allocator: str = "torch", stream=None):  # noqa: D401
        self.L = load()
        self.problems = list(problems)
        self.problem = self.problems[0]
        arr = (XFProblem * len(self.problems))()
        for k, p in enumerate(self.problems):
            arr[k].n_E, arr[k].n_u, arr[k].n_flavor, arr[k].reserved = p.n_E, p.n_u, p.n_f, 0
            arr[k].params = params_from(p)
        h = _P()
        self._allocator = _TorchAllocator() if allocator == "torch" else None
        alloc = ctypes.byref(self._allocator.struct) if self._allocator else None
        rc = self.L.xf_create_batch(len(self.problems), arr, alloc, ctypes.byref(h))
        if rc != XF_OK:
            raise XFError(rc, self.L.xf_last_error(None).decode())
        self.h = h
        self.n_f = self.problem.n_f
        self.n_bins = self.problem.n_bins
        self.n_doubles = self.n_bins * self.n_f * self.n_f
        if stream is not None:
            self.set_stream(stream)

    def __len__(self):
        return len(self.problems)

    def _size(self, i):
        p = self.problems[i]
        return p.n_bins * p.n_f * p.n_f

    def set_state_i(self, i: int, rho: np.ndarray, r_km: float):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        return self._check(self.L.xf_batch_set_state(self.h, i, _dp(rho), rho.size, float(r_km)))

    def init_state_i(self, i: int, r_km: float):
        return self._check(self.L.xf_batch_init_state(self.h, i, float(r_km)))

    def get_state_i(self, i: int, out: np.ndarray | None = None):
        rho = out if out is not None else np.empty(self._size(i))
        r = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._check(self.L.xf_batch_get_state(self.h, i, _dp(rho), rho.size, ctypes.byref(r), ctypes.byref(n)))
        return rho, r.value, n.value

    def outputs_i(self, i: int):
        p = self.problems[i]
        nb = p.n_bins
        a, b, c = np.empty(nb), np.empty(nb), np.empty(nb)
        self._check(self.L.xf_batch_outputs(self.h, i, _dp(a), _dp(b), _dp(c), nb))
        return a, b, c

    def step_all(self, n_steps: int, dr_km=None):
        dr = None if dr_km is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(dr_km, dtype=np.float64), (len(self.problems),)))
        return self._check(self.L.xf_batch_step(self.h, int(n_steps), _dp(dr) if dr is not None else None))

    def evolve_all(self, r_end_km, max_iters: int = 1 << 40, dr0_km=None):
        n = len(self.problems)
        re = np.ascontiguousarray(np.broadcast_to(np.asarray(r_end_km, dtype=np.float64), (n,)))
        d0 = None if dr0_km is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(dr0_km, dtype=np.float64), (n,)))
        return self._check(self.L.xf_batch_evolve(self.h, _dp(re), int(max_iters),
                                                  _dp(d0) if d0 is not None else None))

    def status_i(self, i: int):
        st, n, r = ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_double(0.0)
        self._check(self.L.xf_batch_status(self.h, i, ctypes.byref(st), ctypes.byref(n), ctypes.byref(r)))
        return STATUS.get(st.value, st.value), n.value, r.value


PEAK_FP64_FMA, PEAK_FP32_FMA, PEAK_FP64_RSQRT, PEAK_FP64_SINCOS = 0, 1, 2, 3


def peak(which: int) -> float:
    """Measured FMA throughput (FLOP/s), or calls/s of the FP64 reciprocal
    square root or sine-cosine pair, on the current device."""
    v = ctypes.c_double(0.0)
    rc = load().xf_peak(int(which), ctypes.byref(v))
    if rc != XF_OK:
        raise XFError(rc, "xf_peak failed")
    return v.value


def status_str(code: int) -> str:
    return load().xf_status_str(code).decode()


class Server:
    """Continuous-batching job server (xf_server_*): jobs are admitted into
    GPU slots as slots and memory free up and advance together in chunks."""

    def __init__(self, max_jobs: int, mem_budget_bytes: int, chunk_steps: int, *, stepper=I.EXPH,
                 precision=I.FP32_M64, n_flavor: int = 2, queue_cap: int = 100000, tile_pairs: int = 0):
        self.L = load()
        cfg = XFServerCfg()
        cfg.size = ctypes.sizeof(XFServerCfg)
        cfg.max_jobs, cfg.mem_budget_bytes, cfg.chunk_steps = max_jobs, int(mem_budget_bytes), chunk_steps
        cfg.queue_cap, cfg.stepper, cfg.precision, cfg.n_flavor = queue_cap, stepper, precision, n_flavor
        cfg.tile_pairs = tile_pairs
        h = _P()
        rc = self.L.xf_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != XF_OK:
            raise XFError(rc, "xf_server_create failed")
        self.h = h
        self._sizes = {}

    def submit(self, p: I.Problem, rho0: np.ndarray | None = None, keep_state: bool = False,
               r0: float | None = None, dr: float | None = None, n_steps: int | None = None) -> int:
        job = XFJob()
        job.problem.n_E, job.problem.n_u, job.problem.n_flavor, job.problem.reserved = p.n_E, p.n_u, p.n_f, 0
        job.problem.params = params_from(p)
        job.r0_km = p.r0 if r0 is None else r0
        job.dr_km = p.h if dr is None else dr
        job.n_steps = p.n_steps if n_steps is None else n_steps
        keep = None
        if rho0 is not None:
            keep = np.ascontiguousarray(rho0, dtype=np.float64)
            job.rho0 = _dp(keep)
        job.keep_state = 1 if keep_state else 0
        jid = ctypes.c_uint64(0)
        rc = self.L.xf_submit(self.h, ctypes.byref(job), ctypes.byref(jid))
        if rc != XF_OK:
            raise XFError(rc, "xf_submit")
        self._sizes[jid.value] = p.n_bins * p.n_f * p.n_f
        return jid.value

    def poll(self, job_id: int, want_state: bool = False):
        """None while pending, else (result dict, state or None)."""
        res = XFJobResult()
        out = np.empty(self._sizes.get(job_id, 0)) if want_state else None
        rc = self.L.xf_poll(self.h, job_id, ctypes.byref(res), _dp(out) if out is not None else None,
                            out.size if out is not None else 0)
        if rc == XF_PENDING:
            return None
        if rc != XF_OK:
            raise XFError(rc, "xf_poll")
        self._sizes.pop(job_id, None)
        return ({"status": STATUS.get(res.status, res.status), "steps": res.steps_done, "r": res.r_km,
                 "t_submit": res.t_submit, "t_start": res.t_start, "t_done": res.t_done}, out)

    def drain(self, timeout_s: float = 600.0):
        rc = self.L.xf_server_drain(self.h, float(timeout_s))
        if rc != XF_OK:
            raise XFError(rc, "xf_server_drain")

    def stats(self) -> dict:
        st = XFServerStats()
        self.L.xf_server_get_stats(self.h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in XFServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.xf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
