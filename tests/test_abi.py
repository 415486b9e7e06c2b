"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point include/xf.h declares, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "xf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_05560_gb300 import build, xf
    build.build()
    return xf.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("xf_create", "xf_set_state", "xf_step", "xf_get_state", "xf_moments", "xf_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1907_05560_gb300 import xf
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in xf.SIGNATURES, f"binding lacks {name}"


def test_params_default_and_status_strings(lib):
    from paper_1907_05560_gb300 import xf
    p = xf.XFParams()
    lib.xf_params_default(ctypes.byref(p))
    assert p.size == ctypes.sizeof(xf.XFParams)
    assert p.version == 3 and p.stepper == 0 and p.hierarchy == -1 and p.n_phi == 1
    assert (p.eps0, p.ksi, p.dr_max_km) == (1e-6, 0.9, 1.0)
    assert list(p.T_MeV) == [2.76, 4.01, 6.26, 6.26]
    for code, name in xf.STATUS.items():
        assert lib.xf_status_str(code).decode() == name


@pytest.mark.parametrize("mutate,dims", [
    (lambda p: None, (0, 16, 2)),
    (lambda p: None, (32, -1, 2)),
    (lambda p: None, (32, 16, 4)),
    (lambda p: setattr(p, "size", 12), (32, 16, 2)),
    (lambda p: setattr(p, "version", 99), (32, 16, 2)),
    (lambda p: setattr(p, "stepper", 7), (32, 16, 2)),
    (lambda p: (setattr(p, "stepper", 2), setattr(p, "eps0", 0.0)), (32, 16, 2)),
    (lambda p: (setattr(p, "stepper", 2), setattr(p, "ksi", 1.5)), (32, 16, 2)),
    (lambda p: (setattr(p, "stepper", 2), setattr(p, "dr_max_km", -1.0)), (32, 16, 2)),
    (lambda p: setattr(p, "hierarchy", 0), (32, 16, 2)),
    (lambda p: setattr(p, "n_phi", 0), (32, 16, 2)),
    (lambda p: (setattr(p, "n_phi", 4), setattr(p, "geometry", 1)), (32, 16, 2)),  # azimuths: bulb only
    (lambda p: setattr(p, "geometry", 2), (32, 16, 2)),  # single angle needs n_u == 1
    (lambda p: setattr(p, "R_nu_km", float("nan")), (32, 16, 2)),
    (lambda p: setattr(p, "E_max_MeV", 0.5), (32, 16, 2)),
    (lambda p: setattr(p, "mu0_per_km", -1.0), (32, 16, 2)),
    (lambda p: setattr(p, "eps_perturb", float("inf")), (32, 16, 2)),
])
def test_create_rejects_bad_arguments_without_gpu(lib, mutate, dims):
    from paper_1907_05560_gb300 import xf
    p = xf.XFParams()
    lib.xf_params_default(ctypes.byref(p))
    mutate(p)
    h = ctypes.c_void_p(123)
    rc = lib.xf_create(*dims, ctypes.byref(p), ctypes.byref(h))
    assert rc == xf.STATUS_CODE["XF_E_ARG"]
    assert h.value is None
    assert lib.xf_last_error(None).decode() != ""


def test_null_handles_are_errors_not_crashes(lib):
    from paper_1907_05560_gb300 import xf
    E = xf.STATUS_CODE["XF_E_ARG"]
    assert lib.xf_destroy(None) == 0
    assert lib.xf_step(None, 1, 0.1) == E
    assert lib.xf_set_state(None, None, 0, 1.0) == E
    assert lib.xf_get_state(None, None, 0, None, None) == E
    assert lib.xf_moments(None, None, None, 0) == E
    assert lib.xf_create(32, 16, 2, None, None) == E
    assert lib.xf_checkpoint_save(None, 0, None, 0) == E
    assert lib.xf_checkpoint_load(None, 0, None, 0) == E
    assert lib.xf_checkpoint_wait(None) == E
    assert lib.xf_angle_average(None, 0, None, 0) == E
    assert lib.xf_evolve(None, 1.0, 1, 0.1) == E
    assert lib.xf_autotune(None, 1, 0.0, None, 0, None, None) == E


@pytest.mark.parametrize("mutate,want", [
    (lambda p: setattr(p, "precision", 5), "XF_E_ARG"),
    (lambda p: (setattr(p, "precision", 4), setattr(p, "stepper", 0)), "XF_E_UNSUPPORTED"),  # RK4
    (lambda p: (setattr(p, "precision", 4), setattr(p, "stepper", 2)), "XF_E_UNSUPPORTED"),  # error-controlled
    (lambda p: (setattr(p, "precision", 4), setattr(p, "stepper", 1), setattr(p, "n_phi", 4)), "XF_E_UNSUPPORTED"),
    (lambda p: (setattr(p, "precision", 4), setattr(p, "stepper", 1), setattr(p, "form", 1)), "XF_E_UNSUPPORTED"),
    (lambda p: (setattr(p, "precision", 4), setattr(p, "stepper", 1), setattr(p, "geometry", 4)),
     "XF_E_UNSUPPORTED"),
])
def test_float_float_precision_refusals_without_gpu(lib, mutate, want):
    """XF_FP32X2 runs the predictor-corrector on density matrices of the
    bulb-type geometries with one azimuth bin; the rest is refused before
    any device call."""
    from paper_1907_05560_gb300 import xf
    p = xf.XFParams()
    lib.xf_params_default(ctypes.byref(p))
    mutate(p)
    h = ctypes.c_void_p(123)
    rc = lib.xf_create(32, 16, 2, ctypes.byref(p), ctypes.byref(h))
    assert rc == xf.STATUS_CODE[want], lib.xf_last_error(None).decode()
    assert h.value is None
