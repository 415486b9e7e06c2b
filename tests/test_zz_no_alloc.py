"""xf_step_noalloc: stepping a state held in the caller's device memory with no
allocation inside the call.

Some users of the library cannot allocate device memory at the moment they
step a problem: their code runs inside a memory pool that owns the whole
device budget, or inside a host application that forbids allocation on its
hot path.  xf_step_noalloc takes the state from a device buffer the caller
already owns, writes the result back into it, and draws all of its working
memory from a fixed-size device array inside the library.

These tests check, through the C ABI, that it produces the same states as
the regular entry points (xf_create, xf_set_state, xf_step, xf_get_state)
within the parity tolerance of the other GPU tests, on two calls in a row,
and that a problem too large for the fixed array is refused.
"""
import ctypes

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-9  # same gate as the FP64 parity tests: |diff| / tr(rho) per bin


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05560_gb300 import build, xf
    build.build()
    return torch, xf, xf.load()


def _rel(a, b, n_f):
    A = a.reshape(-1, n_f * n_f)
    B = b.reshape(-1, n_f * n_f)
    return float((np.abs(A - B).max(1) / np.abs(B[:, :n_f].sum(1))).max())


CASES = [
    # two flavors, RK4, one CTA
    I.Problem(n_E=32, n_u=16, n_f=2, stepper=I.RK4, mu0=1e5, r0=50.0, r1=51.0, n_steps=100,
              eps=1e-2, seed=21),
    # three flavors, predictor-corrector with matter, a multi-CTA grid with a ragged tail
    I.Problem(n_E=64, n_u=61, n_f=3, stepper=I.EXPH, mu0=1e5, dm2=(7.5e-5, 2.4e-3),
              theta=(0.59, 0.15, 0.72), hierarchy=+1, matter=I.MATTER_POWER, ne_ref=1e33,
              r0=50.0, r1=50.5, n_steps=50, eps=1e-2, seed=22),
]


@pytest.mark.parametrize("p", CASES, ids=["2f-rk4", "3f-exph-multicta"])
def test_noalloc_matches_regular_entry_points_on_two_calls(env, p):
    torch, xf, L = env
    # reference: the regular, allocating entry points
    ctx = xf.Context(p)
    ctx.init_state(p.r0)
    rho0, _, _ = ctx.get_state()
    ctx.step(p.n_steps, p.h)
    ref1, r1, _ = ctx.get_state()
    ctx.step(p.n_steps, p.h)
    ref2, r2, _ = ctx.get_state()
    ctx.close()

    # the same two calls through xf_step_noalloc on a caller-owned device buffer
    prm = xf.params_from(p)
    dev = torch.tensor(rho0, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.xf_step_noalloc(p.n_E, p.n_u, p.n_f, ctypes.byref(prm), ctypes.c_void_p(dev.data_ptr()),
                           p.r0, p.n_steps, p.h, stream)
    assert rc == 0, xf.status_str(rc)
    out1 = dev.cpu().numpy().copy()
    rc = L.xf_step_noalloc(p.n_E, p.n_u, p.n_f, ctypes.byref(prm), ctypes.c_void_p(dev.data_ptr()),
                           r1, p.n_steps, p.h, stream)
    assert rc == 0, xf.status_str(rc)
    out2 = dev.cpu().numpy().copy()

    assert np.abs(ref1 - rho0).max() > 1e-6  # the state moved
    assert _rel(out1, ref1, p.n_f) < TOL
    assert _rel(out2, ref2, p.n_f) < TOL


def test_noalloc_refuses_problem_larger_than_its_array(env):
    torch, xf, L = env
    p = I.bulb3f_1000x200()  # 400,000 3x3 bins: about 150 MB of FP64 working memory
    prm = xf.params_from(p)
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")  # never touched
    rc = L.xf_step_noalloc(p.n_E, p.n_u, p.n_f, ctypes.byref(prm), ctypes.c_void_p(dev.data_ptr()),
                           p.r0, 1, p.h, ctypes.c_void_p(0))
    assert xf.STATUS[rc] == "XF_E_TOO_BIG"
