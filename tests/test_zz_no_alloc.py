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
in every precision, and the FP64 ones against the oracle too; that a run
longer than one launch (65536 steps) matches; that zero steps leave the
buffer as it was; that a non-finite input is refused before any step and a
run that blows up stops at its last finite state as xf_step does; and that a
problem too large for the fixed array is refused, each failure with its
message in xf_last_error(NULL).
"""
import ctypes

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-9  # same gate as the FP64 parity tests: |diff| / tr(rho) per bin
TOL32 = 1e-5  # FP32 bins against FP32 bins of the regular path (the batch tests' gate)


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


def _noalloc(torch, xf, L, p, dev, r0, n_steps):
    prm = xf.params_from(p)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.xf_step_noalloc(p.n_E, p.n_u, p.n_f, ctypes.byref(prm), ctypes.c_void_p(dev.data_ptr()),
                             r0, n_steps, p.h, stream)


def _message(L):
    m = L.xf_last_error(None)
    return m.decode() if m else ""


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
    assert _message(L) == ""


@pytest.mark.parametrize("p", CASES, ids=["2f-rk4", "3f-exph-multicta"])
def test_noalloc_matches_the_oracle(env, orc, p):
    """The FP64 result against the CPU oracle on the same seeded state."""
    torch, xf, L = env
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps)
    assert st == 0
    dev = torch.tensor(rho0, dtype=torch.float64, device="cuda")
    rc = _noalloc(torch, xf, L, p, dev, p.r0, p.n_steps)
    assert rc == 0, xf.status_str(rc)
    assert _rel(dev.cpu().numpy(), ref, p.n_f) < TOL


@pytest.mark.parametrize("precision", [I.FP32_M64, I.FP32_COMP, I.FP32_M64_RENORM],
                         ids=["fp32_m64", "fp32_comp", "fp32_m64_renorm"])
@pytest.mark.parametrize("base", CASES, ids=["2f-rk4", "3f-exph-multicta"])
def test_noalloc_fp32_precisions_match_regular_entry_points(env, base, precision):
    """FP32 bins (every precision variant) against xf_step in the same
    precision, on two calls in a row."""
    torch, xf, L = env
    p = base.replace(precision=precision)
    ctx = xf.Context(p)
    ctx.init_state(p.r0)
    rho0, _, _ = ctx.get_state()
    ctx.step(p.n_steps, p.h)
    ref1, r1, _ = ctx.get_state()
    ctx.step(p.n_steps, p.h)
    ref2, _, _ = ctx.get_state()
    ctx.close()
    dev = torch.tensor(rho0, dtype=torch.float64, device="cuda")
    assert _noalloc(torch, xf, L, p, dev, p.r0, p.n_steps) == 0, _message(L)
    out1 = dev.cpu().numpy().copy()
    assert _noalloc(torch, xf, L, p, dev, r1, p.n_steps) == 0, _message(L)
    out2 = dev.cpu().numpy().copy()
    assert np.abs(ref1 - rho0).max() > 1e-6
    assert _rel(out1, ref1, p.n_f) < TOL32
    assert _rel(out2, ref2, p.n_f) < TOL32


def test_noalloc_longer_than_one_launch(env):
    """More than 65536 steps: the call splits them over several launches
    that share one progress record; the result equals xf_step's."""
    torch, xf, L = env
    p = I.Problem(n_E=4, n_u=2, n_f=2, stepper=I.EXPH, mu0=1e3, r0=50.0, r1=50.0 + 70001 * 1e-4,
                  n_steps=70001, eps=1e-2, seed=23)
    ctx = xf.Context(p)
    ctx.init_state(p.r0)
    rho0, _, _ = ctx.get_state()
    ctx.step(p.n_steps, p.h)
    ref, _, n = ctx.get_state()
    ctx.close()
    assert n == p.n_steps
    dev = torch.tensor(rho0, dtype=torch.float64, device="cuda")
    assert _noalloc(torch, xf, L, p, dev, p.r0, p.n_steps) == 0, _message(L)
    out = dev.cpu().numpy()
    assert np.abs(ref - rho0).max() > 1e-4
    assert _rel(out, ref, p.n_f) < TOL


def test_noalloc_zero_steps_leaves_the_buffer(env):
    torch, xf, L = env
    p = CASES[1]
    rng = np.random.default_rng(5)
    x = rng.normal(size=2 * p.n_u * p.n_E * p.n_f * p.n_f)
    dev = torch.tensor(x, dtype=torch.float64, device="cuda")
    assert _noalloc(torch, xf, L, p, dev, p.r0, 0) == 0
    assert np.array_equal(dev.cpu().numpy(), x)


def test_noalloc_refuses_non_finite_input_before_stepping(env):
    torch, xf, L = env
    p = CASES[0]
    ctx = xf.Context(p)
    ctx.init_state(p.r0)
    rho0, _, _ = ctx.get_state()
    ctx.close()
    rho0 = rho0.copy()
    rho0[17] = np.nan
    dev = torch.tensor(rho0, dtype=torch.float64, device="cuda")
    rc = _noalloc(torch, xf, L, p, dev, p.r0, 10 ** 6)   # would take seconds if it ran
    assert xf.STATUS[rc] == "XF_E_STATE"
    assert "non-finite" in _message(L)
    got = dev.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(rho0)) and np.array_equal(got[~np.isnan(got)],
                                                                             rho0[~np.isnan(rho0)])


def test_noalloc_stops_at_the_last_finite_state_like_xf_step(env):
    """Explicit RK4 far outside its stability region (two-flavor bulb from
    10 km with h = 0.095 km) turns non-finite; both entry points report it
    and hand back a finite last state.  Past the blow-up the states are of
    order 1e280 and rounding differences have grown with them, so the two
    are compared by size, not entry by entry (as the parity tests do)."""
    torch, xf, L = env
    p = I.bulb2f_16x32().replace(stepper=I.RK4, n_steps=400)
    ctx = xf.Context(p)
    ctx.init_state(p.r0)
    rho0, _, _ = ctx.get_state()
    with pytest.raises(xf.XFError) as e:
        ctx.step(p.n_steps, p.h)
    assert e.value.name == "XF_E_NONFINITE"
    ref, _, n = ctx.get_state()
    ctx.close()
    assert 0 < n < p.n_steps
    dev = torch.tensor(rho0, dtype=torch.float64, device="cuda")
    rc = _noalloc(torch, xf, L, p, dev, p.r0, p.n_steps)
    assert xf.STATUS[rc] == "XF_E_NONFINITE"
    assert "non-finite" in _message(L)
    out = dev.cpu().numpy()
    assert np.isfinite(out).all()
    big_ref, big_out = np.abs(ref).max(), np.abs(out).max()
    assert big_ref > 1e100 and 0.1 < big_out / big_ref < 10.0


def test_noalloc_reports_why_an_argument_is_refused(env):
    torch, xf, L = env
    p = CASES[0]
    prm = xf.params_from(p)
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = L.xf_step_noalloc(p.n_E, p.n_u, 4, ctypes.byref(prm), ctypes.c_void_p(dev.data_ptr()),
                           p.r0, 1, p.h, ctypes.c_void_p(0))
    assert xf.STATUS[rc] == "XF_E_ARG"
    assert "n_flavor" in _message(L)


def test_noalloc_refuses_problem_larger_than_its_array(env):
    torch, xf, L = env
    p = I.bulb3f_1000x200()  # 400,000 3x3 bins: about 150 MB of FP64 working memory
    prm = xf.params_from(p)
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")  # never touched
    rc = L.xf_step_noalloc(p.n_E, p.n_u, p.n_f, ctypes.byref(prm), ctypes.c_void_p(dev.data_ptr()),
                           p.r0, 1, p.h, ctypes.c_void_p(0))
    assert xf.STATUS[rc] == "XF_E_TOO_BIG"
    assert "XF_NOALLOC_SCRATCH_BYTES" in _message(L)
