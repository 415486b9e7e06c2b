"""The cylinder/line model (Sec. 3.2.5, Eq. 3.20: latitude x emission-angle
trajectories, the background read at the latitude Phi' it left from) on the
GPU against the oracle, through the C ABI."""
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
TOL = 1e-9


@pytest.fixture(scope="module")
def xf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05560_gb300 import build, xf as X
    build.build()
    X.load()
    return X


def rel_err(a, b, n_f):
    A = a.reshape(-1, n_f * n_f)
    B = b.reshape(-1, n_f * n_f)
    return float((np.abs(A - B).max(1) / np.abs(B[:, :n_f].sum(1))).max())


CYL = dict(geometry=I.CYLINDER)
THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1)
CASES = {
    "2f-exph": I.Problem(n_E=12, n_u=16, n_phi=8, stepper=I.EXPH, mu0=1e3, eps=1e-2, r0=20.0, r1=21.0,
                         n_steps=100, seed=71, **CYL),
    "2f-rk4-ragged": I.Problem(n_E=7, n_u=9, n_phi=5, stepper=I.RK4, mu0=3e2, eps=1e-2, r0=20.0, r1=21.0,
                               n_steps=100, seed=72, **CYL),
    "3f-exph-matter": I.Problem(n_E=9, n_u=11, n_phi=6, stepper=I.EXPH, mu0=1e3, eps=1e-2, r0=20.0, r1=20.5,
                                n_steps=50, matter=I.MATTER_POWER, ne_ref=1e30, seed=73, **THREE, **CYL),
    "3f-rk4": I.Problem(n_E=8, n_u=10, n_phi=3, stepper=I.RK4, mu0=1e2, eps=1e-2, r0=20.0, r1=20.5,
                        n_steps=50, seed=74, **THREE, **CYL),
    "2f-exph-one-latitude": I.Problem(n_E=16, n_u=33, n_phi=1, stepper=I.EXPH, mu0=1e3, eps=1e-2, r0=20.0,
                                      r1=21.0, n_steps=100, seed=75, **CYL),
    "2f-exph-many-ctas": I.Problem(n_E=40, n_u=64, n_phi=40, stepper=I.EXPH, mu0=1e3, eps=1e-2, r0=20.0,
                                   r1=20.5, n_steps=50, seed=76, **CYL),
}


def run(xf, p, rho0, n, grid=0):
    c = xf.Context(p)
    if grid:
        c.set_option(xf.OPT_GRID, grid)
    c.set_state(rho0, p.r0)
    c.step(n, p.h)
    out = c.get_state()
    c.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_matches_oracle(xf, orc, name):
    p = CASES[name]
    rho0 = orc.init_state(p)
    ref, st, done = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    assert st == 0 and done == p.n_steps
    got, r, n = run(xf, p, rho0, p.n_steps)
    assert n == p.n_steps and r == pytest.approx(p.r1, rel=1e-12)
    assert np.abs(ref - rho0).max() > 1e-5  # the flavors moved
    assert rel_err(got, ref, p.n_f) < TOL


def test_few_ctas_equal_many(xf, orc):
    """The result does not depend on how trajectories are split over CTAs."""
    p = CASES["2f-exph-many-ctas"]
    rho0 = orc.init_state(p)
    a = run(xf, p, rho0, 20)[0]
    b = run(xf, p, rho0, 20, grid=7)[0]
    assert np.array_equal(a, b)


def test_chunks_and_graph_replay_are_bitwise(xf, orc):
    p = CASES["3f-exph-matter"]
    rho0 = orc.init_state(p)
    want = run(xf, p, rho0, 40)[0]
    c = xf.Context(p)
    c.set_option(xf.OPT_GRAPH, 1)
    c.set_state(rho0, p.r0)
    for _ in range(4):
        c.step(10, p.h)
    got, r, n = c.get_state()
    c.close()
    assert n == 40 and np.array_equal(got, want)


def test_uniform_latitudes_equal_one_latitude(xf, orc):
    """A state the same at every latitude evolves like the model with one
    latitude bin (three moments) in every latitude."""
    p = CASES["2f-exph"]
    one = p.replace(n_phi=1)
    rho1 = orc.init_state(one)
    rho = np.ascontiguousarray(np.broadcast_to(rho1.reshape(2, p.n_u, 1, p.n_E, 4),
                                               (2, p.n_u, p.n_phi, p.n_E, 4))).reshape(-1)
    a = run(xf, p, rho, 50)[0].reshape(2, p.n_u, p.n_phi, p.n_E, 4)
    b = run(xf, one, rho1, 50)[0].reshape(2, p.n_u, 1, p.n_E, 4)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_fp32_bins(xf, orc):
    p = CASES["2f-exph"].replace(precision=I.FP32_M64)
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    got = run(xf, p, rho0, p.n_steps)[0]
    assert rel_err(got, ref, p.n_f) < 1e-4


def test_moments_outputs_and_checkpoint(xf, orc):
    p = CASES["3f-rk4"]
    c = xf.Context(p)
    c.init_state(p.r0)
    seeded = orc.init_state(p)
    assert np.abs(c.get_state()[0] - seeded).max() < 1e-14 * np.abs(seeded).max()  # the traceless pack round trip
    c.step(20, p.h)
    rho, r, _ = c.get_state()
    M = c.moments_ex()
    ref = orc.moments_ex(p, rho, r)
    assert np.abs(M - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(ref[2]).max() > 1e-6 * np.abs(ref[0]).max()  # the sin(alpha) moment
    ck = c.checkpoint_save()
    c.step(20, p.h)
    want = c.get_state()[0]
    c.close()
    d = xf.Context(p)
    d.checkpoint_load(ck)
    d.step(20, p.h)
    assert np.array_equal(d.get_state()[0], want)
    d.close()


def test_nonfinite_stop_like_oracle(xf, orc):
    """Explicit RK4 with mu0 1e4 at 12 km and h = 0.002 km diverges within a
    few steps; both sides stop and keep the last finite state."""
    p = I.Problem(n_E=8, n_u=10, n_phi=4, stepper=I.RK4, mu0=1e4, eps=1e-2, r0=12.0, r1=12.8, n_steps=400,
                  seed=61, **CYL)
    rho0 = orc.init_state(p)
    _, st, done_o = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    assert st == 1
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    with pytest.raises(xf.XFError) as ei:
        c.step(p.n_steps, p.h)
    assert ei.value.name == "XF_E_NONFINITE"
    got, r, done = c.get_state()
    c.close()
    assert np.isfinite(got).all()
    assert abs(done - done_o) <= 1


def test_unsupported_combinations_are_refused(xf):
    p = CASES["2f-exph"]
    for q in (p.replace(stepper=I.EXPH_ADAPTIVE), p.replace(precision=I.FP32_COMP),
              p.replace(precision=I.FP32_M64_RENORM), p.replace(form=I.FORM_PSI), p.replace(strict=1),
              p.replace(n_u=4096)):
        with pytest.raises(xf.XFError) as ei:
            xf.Context(q)
        assert ei.value.name == "XF_E_UNSUPPORTED"
    with pytest.raises(xf.XFError) as ei:
        xf.Batch([p, p.replace(seed=9)])
    assert ei.value.name == "XF_E_UNSUPPORTED"
    c = xf.Context(p)
    c.init_state(p.r0)
    c.step(2, p.h)
    with pytest.raises(xf.XFError) as ei:
        c.run_moments()
    assert ei.value.name == "XF_E_UNSUPPORTED"
    c.close()
