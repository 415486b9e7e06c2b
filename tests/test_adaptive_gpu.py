"""The error-controlled step (stepper XF_EXPH_ADAPTIVE: Sec. 4.2.3, Fig. 4.9,
S1-S5) on the GPU against the oracle's orc_evolve_adaptive.  Both sides take
every accept / reject decision in FP64 from the same error estimate, so the
step sequences must agree exactly (accepted and rejected counts, final radius,
next step size) and the states within the parity tolerance."""
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


THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1)
CASES = {
    "2f-bulb": I.Problem(n_E=24, n_u=12, mu0=1e5, eps=1e-3, seed=11, r0=50.0, eps0=1e-6, dr_max=0.2),
    "2f-bulb-multicta": I.Problem(n_E=57, n_u=40, mu0=3e4, eps=1e-3, seed=12, r0=50.0, eps0=3e-7, dr_max=0.5),
    "3f-matter": I.Problem(n_E=20, n_u=9, mu0=1e4, eps=1e-3, seed=13, r0=60.0, matter=I.MATTER_POWER,
                           ne_ref=1e31, eps0=1e-6, dr_max=0.5, **THREE),
    "2f-single-angle": I.Problem(n_E=15, n_u=1, geometry=I.SINGLE_ANGLE, mu0=1e5, eps=1e-2, seed=14, r0=40.0,
                                 eps0=1e-7, dr_max=0.5),
    "2f-mu-r4": I.Problem(n_E=16, n_u=8, geometry=I.MU_R4, mu0=1e5, eps=1e-3, seed=15, r0=50.0, eps0=1e-6,
                          dr_max=0.3),
}
SPAN = {"2f-bulb": 3.0, "2f-bulb-multicta": 4.0, "3f-matter": 2.0, "2f-single-angle": 2.0, "2f-mu-r4": 3.0}


def run_gpu(xf, p, rho0, r_end, h0, max_iters=1 << 40, tile=0):
    c = xf.Context(p.replace(stepper=I.EXPH_ADAPTIVE))
    if tile:
        c.set_option(xf.OPT_TILE_PAIRS, tile)
    c.set_state(rho0, p.r0)
    try:
        c.evolve(r_end, max_iters, h0)
        code = "XF_OK"
    except xf.XFError as e:
        code = e.name
    st = c.adapt_status()
    got, r, _ = c.get_state()
    c.close()
    return got, st, code


@pytest.mark.parametrize("name", list(CASES))
def test_matches_oracle_step_for_step(xf, orc, name):
    p = CASES[name]
    r_end = p.r0 + SPAN[name]
    rho0 = orc.init_state(p)
    ref, st, r, h, na, nr = orc.evolve_adaptive(p, rho0, p.r0, r_end, 0.3, n_threads=THREADS)
    assert st == 0 and na > 5
    got, gs, code = run_gpu(xf, p, rho0, r_end, 0.3, tile=128 if "multicta" in name else 0)
    assert code == "XF_OK" and gs["status"] == "XF_OK"
    assert (gs["n_accepted"], gs["n_rejected"]) == (na, nr)
    assert gs["r"] == r_end and gs["h_next"] == pytest.approx(h, rel=1e-9)
    assert rel_err(got, ref, p.n_f) < TOL


def test_two_calls_and_budget_match_oracle(xf, orc):
    """A run cut by the attempt budget continues where it stopped: the GPU's
    sequence of calls equals the oracle's same sequence."""
    p = CASES["2f-bulb"]
    rho0 = orc.init_state(p)
    o1, st1, r1, h1, na1, nr1 = orc.evolve_adaptive(p, rho0, p.r0, p.r0 + 3.0, 0.3, max_iters=7)
    assert st1 == 2 and na1 + nr1 == 7
    o2, st2, r2, h2, na2, nr2 = orc.evolve_adaptive(p, o1, r1, p.r0 + 3.0, h1)
    assert st2 == 0
    c = xf.Context(p.replace(stepper=I.EXPH_ADAPTIVE))
    c.set_state(rho0, p.r0)
    with pytest.raises(xf.XFError) as ei:
        c.evolve(p.r0 + 3.0, 7, 0.3)
    assert ei.value.name == "XF_E_BUDGET"
    s1 = c.adapt_status()
    assert (s1["n_accepted"], s1["n_rejected"], s1["r"]) == (na1, nr1, pytest.approx(r1, rel=1e-13))
    assert rel_err(c.get_state()[0], o1, 2) < TOL
    c.evolve(p.r0 + 3.0, 1 << 40, 0.0)  # keeps the step the budget stop left
    s2 = c.adapt_status()
    assert (s2["n_accepted"], s2["n_rejected"]) == (na2, nr2) and s2["r"] == p.r0 + 3.0
    assert rel_err(c.get_state()[0], o2, 2) < TOL
    c.close()


def test_vacuum_takes_dr_max_steps(xf, orc):
    p = I.Problem(n_E=12, n_u=5, eps=0.0, mu0=0.0, theta=(0.3, 0, 0), E_min=1.0, E_max=13.0, r0=20.0,
                  eps0=1e-10, dr_max=0.25, seed=16)
    rho0 = orc.init_state(p)
    ref, st, r, h, na, nr = orc.evolve_adaptive(p, rho0, 20.0, 30.0, 0.01)
    got, gs, code = run_gpu(xf, p, rho0, 30.0, 0.01)
    assert code == "XF_OK" and gs["n_rejected"] == 0 and (gs["n_accepted"], gs["n_rejected"]) == (na, nr)
    assert rel_err(got, ref, 2) < TOL


def test_step_size_underflow(xf, orc):
    p = CASES["2f-bulb"].replace(eps0=1e-300)
    rho0 = orc.init_state(p)
    ref, st, r, h, na, nr = orc.evolve_adaptive(p, rho0, p.r0, p.r0 + 1.0, 0.1)
    assert st == 3 and na == 0
    got, gs, code = run_gpu(xf, p, rho0, p.r0 + 1.0, 0.1)
    assert code == "XF_E_STEPSIZE" and gs["n_rejected"] == nr and gs["r"] == p.r0
    assert np.abs(got - rho0).max() <= 1e-15 * np.abs(rho0).max()  # state untouched


def _batch(xf, probs, rho0s, r_end, tile=64):
    b = xf.Batch([p.replace(stepper=I.EXPH_ADAPTIVE) for p in probs])
    b.set_option(xf.OPT_TILE_PAIRS, tile)
    for i, (p, r0) in enumerate(zip(probs, rho0s)):
        b.set_state_i(i, r0, p.r0)
    b.evolve_all(r_end, 1 << 40, 0.3)
    out = [(b.get_state_i(i)[0], b.adapt_status(i)) for i in range(len(probs))]
    b.close()
    return out


def test_batch_each_problem_follows_its_own_steps(xf, orc):
    """Problems of different sizes, flavors, tolerances and end radii in one
    launch: each takes its own step sequence, equal to the oracle's, and its
    state equals the same problem run alone (a mixed 2/3-flavor pack runs
    128-thread CTAs, so the 2-flavor problems' sums round differently from
    their 256-thread runs alone: equal to 1e-12, not bitwise)."""
    probs = [CASES["2f-bulb"], CASES["3f-matter"], CASES["2f-mu-r4"],
             CASES["2f-bulb"].replace(seed=21, eps0=1e-5, n_E=7, n_u=30)]
    r_end = [p.r0 + s for p, s in zip(probs, (3.0, 2.0, 2.5, 1.5))]
    rho0s = [orc.init_state(p) for p in probs]
    for p, r0, re, (got, s) in zip(probs, rho0s, r_end, _batch(xf, probs, rho0s, r_end)):
        ref, st, r, h, na, nr = orc.evolve_adaptive(p, r0, p.r0, re, 0.3, n_threads=THREADS)
        assert s["status"] == "XF_OK" and (s["n_accepted"], s["n_rejected"]) == (na, nr) and s["r"] == re
        assert rel_err(got, ref, p.n_f) < TOL
        alone, _, _ = run_gpu(xf, p, r0, re, 0.3, tile=64)
        assert rel_err(got, alone, p.n_f) < 1e-12


def test_same_flavor_batch_is_bitwise_alone(xf, orc):
    probs = [CASES["2f-bulb"], CASES["2f-mu-r4"], CASES["2f-bulb"].replace(seed=21, eps0=1e-5, n_E=7, n_u=30)]
    r_end = [p.r0 + s for p, s in zip(probs, (3.0, 2.5, 1.5))]
    rho0s = [orc.init_state(p) for p in probs]
    for p, r0, re, (got, s) in zip(probs, rho0s, r_end, _batch(xf, probs, rho0s, r_end)):
        alone, sa, _ = run_gpu(xf, p, r0, re, 0.3, tile=64)
        assert (s["n_accepted"], s["n_rejected"]) == (sa["n_accepted"], sa["n_rejected"])
        assert np.array_equal(got, alone)


def test_fp32_bins_reach_the_end_close_to_the_fp64_run(xf, orc):
    """FP32 bins: the error estimate is computed in FP32, so the step
    sequence may differ slightly; the run still ends on r_end, within the
    tolerance's reach of the FP64 oracle."""
    p = CASES["2f-bulb"].replace(eps0=1e-5)
    rho0 = orc.init_state(p)
    ref, st, r, h, na, nr = orc.evolve_adaptive(p, rho0, p.r0, p.r0 + 3.0, 0.3)
    got, gs, code = run_gpu(xf, p.replace(precision=I.FP32_M64), rho0, p.r0 + 3.0, 0.3)
    assert code == "XF_OK" and gs["r"] == p.r0 + 3.0
    assert abs(gs["n_accepted"] - na) <= 2
    assert rel_err(got, ref, 2) < 1e-3


def test_fixed_step_calls_refused_and_run_moments(xf, orc):
    p = CASES["2f-bulb"]
    c = xf.Context(p.replace(stepper=I.EXPH_ADAPTIVE))
    c.init_state(p.r0)
    with pytest.raises(xf.XFError) as ei:
        c.step(1, 0.01)
    assert ei.value.name == "XF_E_ARG"
    c.evolve(p.r0 + 0.5, 1 << 40, 0.1)
    R0, R1 = c.run_moments()
    F0, F1 = c.moments()
    tr = F0[:2].mean()
    F0 = F0.copy()
    F0[:2] -= tr
    assert np.abs(R0 - F0).max() <= 1e-12 * np.abs(F0).max()
    c.close()
