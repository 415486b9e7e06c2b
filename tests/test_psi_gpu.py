"""The wavefunction form (Eq. 3.9-3.11: one wavefunction per initial flavor,
rho = sum_a phi_a psi_a psi_a^+) on the GPU against the oracle, through the
C ABI: the seeded wavefunctions, fixed RK4 and predictor-corrector steps in
two and three flavors, the density matrices and moments computed from them,
checkpoints, and the combinations that are refused."""
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
TOL = 1e-9  # |psi| <= 1: absolute difference of the FP64 wavefunctions


@pytest.fixture(scope="module")
def xf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05560_gb300 import build, xf as X
    build.build()
    X.load()
    return X


THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1, mu0=1e4)
PSI = dict(form=I.FORM_PSI)
CASES = {
    "2f-exph": I.Problem(n_E=24, n_u=20, stepper=I.EXPH, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0, n_steps=100,
                         seed=51, **PSI),
    "2f-rk4-ragged": I.Problem(n_E=7, n_u=5, stepper=I.RK4, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0, n_steps=200,
                               seed=52, **PSI),
    "3f-exph-matter": I.Problem(n_E=20, n_u=17, stepper=I.EXPH, eps=1e-2, r0=60.0, r1=60.8, n_steps=80,
                                matter=I.MATTER_POWER, ne_ref=1e31, seed=53, **THREE, **PSI),
    "3f-rk4": I.Problem(n_E=13, n_u=9, stepper=I.RK4, eps=1e-2, r0=60.0, r1=60.4, n_steps=80, seed=54,
                        **THREE, **PSI),
    "2f-exph-multicta": I.Problem(n_E=40, n_u=48, stepper=I.EXPH, mu0=3e4, eps=1e-2, r0=50.0, r1=50.5,
                                  n_steps=50, seed=55, **PSI),
}


def run(xf, p, psi0, n, tile=0):
    c = xf.Context(p)
    if tile:
        c.set_option(xf.OPT_TILE_PAIRS, tile)
    c.set_psi(psi0, p.r0)
    c.step(n, p.h)
    out = c.get_psi()[0]
    c.close()
    return out


def test_seeded_wavefunctions_match_the_oracle(xf, orc):
    for name in ("2f-exph", "3f-rk4"):
        p = CASES[name]
        c = xf.Context(p)
        c.init_state(p.r0)
        got, r, n = c.get_psi()
        c.close()
        want = orc.init_psi(p)
        assert r == p.r0 and n == 0
        assert np.abs(got - want).max() < 1e-15


@pytest.mark.parametrize("name", list(CASES))
def test_matches_oracle(xf, orc, name):
    p = CASES[name]
    psi0 = orc.init_psi(p)
    ref, st, done = orc.evolve_psi(p, psi0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    assert st == 0 and done == p.n_steps
    got = run(xf, p, psi0, p.n_steps, tile=128 if "multicta" in name else 0)
    assert np.abs(ref - psi0).max() > 1e-6  # the flavors moved
    assert np.abs(got - ref).max() < TOL


def test_density_matrices_and_moments_from_the_wavefunctions(xf, orc):
    p = CASES["3f-exph-matter"]
    psi0 = orc.init_psi(p)
    c = xf.Context(p)
    c.set_psi(psi0, p.r0)
    c.step(30, p.h)
    psi, r, n = c.get_psi()
    rho = c.get_state()[0]
    want = orc.psi_to_rho(p, psi)
    assert np.abs(rho - want).max() < 1e-14 * np.abs(want).max()
    M = c.moments_ex()
    ref = orc.moments_ex(p, want, r)
    assert np.abs(M - ref).max() < 1e-12 * np.abs(ref).max()
    outs = c.outputs()
    nf2 = p.n_f * p.n_f
    R = want.reshape(-1, nf2)
    assert np.abs(outs[1] - R[:, :p.n_f].sum(1)).max() < 1e-14 * np.abs(outs[1]).max()
    d = xf.Context(p.replace(form=I.FORM_RHO))  # the same outputs of the same density matrices
    d.set_state(want, r)
    for x, y in zip(outs, d.outputs()):
        assert np.abs(x - y).max() < 1e-12
    d.close()
    avg = c.angle_average().reshape(2, p.n_u, nf2)
    assert np.abs(avg - want.reshape(2, p.n_u, p.n_E, nf2).mean(axis=2)).max() <= 1e-14 * np.abs(want).max()
    c.close()


def test_norms_are_kept_without_self_interaction(xf):
    """Without the nu-nu term the Hamiltonian does not depend on the state, the
    predictor and the corrector propagate by the same unitary matrix, and
    every |psi_a| stays one to rounding."""
    p = CASES["3f-rk4"].replace(stepper=I.EXPH, mu0=0.0)  # vacuum: the same Hamiltonian at every radius
    c = xf.Context(p)
    c.init_state(p.r0)
    c.step(p.n_steps, p.h)
    psi = c.get_psi()[0].reshape(-1, p.n_f, p.n_f, 2)
    c.close()
    assert np.abs((psi ** 2).sum(axis=(2, 3)) - 1.0).max() < 1e-12


def test_batch_mixes_two_and_three_flavors(xf, orc):
    probs = [CASES["2f-exph"], CASES["3f-exph-matter"].replace(r0=50.0, r1=50.8), CASES["2f-exph"].replace(seed=56)]
    psi0s = [orc.init_psi(q) for q in probs]
    b = xf.Batch(probs)
    for i, (q, x) in enumerate(zip(probs, psi0s)):
        b.set_psi(x, q.r0, i)
    b.step_all(40, [q.h for q in probs])
    for i, (q, x) in enumerate(zip(probs, psi0s)):
        ref, st, _ = orc.evolve_psi(q, x, q.r0, q.h, 40, n_threads=THREADS)
        assert st == 0
        assert np.abs(b.get_psi(i)[0] - ref).max() < TOL
    b.close()


def test_fp32_bins(xf, orc):
    p = CASES["2f-exph"].replace(precision=I.FP32_M64)
    psi0 = orc.init_psi(p)
    ref, st, _ = orc.evolve_psi(p, psi0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    got = run(xf, p, psi0, p.n_steps)
    assert np.abs(got - ref).max() < 1e-4


def test_resume_from_checkpoint_is_bitwise(xf):
    p = CASES["3f-rk4"]
    a = xf.Context(p)
    a.init_state(p.r0)
    a.step(p.n_steps, p.h)
    want = a.get_psi()[0]
    a.close()
    b = xf.Context(p)
    b.init_state(p.r0)
    b.step(33, p.h)
    ck = b.checkpoint_save()
    b.close()
    c = xf.Context(p)
    c.checkpoint_load(ck)
    c.step(p.n_steps - 33, p.h)
    assert np.array_equal(c.get_psi()[0], want)
    rho_form = xf.Context(p.replace(form=I.FORM_RHO))
    with pytest.raises(xf.XFError) as ei:
        rho_form.checkpoint_load(ck)
    assert ei.value.name == "XF_E_ARG"
    rho_form.close()
    c.close()


def test_the_two_forms_approach_the_same_flow(xf, orc):
    """Both forms integrate the same equation of motion: with the step halved
    their difference shrinks more than threefold."""
    base = CASES["2f-exph"].replace(n_steps=50)
    diffs = []
    for n in (50, 100):
        p = base.replace(n_steps=n)
        c = xf.Context(p)
        c.init_state(p.r0)
        rho0 = c.get_state()[0]
        c.step(n, p.h)
        rho_psi = c.get_state()[0]
        c.close()
        d = xf.Context(p.replace(form=I.FORM_RHO))
        d.set_state(rho0, p.r0)
        d.step(n, p.h)
        rho_rho = d.get_state()[0]
        d.close()
        diffs.append(np.abs(rho_psi - rho_rho).max())
    assert diffs[1] < diffs[0] / 3.0


def test_unsupported_combinations_are_refused(xf, orc):
    p = CASES["2f-exph"]
    for q in (p.replace(stepper=I.EXPH_ADAPTIVE), p.replace(precision=I.FP32_COMP),
              p.replace(precision=I.FP32_M64_RENORM), p.replace(n_phi=4)):
        with pytest.raises(xf.XFError) as ei:
            xf.Context(q)
        assert ei.value.name == "XF_E_UNSUPPORTED"
    c = xf.Context(p)
    with pytest.raises(xf.XFError) as ei:
        c.set_state(np.zeros(p.n_bins * p.n_f ** 2), p.r0)
    assert ei.value.name == "XF_E_UNSUPPORTED"
    bad = orc.init_psi(p)
    bad[5] = np.nan
    with pytest.raises(xf.XFError) as ei:
        c.set_psi(bad, p.r0)
    assert ei.value.name == "XF_E_STATE"
    c.close()
    r = xf.Context(p.replace(form=I.FORM_RHO))
    with pytest.raises(xf.XFError) as ei:
        r.set_psi(orc.init_psi(p), p.r0)
    assert ei.value.name == "XF_E_UNSUPPORTED"
    r.close()
    with pytest.raises(xf.XFError):
        xf.Batch([p, p.replace(form=I.FORM_RHO)])
