"""The extended bulb model (Eq. 3.18: azimuth bins, four moments) on the GPU
against the oracle, through the C ABI."""
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


THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1, mu0=1e4)
CASES = {
    "2f-exph": I.Problem(n_E=12, n_u=6, n_phi=6, stepper=I.EXPH, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0,
                         n_steps=100, seed=41),
    "2f-rk4-ragged": I.Problem(n_E=7, n_u=5, n_phi=9, stepper=I.RK4, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0,
                               n_steps=100, seed=42),
    "3f-exph-matter": I.Problem(n_E=9, n_u=5, n_phi=4, stepper=I.EXPH, eps=1e-2, r0=60.0, r1=60.6, n_steps=60,
                                matter=I.MATTER_POWER, ne_ref=1e31, seed=43, **THREE),
    "2f-exph-multicta": I.Problem(n_E=20, n_u=24, n_phi=16, stepper=I.EXPH, mu0=3e4, eps=1e-2, r0=50.0,
                                  r1=50.5, n_steps=50, seed=44),
}


def run(xf, p, rho0, n, tile=0):
    c = xf.Context(p)
    if tile:
        c.set_option(xf.OPT_TILE_PAIRS, tile)
    c.set_state(rho0, p.r0)
    c.step(n, p.h)
    out = c.get_state()[0]
    c.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_matches_oracle(xf, orc, name):
    p = CASES[name]
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    assert st == 0
    got = run(xf, p, rho0, p.n_steps, tile=128 if "multicta" in name else 0)
    assert np.abs(ref - rho0).max() > 1e-6
    assert rel_err(got, ref, p.n_f) < TOL


def test_moments_match_oracle(xf, orc):
    p = CASES["3f-exph-matter"]
    rho0 = orc.init_state(p)
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    M = c.moments_ex()
    c.close()
    ref = orc.moments_ex(p, rho0, p.r0)
    assert np.abs(M - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(ref[2:]).max() > 1e-6 * np.abs(ref[:2]).max()  # the azimuthal moments are not zero


def test_symmetric_azimuths_equal_the_bulb_kernel(xf, orc):
    """The four-moment kernel on a state equal in every azimuth bin gives the
    two-moment bulb kernel's result in every bin."""
    p = CASES["2f-exph"]
    ma = p.replace(n_phi=1)
    rho_ma = orc.init_state(ma)
    x = rho_ma.reshape(2, p.n_u, 1, p.n_E, 4)
    rho = np.ascontiguousarray(np.broadcast_to(x, (2, p.n_u, p.n_phi, p.n_E, 4))).reshape(-1)
    got = run(xf, p, rho, p.n_steps).reshape(2, p.n_u, p.n_phi, p.n_E, 4)
    want = run(xf, ma, rho_ma, p.n_steps).reshape(2, p.n_u, 1, p.n_E, 4)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_batch_mixes_azimuth_and_plain_problems(xf, orc):
    """A pack with an azimuth problem runs the four-moment kernel; its plain
    bulb problems (one azimuth bin) still match the oracle."""
    probs = [CASES["2f-exph"], CASES["2f-exph"].replace(n_phi=1, seed=45), CASES["3f-exph-matter"].replace(
        r0=50.0, r1=50.6)]
    probs = [q.replace(stepper=I.EXPH, r1=q.r0 + 0.6, n_steps=60) for q in probs]
    rho0s = [orc.init_state(q) for q in probs]
    b = xf.Batch(probs)
    for i, (q, r0) in enumerate(zip(probs, rho0s)):
        b.set_state_i(i, r0, q.r0)
    b.step_all(60, [q.h for q in probs])
    for i, (q, r0) in enumerate(zip(probs, rho0s)):
        ref, st, _ = orc.evolve(q, r0, q.r0, q.h, 60, n_threads=THREADS)
        assert rel_err(b.get_state_i(i)[0], ref, q.n_f) < TOL
    b.close()


def test_fp32_bins(xf, orc):
    p = CASES["2f-exph"].replace(precision=I.FP32_M64)
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    got = run(xf, p, rho0, p.n_steps)
    assert rel_err(got, ref, p.n_f) < 1e-4


def test_outputs_and_checkpoint(xf, orc):
    p = CASES["2f-rk4-ragged"]
    c = xf.Context(p)
    c.init_state(p.r0)
    c.step(30, p.h)
    ck = c.checkpoint_save()
    c.step(30, p.h)
    want = c.get_state()[0]
    rho = want.reshape(2, p.n_u * p.n_phi, p.n_E, 4)
    avg = c.angle_average().reshape(2, p.n_u * p.n_phi, 4)
    assert np.abs(avg - rho.mean(axis=2)).max() <= 1e-14 * np.abs(rho).max()
    c.close()
    d = xf.Context(p)
    d.checkpoint_load(ck)
    d.step(30, p.h)
    assert np.array_equal(d.get_state()[0], want)
    d.close()


def test_unsupported_combinations_are_refused(xf):
    p = CASES["2f-exph"]
    with pytest.raises(xf.XFError) as ei:
        xf.Context(p.replace(stepper=I.EXPH_ADAPTIVE))
    assert ei.value.name == "XF_E_UNSUPPORTED"
    with pytest.raises(xf.XFError) as ei:
        xf.Context(p.replace(precision=I.FP32_COMP))
    assert ei.value.name == "XF_E_UNSUPPORTED"
