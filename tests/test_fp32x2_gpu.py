"""XF_FP32X2: FP64 state, tables and sums, the predictor-corrector's propagator
(Eq. 3.10-3.12) in float-float arithmetic on the FP32 pipes.

Against the FP64 oracle of the same method:
* small 2- and 3-flavor problems with ragged tails over several CTAs, matter
  and the literal (R/r)^4 coupling, element by element at the FP64 gate
  (|d rho| / tr rho <= 1e-9);
* the 400,000-bin three-flavor workload over 200 steps on every bin, in the
  bench's launch shape;
* the ensemble problems on which FP32 bins miss the 1e-3 survival-probability
  target (large mu0, two and three flavors), whole 1000-step runs in one
  batch, gated at 1e-3 like the FP32 target (and printed);
and the pack rules: a batch and a server equal each problem alone bitwise, and the
steppers the precision does not run are refused.
"""
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL64 = 1e-9
THREADS = os.cpu_count() or 1
THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1)


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
    tr = np.abs(B[:, :n_f].sum(1))
    return float((np.abs(A - B).max(1) / tr).max())


def p_surv_error(got, ref, rho0, n_f):
    """max |P_surv(got) - P_surv(ref)| over bins whose spectra are
    distinguishable (|phi_e - phi_x| >= 1e-2 of the species' largest)."""
    m = n_f * n_f
    g, r, x0 = got.reshape(2, -1, m), ref.reshape(2, -1, m), rho0.reshape(2, -1, m)
    worst = 0.0
    for s in range(2):
        sep = x0[s, :, 0] - x0[s, :, 1]
        mask = np.abs(sep) >= 1e-2 * np.abs(sep).max()
        worst = max(worst, float(np.abs((g[s, mask, 0] - r[s, mask, 0]) / sep[mask]).max()))
    return worst


def small(**kw):
    base = dict(n_E=37, n_u=23, n_f=2, stepper=I.EXPH, precision=I.FP32X2, mu0=1e5, r0=50.0, r1=52.0,
                n_steps=200, eps=1e-2, seed=21)
    base.update(kw)
    return I.Problem(**base)


CASES = {
    "2f-bulb": small(),
    "3f-bulb": small(**THREE),
    "3f-matter": small(**THREE, matter=I.MATTER_POWER, ne_ref=1e33, r0=20.0, r1=21.0, seed=22),
    "3f-mu-r4-inverted": small(**dict(THREE, hierarchy=-1), geometry=I.MU_R4, seed=23),
    "2f-matter-exp": small(matter=I.MATTER_EXP, nb0=1e34, h_ns=2.0, r0=30.0, r1=31.0, seed=24),
}


@pytest.mark.parametrize("name", list(CASES))
def test_matches_oracle(xf, orc, name):
    p = CASES[name]
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    assert st == 0
    c = xf.Context(p)
    c.set_option(xf.OPT_TILE_PAIRS, 128)  # several tiles and CTAs, ragged last tile
    c.set_state(rho0, p.r0)
    c.step(p.n_steps, p.h)
    got, r, done = c.get_state()
    c.close()
    assert done == p.n_steps and r == pytest.approx(p.r1, rel=1e-13)
    assert np.abs(ref - rho0).max() > 1e-6 * np.abs(rho0).max()
    err = rel_err(got, ref, p.n_f)
    print(f"{name}: FP32X2 max |d rho| / tr rho after {p.n_steps} steps = {err:.3e}")
    assert err < TOL64


def test_three_flavor_full_size(xf, orc):
    """The 400,000-bin three-flavor workload (matter r^-3), 200 steps from
    10 km in 100-step launches, every bin against the oracle."""
    p = I.bulb3f_1000x200().replace(precision=I.FP32X2)
    rho0 = orc.init_state(p)
    n, chunk = 200, 100
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, n, n_threads=THREADS)
    assert st == 0
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    for _ in range(n // chunk):
        c.step_async(chunk, p.h)
    c.sync()
    got, r, done = c.get_state()
    c.close()
    assert done == n
    err = rel_err(got, ref, 3)
    print(f"FP32X2 400,000 bins: max |d rho| / tr rho after {n} steps = {err:.3e}")
    assert err < TOL64


# ensemble problems where FP32 bins miss the target (mu0 > 1e5): FP32 errors
# 2.2e-2 (70), 1.2e-2 (57), 1.0e-3 (100), 5.3e-3 (172), 4.4e-2 (235)
UNSTABLE = [70, 57, 100, 172, 235]


def test_unstable_ensemble_problems_meet_target(xf, orc):
    probs = I.ensemble_problems()
    ps = [probs[i].replace(precision=I.FP32X2) for i in UNSTABLE]
    b = xf.Batch(ps)
    b.set_option(xf.OPT_GRAPH, 1)
    b.init_state_i(-1, ps[0].r0)
    n = ps[0].n_steps
    for _ in range(n // 10):
        b.step_all(10, ps[0].h)
    worst = 0.0
    for k, (i, q) in enumerate(zip(UNSTABLE, ps)):
        st = b.status_i(k)
        assert st[0] == "XF_OK" and st[1] == n
        got = b.get_state_i(k)[0]
        rho0 = orc.init_state(q)
        ref, ok, _ = orc.evolve(q, rho0, q.r0, q.h, n, n_threads=THREADS)
        assert ok == 0
        e = p_surv_error(got, ref, rho0, q.n_f)
        print(f"ensemble problem {i} ({q.n_f} flavors, mu0 {q.mu0:.3g}): FP32X2 max |dP_surv| = {e:.3e}, "
              f"max |d rho| / tr rho = {rel_err(got, ref, q.n_f):.3e}")
        worst = max(worst, e)
    b.close()
    assert worst < 1e-3


def test_batch_equals_alone_bitwise(xf, orc):
    base = dict(stepper=I.EXPH, precision=I.FP32X2, r0=50.0, r1=50.5, n_steps=50, eps=1e-3)
    probs = [I.Problem(n_E=20, n_u=9, seed=41, **base),
             I.Problem(n_E=33, n_u=5, mu0=3e4, seed=42, **base),
             I.Problem(n_E=17, n_u=11, seed=43, **THREE, **base),
             I.Problem(n_E=8, n_u=30, mu0=1e3, matter=I.MATTER_POWER, ne_ref=1e31, seed=44,
                       **dict(THREE, hierarchy=-1), **base)]
    rho0s = [orc.init_state(q) for q in probs]
    b = xf.Batch(probs)
    b.set_option(xf.OPT_TILE_PAIRS, 64)
    for i, r in enumerate(rho0s):
        b.set_state_i(i, r, 50.0)
    b.step_all(50, 0.01)
    for i, (q, r) in enumerate(zip(probs, rho0s)):
        assert b.status_i(i)[0] == "XF_OK"
        c = xf.Context(q)
        c.set_option(xf.OPT_TILE_PAIRS, 64)
        c.set_state(r, 50.0)
        c.step(50, 0.01)
        assert np.array_equal(b.get_state_i(i)[0], c.get_state()[0])
        c.close()
    b.close()


@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH_ADAPTIVE])
def test_other_steppers_are_refused(xf, stepper):
    p = small(stepper=stepper, n_E=4, n_u=3)
    with pytest.raises(xf.XFError) as e:
        xf.Context(p)
    assert "XF_E_UNSUPPORTED" in str(e.value)


def test_served_jobs_equal_alone(xf, orc):
    """A server in FP32X2: jobs queued behind each other share launches and
    each result is bitwise that of the job alone (same tile size)."""
    g = I.SplitMix64(77)
    ps = []
    for k in range(4):
        steps = g.randint(30, 90)
        ps.append(I.Problem(n_E=g.randint(8, 40), n_u=g.randint(8, 60), n_f=2, mu0=10 ** (4 + 2 * g.uniform()),
                            hierarchy=1 if k % 2 else -1, theta=(0.1 + 0.4 * g.uniform(), 0, 0), stepper=I.EXPH,
                            precision=I.FP32X2, r0=50.0, r1=50.0 + 0.01 * steps, n_steps=steps, eps=1e-3,
                            seed=700 + k))
    rho0s = [orc.init_state(p) for p in ps]
    tile = 512
    srv = xf.Server(max_jobs=2, mem_budget_bytes=1 << 30, chunk_steps=20, stepper=I.EXPH,
                    precision=I.FP32X2, tile_pairs=tile)
    ids = [srv.submit(p, rho0=r, keep_state=True) for p, r in zip(ps, rho0s)]
    srv.drain(timeout_s=120.0)
    for j, p, r in zip(ids, ps, rho0s):
        meta, got = srv.poll(j, want_state=True)
        assert meta["status"] == "XF_OK" and meta["steps"] == p.n_steps
        c = xf.Context(p)
        c.set_option(xf.OPT_TILE_PAIRS, tile)
        c.set_state(r, p.r0)
        c.step(p.n_steps, p.h)
        assert np.array_equal(got, c.get_state()[0])
        c.close()
    assert srv.stats()["max_resident"] == 2
    srv.close()


def test_chunked_launches_equal_one_launch(xf, orc):
    """The moments a launch's prologue forms from the stored state equal those
    the previous launch formed from its last stage's output, bit for bit, so
    a run split into launches is the run in one launch."""
    for kw in ({}, THREE):
        p = small(n_E=23, n_u=31, n_steps=60, r1=50.6, seed=31, **kw)
        rho0 = orc.init_state(p)
        out = []
        for chunks in ([60], [20, 20, 20], [7, 53]):
            c = xf.Context(p)
            c.set_option(xf.OPT_TILE_PAIRS, 512)
            c.set_state(rho0, p.r0)
            for n in chunks:
                c.step(n, p.h)
            out.append(c.get_state()[0])
            c.close()
        assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
