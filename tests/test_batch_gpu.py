"""Batches: many problems in one persistent launch (C ABI xf_create_batch /
xf_batch_*).  Each problem's moments come from its own tiles only, so its
result must not depend on what it is packed with."""
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


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


def two_flavor_mix(precision=I.FP64, stepper=I.EXPH):
    return [
        I.Problem(n_E=32, n_u=16, mu0=1e5, hierarchy=-1, theta=(0.1, 0, 0), seed=31),
        I.Problem(n_E=57, n_u=9, mu0=3e4, hierarchy=+1, theta=(0.3, 0, 0), seed=32),
        I.Problem(n_E=8, n_u=200, mu0=1e3, hierarchy=-1, theta=(0.05, 0, 0), seed=33),
        I.Problem(n_E=1, n_u=1, mu0=50.0, geometry=I.CONST, seed=34),
    ], dict(precision=precision, stepper=stepper, r0=50.0, r1=50.5, n_steps=50, eps=1e-3)


def mixed(precision=I.FP64, stepper=I.EXPH):
    probs, common = two_flavor_mix(precision, stepper)
    probs.append(I.Problem(n_E=40, n_u=30, n_f=3, mu0=1e4, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72),
                           hierarchy=+1, seed=35))
    probs.append(I.Problem(n_E=17, n_u=11, n_f=3, mu0=1e5, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72),
                           hierarchy=-1, matter=I.MATTER_POWER, ne_ref=1e31, seed=36))
    return probs, common


def _run_batch(xf, probs, rho0s, p, steps, tile=256, graph=False, chunks=1):
    b = xf.Batch(probs)
    b.set_option(xf.OPT_TILE_PAIRS, tile)
    if graph:
        b.set_option(xf.OPT_GRAPH, 1)
    for i, r in enumerate(rho0s):
        b.set_state_i(i, r, p.r0)
    for _ in range(chunks):
        b.step_all(steps // chunks, p.h)
    out = [b.get_state_i(i)[0] for i in range(len(probs))]
    st = [b.status_i(i) for i in range(len(probs))]
    b.close()
    return out, st


def _run_alone(xf, prob, rho0, p, steps, tile=256):
    c = xf.Context(prob)
    c.set_option(xf.OPT_TILE_PAIRS, tile)
    c.set_state(rho0, p.r0)
    c.step(steps, p.h)
    out = c.get_state()[0]
    c.close()
    return out


@pytest.mark.parametrize("precision", [I.FP64, I.FP32_M64])
def test_same_flavor_batch_equals_alone_bitwise(xf, orc, precision):
    probs, common = two_flavor_mix(precision)
    probs = [q.replace(**common) for q in probs]
    p = probs[0]
    rho0s = [orc.init_state(q) for q in probs]
    got, st = _run_batch(xf, probs, rho0s, p, p.n_steps)
    assert all(s[0] == "XF_OK" and s[1] == p.n_steps for s in st)
    for q, r0, g in zip(probs, rho0s, got):
        alone = _run_alone(xf, q, r0, p, p.n_steps)
        assert np.array_equal(g, alone)


def test_mixed_batch_matches_oracle_and_alone(xf, orc):
    probs, common = mixed(I.FP64)
    probs = [q.replace(**common) for q in probs]
    p = probs[0]
    rho0s = [orc.init_state(q) for q in probs]
    got, st = _run_batch(xf, probs, rho0s, p, p.n_steps)
    for q, r0, g, s in zip(probs, rho0s, got, st):
        assert s[0] == "XF_OK" and s[1] == p.n_steps and s[2] == pytest.approx(p.r1, rel=1e-14)
        ref, ok, _ = orc.evolve(q, r0, p.r0, p.h, p.n_steps, n_threads=THREADS)
        assert ok == 0
        assert rel_err(g, ref, q.n_f) < 1e-9
        alone = _run_alone(xf, q, r0, p, p.n_steps)
        assert rel_err(g, alone, q.n_f) < 1e-12


def test_nonfinite_problem_stops_alone(xf, orc):
    """A problem whose explicit RK4 blows up (10 km, h = 0.095 km) stops at its
    last finite state; its neighbours in the launch run to the end unchanged."""
    probs, common = two_flavor_mix(I.FP64, I.RK4)
    common.update(r1=50.0 + 0.095 * 50)
    probs = [q.replace(**common) for q in probs]
    good_h = 0.01
    bad = probs[0].replace(r0=10.0, r1=10.0 + 0.095 * 50, mu0=1e5)
    probs[0] = bad
    rho0s = [orc.init_state(q) for q in probs]
    b = xf.Batch(probs)
    b.set_option(xf.OPT_TILE_PAIRS, 256)
    b.set_state_i(0, rho0s[0], 10.0)
    for i in range(1, len(probs)):
        b.set_state_i(i, rho0s[i], 50.0)
    b.step_all(50, [0.095] + [good_h] * (len(probs) - 1))
    st = [b.status_i(i) for i in range(len(probs))]
    assert st[0][0] == "XF_E_NONFINITE" and st[0][1] < 50
    assert np.isfinite(b.get_state_i(0)[0]).all()
    for i in range(1, len(probs)):
        assert st[i][0] == "XF_OK" and st[i][1] == 50
        alone = _run_alone(xf, probs[i], rho0s[i], probs[i].replace(r0=50.0, r1=50.5, n_steps=50), 50)
        assert np.array_equal(b.get_state_i(i)[0], alone)
    b.close()


def test_graph_replay_equals_plain_launches(xf, orc):
    probs, common = mixed(I.FP32_M64)
    probs = [q.replace(**common) for q in probs]
    p = probs[0]
    rho0s = [orc.init_state(q) for q in probs]
    plain, _ = _run_batch(xf, probs, rho0s, p, 60, chunks=1)
    graph, st = _run_batch(xf, probs, rho0s, p, 60, graph=True, chunks=3)
    assert all(s[1] == 60 for s in st)
    for a, g in zip(plain, graph):
        assert np.array_equal(a, g)


def test_full_c4_batch_sampled_against_oracle(xf, orc):
    """The 256-problem batched ensemble (about 40 M bins, FP32 bins with FP64
    moments), a few steps in the bench's launch configuration; a sample of
    problems is checked against the FP64 oracle on every bin."""
    import torch
    probs = I.ensemble_problems()
    b = xf.Batch(probs)
    b.init_state_i(-1, probs[0].r0)
    n = 3
    b.step_all(n, probs[0].h)
    picks = [0, 17, 101, 255]
    for i in picks:
        q = probs[i]
        rho0 = orc.init_state(q)
        ref, ok, _ = orc.evolve(q, rho0, q.r0, q.h, n, n_threads=THREADS)
        got, r, done = b.get_state_i(i)
        assert done == n and ok == 0
        # FP32 bins: the phase per step reaches ~40 rad at h = 0.2 km, and the
        # FP32 rounding of the rotation rate (6e-8 relative) shows at ~1e-6
        assert rel_err(got, ref, q.n_f) < 1e-5, i
    b.close()
    torch.cuda.synchronize()


def test_autotune_restores_state_and_keeps_the_chosen_tile(xf, orc):
    """The tile search steps the pack, then puts every state, radius and
    step count back; later steps run with the chosen tile, bitwise like a
    pack that was set to that tile by hand."""
    probs, common = two_flavor_mix(I.FP32_M64)
    probs = [q.replace(**common) for q in probs]
    h = probs[0].h
    rho0s = [orc.init_state(q) for q in probs]

    def fresh():
        b = xf.Batch(probs)
        for i, (q, r0) in enumerate(zip(probs, rho0s)):
            b.set_state_i(i, r0, q.r0)
        b.step_all(5, h)
        return b

    b = fresh()
    before = [b.get_state_i(i) for i in range(len(probs))]
    tile, ms = b.autotune(4, h, [64, 256, 1024])
    assert tile in (64, 256, 1024) and ms > 0
    assert b.get_option(xf.OPT_TILE_PAIRS) == tile and b.get_option(xf.OPT_DYNAMIC_TILES) in (0, 1)
    with pytest.raises(xf.XFError) as ei:
        b.get_option(99)
    assert ei.value.name == "XF_E_ARG"
    for i, (x, r, n) in enumerate(before):
        y, r2, n2 = b.get_state_i(i)
        assert np.array_equal(x, y) and r == r2 and n == n2
    b.step_all(5, h)
    got = [b.get_state_i(i)[0] for i in range(len(probs))]
    b.close()
    c = fresh()
    c.set_option(xf.OPT_TILE_PAIRS, tile)
    c.step_all(5, h)
    for i in range(len(probs)):
        assert np.array_equal(got[i], c.get_state_i(i)[0])
    c.close()


@pytest.mark.parametrize("precision", [I.FP32_M64, I.FP64])
def test_dynamic_tile_claiming_is_bitwise_the_static_split(xf, orc, precision):
    """Claiming a stage's tiles from a counter gives every problem bitwise the
    result of the static split of tiles over CTAs (a tile's arithmetic and
    the tile order of the moment sums do not depend on which CTA ran it)."""
    probs = [p.replace(n_steps=20, precision=precision) for p in I.ensemble_problems(n_instances=12)]
    outs = []
    for dyn in (0, 1):
        b = xf.Batch(probs)
        b.set_option(xf.OPT_TILE_PAIRS, 256)
        b.set_option(xf.OPT_GRID, 16)  # many more tiles than CTAs
        b.set_option(xf.OPT_DYNAMIC_TILES, dyn)
        assert b.get_option(xf.OPT_DYNAMIC_TILES) == dyn and b.get_option(xf.OPT_TILE_PAIRS) == 256
        b.init_state_i(-1, probs[0].r0)
        b.step_all(20, [q.h for q in probs])
        outs.append([b.get_state_i(i)[0] for i in range(len(probs))])
        b.close()
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
