"""Serving: the continuous-batching job server (xf_server_*).  Jobs that
arrive while others run are admitted as slots and memory free up, share the
GPU with them, and give the same result as when run alone."""
import time

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TILE = 1024


@pytest.fixture(scope="module")
def xf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05560_gb300 import build, xf as X
    build.build()
    X.load()
    return X


def jobs(precision=I.FP32_M64, stepper=I.EXPH, n=6, seed=50):
    g = I.SplitMix64(seed)
    out = []
    for k in range(n):
        n_u = g.randint(8, 120)
        n_E = g.randint(8, 64)
        steps = g.randint(30, 160)
        out.append(I.Problem(n_E=n_E, n_u=n_u, n_f=2, mu0=10 ** (3 + 2 * g.uniform()),
                             hierarchy=1 if g.uniform() < 0.5 else -1, theta=(0.01 + 0.5 * g.uniform(), 0, 0),
                             stepper=stepper, precision=precision, r0=50.0, r1=50.0 + 0.01 * steps,
                             n_steps=steps, eps=1e-3, seed=seed + k))
    return out


def alone(xf, p, rho0):
    c = xf.Context(p)
    c.set_option(xf.OPT_TILE_PAIRS, TILE)
    c.set_state(rho0, p.r0)
    c.step(p.n_steps, p.h)
    out = c.get_state()[0]
    c.close()
    return out


def collect(srv, ids, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(ids) and time.time() - t0 < timeout:
        for j in ids:
            if j not in res:
                r = srv.poll(j, want_state=True)
                if r is not None:
                    res[j] = r
        time.sleep(0.002)
    assert len(res) == len(ids), "jobs did not finish"
    return res


def test_results_equal_alone_with_queueing(xf, orc):
    ps = jobs()
    rho0s = [orc.init_state(p) for p in ps]
    srv = xf.Server(max_jobs=3, mem_budget_bytes=1 << 30, chunk_steps=25, tile_pairs=TILE)
    ids = [srv.submit(p, rho0=r, keep_state=True) for p, r in zip(ps, rho0s)]
    res = collect(srv, ids)
    st = srv.stats()
    assert st["completed"] == len(ps) and st["max_resident"] <= 3
    for p, r0, j in zip(ps, rho0s, ids):
        meta, state = res[j]
        assert meta["status"] == "XF_OK" and meta["steps"] == p.n_steps
        assert meta["r"] == pytest.approx(p.r1, rel=1e-12)
        assert meta["t_submit"] <= meta["t_start"] <= meta["t_done"]
        assert np.array_equal(state, alone(xf, p, r0))
    srv.close()


def test_jobs_arriving_during_a_run_overlap_and_match_alone(xf, orc):
    first = jobs(n=2, seed=70)
    first = [p.replace(n_steps=400, r1=50.0 + 0.01 * 400) for p in first]
    later = jobs(n=4, seed=80)
    rho = {id(p): orc.init_state(p) for p in first + later}
    srv = xf.Server(max_jobs=8, mem_budget_bytes=1 << 30, chunk_steps=20, tile_pairs=TILE)
    ids1 = [srv.submit(p, rho0=rho[id(p)], keep_state=True) for p in first]
    # wait until the first jobs are on the GPU, then submit more
    t0 = time.time()
    while srv.stats()["resident"] < 2 and time.time() - t0 < 30:
        time.sleep(0.001)
    ids2 = [srv.submit(p, rho0=rho[id(p)], keep_state=True) for p in later]
    res = collect(srv, ids1 + ids2)
    st = srv.stats()
    assert st["max_resident"] >= 3  # later jobs ran next to the first ones
    t_done_first = min(res[j][0]["t_done"] for j in ids1)
    assert any(res[j][0]["t_start"] < t_done_first for j in ids2)
    for p, j in zip(first + later, ids1 + ids2):
        meta, state = res[j]
        assert meta["status"] == "XF_OK" and meta["steps"] == p.n_steps
        assert np.array_equal(state, alone(xf, p, rho[id(p)]))
    srv.close()


def test_admission_errors_and_poll_states(xf):
    p = jobs(n=1, seed=90)[0].replace(n_steps=3000, r1=50.0 + 0.01 * 3000)
    srv = xf.Server(max_jobs=1, mem_budget_bytes=64 << 20, chunk_steps=10, queue_cap=1, tile_pairs=TILE)
    big = p.replace(n_u=4096, n_E=4096)
    with pytest.raises(xf.XFError) as ei:
        srv.submit(big)
    assert ei.value.name == "XF_E_TOO_BIG"
    a = srv.submit(p)
    t0 = time.time()
    while srv.stats()["resident"] < 1 and time.time() - t0 < 30:
        time.sleep(0.001)
    b = srv.submit(p)  # queued behind the resident job
    with pytest.raises(xf.XFError) as ei:
        srv.submit(p)  # queue full
    assert ei.value.name == "XF_E_BUSY"
    assert srv.poll(b) is None  # pending
    with pytest.raises(xf.XFError) as ei:
        srv.poll(987654321)
    assert ei.value.name == "XF_E_NOTFOUND"
    srv.drain(120.0)
    assert srv.poll(a)[0]["status"] == "XF_OK" and srv.poll(b)[0]["status"] == "XF_OK"
    srv.close()


def test_memory_budget_bounds_residency(xf, orc):
    ps = [p.replace(n_u=100, n_E=64) for p in jobs(n=5, seed=110)]
    srv0 = xf.Server(max_jobs=8, mem_budget_bytes=1 << 30, chunk_steps=10, tile_pairs=TILE)
    srv0.close()
    # block of one job: 3 state buffers of 2 x 3 x 6400 floats + trace + tables
    per_job = 3 * (2 * 3 * 6400 * 4) + 2 * 6400 * 8 + 64 * 3 * 4 + 4 * 64 * 8
    srv = xf.Server(max_jobs=8, mem_budget_bytes=int(2.5 * per_job) + 4096, chunk_steps=10, tile_pairs=TILE)
    ids = [srv.submit(p) for p in ps]
    srv.drain(120.0)
    st = srv.stats()
    assert st["completed"] == 5 and st["max_resident"] == 2
    assert st["mem_peak_bytes"] <= int(2.5 * per_job) + 4096
    for j in ids:
        assert srv.poll(j)[0]["status"] == "XF_OK"
    srv.close()


def test_failing_job_does_not_disturb_others(xf, orc):
    ps = jobs(precision=I.FP64, stepper=I.RK4, n=3, seed=130)
    bad = ps[0].replace(r0=10.0, mu0=1e5, n_steps=200, r1=10.0 + 0.095 * 200)
    rho0s = [orc.init_state(p) for p in ps]
    srv = xf.Server(max_jobs=4, mem_budget_bytes=1 << 30, chunk_steps=40, stepper=I.RK4, precision=I.FP64,
                    tile_pairs=TILE)
    jb = srv.submit(bad, rho0=orc.init_state(bad), keep_state=True)
    ids = [srv.submit(p, rho0=r, keep_state=True) for p, r in zip(ps[1:], rho0s[1:])]
    res = collect(srv, [jb] + ids)
    assert res[jb][0]["status"] == "XF_E_NONFINITE" and res[jb][0]["steps"] < 200
    assert np.isfinite(res[jb][1]).all()
    for p, r0, j in zip(ps[1:], rho0s[1:], ids):
        assert res[j][0]["status"] == "XF_OK"
        assert np.array_equal(res[j][1], alone(xf, p, r0))
    srv.close()
