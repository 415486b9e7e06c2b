"""The FP32 accuracy target at batched and served sizes.

FP32 bins with FP64 moments, radius and phase (XF_FP32_M64) must stay within
1e-3 survival-probability error of the FP64 oracle (the same method, the
paper's predictor-corrector with the exact propagator, Eq. 3.10-3.12) on the
workloads where that precision is used:

* the 256-problem batched ensemble, for its full 1000 steps (50 -> 250 km) in
  the bench's launch configuration (10 steps per replay of a captured CUDA
  graph), checked on its largest three-flavor problem, its largest two-flavor
  problem and two seeded picks;
* a served job of the job stream's largest size (1024 angles x 256 energies,
  two flavors) taken 20000 steps (50 -> 250 km) by the continuous-batching
  server while other jobs share the GPU with it.

P_surv(b) = (rho_ee(b) - phi_x) / (phi_e - phi_x), with phi_e, phi_x the
bin's initial diagonal; bins where the two spectra cross (|phi_e - phi_x| <
1e-2 of the species' largest separation) are left out of the maximum, since
there P_surv is 0/0 (the spectral-crossing reading of the paper's outputs).
Set XF_TARGET_REPORT=<path> to write the measured errors as JSON.
"""
import json
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
TARGET = 1e-3


@pytest.fixture(scope="module")
def xf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05560_gb300 import build, xf as X
    build.build()
    X.load()
    return X


def p_surv_error(got, ref, rho0, p):
    """max |P_surv(got) - P_surv(ref)| over the bins whose spectra are
    distinguishable, and the largest |d rho_ee| / tr rho over all bins."""
    m = p.n_f * p.n_f
    g = got.reshape(2, -1, m)
    r = ref.reshape(2, -1, m)
    x0 = rho0.reshape(2, -1, m)
    worst, worst_ee = 0.0, 0.0
    for s in range(2):
        sep = x0[s, :, 0] - x0[s, :, 1]
        mask = np.abs(sep) >= 1e-2 * np.abs(sep).max()
        ps_g = (g[s, mask, 0] - x0[s, mask, 1]) / sep[mask]
        ps_r = (r[s, mask, 0] - x0[s, mask, 1]) / sep[mask]
        worst = max(worst, float(np.abs(ps_g - ps_r).max()))
        tr = x0[s, :, :p.n_f].sum(1)
        worst_ee = max(worst_ee, float((np.abs(g[s, :, 0] - r[s, :, 0]) / tr).max()))
    return worst, worst_ee


def _report(rows):
    path = os.environ.get("XF_TARGET_REPORT")
    for r in rows:
        print(json.dumps(r))
    if path:
        old = json.load(open(path)) if os.path.exists(path) else []
        keys = {r["case"] for r in rows}
        with open(path, "w") as f:
            json.dump([r for r in old if r["case"] not in keys] + rows, f, indent=1)


def test_batched_ensemble_full_run_meets_target(xf, orc):
    probs = I.ensemble_problems()
    h = probs[0].h
    b = xf.Batch(probs)
    b.set_option(xf.OPT_GRAPH, 1)
    b.init_state_i(-1, probs[0].r0)
    n = probs[0].n_steps
    for _ in range(n // 10):
        b.step_all(10, h)
    sizes = [(q.n_bins, i) for i, q in enumerate(probs)]
    big3 = max(s for s in sizes if probs[s[1]].n_f == 3)[1]
    big2 = max(s for s in sizes if probs[s[1]].n_f == 2)[1]
    g = I.SplitMix64(40)
    picks = [big3, big2] + [g.randint(0, len(probs) - 1) for _ in range(2)]
    rows = []
    for i in picks:
        assert b.status_i(i)[0] == "XF_OK"
        q = probs[i]
        got, r, done = b.get_state_i(i)
        assert done == n and r == pytest.approx(q.r1, rel=1e-12)
        rho0 = orc.init_state(q)
        ref, st, k = orc.evolve(q, rho0, q.r0, q.h, n, n_threads=THREADS)
        assert st == 0 and k == n
        err, err_ee = p_surv_error(got, ref, rho0, q)
        rows.append(dict(case=f"ensemble problem {i}", n_f=q.n_f, n_u=q.n_u, n_E=q.n_E, bins=q.n_bins,
                         mu0=q.mu0, hierarchy=q.hierarchy, steps=n, r_km=q.r1, max_dP_surv=err,
                         max_drho_ee_over_tr=err_ee))
    _report(rows)
    for row in rows:
        assert row["max_dP_surv"] < TARGET, row


def test_served_job_of_the_largest_size_meets_target(xf, orc):
    stream = I.job_arrivals(rate_per_s=200.0, window_s=60.0, seed=5)
    big = max((p for _, p in stream), key=lambda p: p.n_u * p.n_E)
    big = big.replace(n_u=1024, n_E=256, n_steps=20000, r1=50.0 + 0.01 * 20000)
    others = [p.replace(n_steps=min(p.n_steps, 3000), r1=50.0 + 0.01 * min(p.n_steps, 3000))
              for _, p in stream[:3]]
    import torch
    free, _ = torch.cuda.mem_get_info()
    srv = xf.Server(max_jobs=16, mem_budget_bytes=int(min(8e9, free // 4)), chunk_steps=200)
    rho0 = orc.init_state(big)
    jid = srv.submit(big, rho0=rho0, keep_state=True)
    ids = [srv.submit(p) for p in others]   # they share the GPU with the big job
    srv.drain(timeout_s=600.0)
    meta, got = srv.poll(jid, want_state=True)
    assert meta["status"] == "XF_OK" and meta["steps"] == big.n_steps
    assert all(srv.poll(j)[0]["status"] == "XF_OK" for j in ids)
    assert srv.stats()["max_resident"] >= 2
    srv.close()
    ref, st, k = orc.evolve(big, rho0, big.r0, big.h, big.n_steps, n_threads=THREADS)
    assert st == 0 and k == big.n_steps
    err, err_ee = p_surv_error(got, ref, rho0, big)
    row = dict(case="served job", n_f=2, n_u=big.n_u, n_E=big.n_E, bins=big.n_bins, mu0=big.mu0,
               hierarchy=big.hierarchy, theta=big.theta[0], steps=big.n_steps, r_km=big.r1,
               max_dP_surv=err, max_drho_ee_over_tr=err_ee)
    _report([row])
    assert err < TARGET, row
