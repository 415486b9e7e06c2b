"""Host logic of bench.py that its JSON line rests on: the survival-probability
error of the batched leg's accuracy check, the sample it checks, the
target-guarded split of the ensemble, and the cross-rank timing helpers."""
import os
import sys

import numpy as np

from paper_1907_05560_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _state(n_f, n_bins, seed):
    """A packed state [s][bin][n_f^2] with distinct e / x diagonals."""
    g = np.random.default_rng(seed)
    m = n_f * n_f
    x = np.zeros((2, n_bins, m))
    x[:, :, 0] = 0.5 + 0.4 * g.random((2, n_bins))
    x[:, :, 1] = 0.1 * g.random((2, n_bins))
    x[:, :, n_f:] = 1e-3 * g.standard_normal((2, n_bins, m - n_f))
    return x.reshape(-1)


def test_p_surv_error_definition():
    """P_surv = (rho_ee - phi_x) / (phi_e - phi_x) with phi from the initial
    diagonal: the same state gives 0, a shift d of rho_ee in one bin gives
    d / (phi_e - phi_x) of that bin, and bins whose spectra cannot be told
    apart (|phi_e - phi_x| below 1e-2 of the largest) are left out."""
    for n_f in (2, 3):
        rho0 = _state(n_f, 50, seed=n_f)
        assert bench.p_surv_error(rho0, rho0, rho0, n_f) == 0.0
        got = rho0.copy().reshape(2, 50, n_f * n_f)
        got[1, 7, 0] += 1e-4
        x0 = rho0.reshape(2, 50, n_f * n_f)
        want = 1e-4 / abs(x0[1, 7, 0] - x0[1, 7, 1])
        assert abs(bench.p_surv_error(got.reshape(-1), rho0, rho0, n_f) - want) < 1e-12 * want
        # a bin with (nearly) equal spectra does not count
        x0m = x0.copy()
        x0m[0, 3, 1] = x0m[0, 3, 0] - 1e-9
        got2 = x0m.copy()
        got2[0, 3, 0] += 0.3
        assert bench.p_surv_error(got2.reshape(-1), x0m.reshape(-1), x0m.reshape(-1), n_f) == 0.0


def test_batch_sample_is_the_k_smallest():
    probs = I.ensemble_problems()
    s = bench.batch_sample(probs, 16)
    assert len(s) == 16 and s == sorted(s)
    largest_in = max(probs[i].n_bins for i in s)
    assert all(probs[i].n_bins >= largest_in for i in range(len(probs)) if i not in s)


def test_target_guarded_split_of_the_ensemble():
    """The split the bench times: FP32 bins up to the measured mu0 bound, the
    rest in float-float bins; every problem lands in exactly one pack."""
    probs = I.ensemble_problems()
    lo = [q for q in probs if q.mu0 <= bench.FP32_TARGET_MU0]
    hi = [q for q in probs if q.mu0 > bench.FP32_TARGET_MU0]
    assert len(lo) + len(hi) == 256
    assert (len(lo), len(hi)) == (167, 89)
    assert bench.P_SURV_TARGET == 1e-3
    # the bound sits below the smallest mu0 at which a sampled FP32 run missed
    # the target (1.39e5, three flavors) and below 7e4 (7.9e-4, the closest)
    assert bench.FP32_TARGET_MU0 < 7e4


def test_whole_job_rate_and_single_rank_max():
    assert bench.whole_job_rate(1e6, 4, 2.0) == 2e6
    assert bench.max_over_ranks(3.5, 1) == 3.5
