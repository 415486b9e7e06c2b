"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element on the same seeded inputs.

Gate (FP64): for every bin b and packed component k,
    |rho_gpu[b,k] - rho_oracle[b,k]| / tr(rho_b)  <=  1e-9.
The oracle's trajectories amplify rounding-level differences only mildly on
these workloads (a 1e-16 relative perturbation grows to ~3e-13 over the full
50 -> 250 km run), so the gate holds over whole runs.
"""
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL64 = 1e-9
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
    tr = np.abs(B[:, :n_f].sum(1))
    return float((np.abs(A - B).max(1) / tr).max())


def gpu_run(X, p, rho0, r0, h, n, allocator="torch"):
    c = X.Context(p, allocator=allocator)
    c.set_state(rho0, r0)
    c.step(n, h)
    rho, r, done = c.get_state()
    c.close()
    return rho, r, done


def small(**kw):
    base = dict(n_E=8, n_u=6, n_f=2, stepper=I.RK4, mu0=1e5, r0=50.0, r1=52.0, n_steps=200,
                eps=1e-2, seed=11)
    base.update(kw)
    return I.Problem(**base)


THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1)


# ------------------------------------------------------------------ set-up

@pytest.mark.parametrize("n_f", [2, 3])
def test_init_state_and_tables_match_oracle(xf, orc, n_f):
    kw = THREE if n_f == 3 else {}
    p = small(n_u=7, n_E=33, eps=1e-6, seed=5, **kw)
    c = xf.Context(p)
    c.init_state(p.r0)
    rho, r, n = c.get_state()
    E, phi = c.tables()
    Eo, uo, phio, Hvo = orc.tables(p)
    assert np.allclose(E, Eo, rtol=1e-15, atol=0)
    assert np.allclose(phi, phio, rtol=1e-12, atol=0)
    ref = orc.init_state(p)
    # both sides compute the spectra with their own quadrature of Eq. 4.2
    assert rel_err(rho, ref, n_f) < 1e-12
    assert r == p.r0 and n == 0


@pytest.mark.parametrize("geometry", [I.BULB, I.MU_R4, I.CONST])
@pytest.mark.parametrize("n_f", [2, 3])
def test_moments_match_oracle(xf, orc, n_f, geometry):
    kw = THREE if n_f == 3 else {}
    p = small(n_u=9, n_E=17, geometry=geometry, **kw)
    rho = orc.init_state(p)
    c = xf.Context(p)
    c.set_state(rho, 23.0)
    M0, M1 = c.moments()
    R0, R1 = orc.moments(p, rho, 23.0)
    scale = np.abs(R0).max()
    assert np.abs(M0 - R0).max() < 1e-13 * scale
    assert np.abs(M1 - R1).max() < 1e-13 * max(scale, np.abs(R1).max())


# ------------------------------------------------------------------ small parity sweep

CASES = [
    # (n_u, n_E, geometry, matter)
    (1, 1, I.CONST, False),
    (3, 7, I.BULB, False),
    (16, 32, I.BULB, False),
    (5, 33, I.BULB, "power"),
    (6, 21, I.BULB, "exp"),
    (4, 9, I.MU_R4, False),
    (4, 9, I.MU_R4, "exp"),
    (1, 13, I.SINGLE_ANGLE, False),
]


@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
@pytest.mark.parametrize("n_f", [2, 3])
@pytest.mark.parametrize("n_u,n_E,geometry,matter", CASES)
def test_parity_small(xf, orc, n_u, n_E, geometry, matter, n_f, stepper):
    kw = dict(THREE) if n_f == 3 else {}
    mu0 = 50.0 if geometry == I.CONST else 1e5
    if matter == "power":
        # A(50 km) ~ 51 km^-1: A h ~ 0.5 keeps explicit RK4 stable
        kw.update(matter=I.MATTER_POWER, ne_ref=1e31, r_ref=10.0, ne_power=3.0)
    elif matter == "exp":
        # Eq. 4.4 with Y_e: A(50 km) ~ 50 km^-1, scale height 20 km
        kw.update(matter=I.MATTER_EXP, nb0=1.15e30, Ye=0.5, h_ns=20.0)
    p = small(n_u=n_u, n_E=n_E, geometry=geometry, stepper=stepper, mu0=mu0, **kw)
    rho0 = orc.init_state(p)
    ref, st, done = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    assert st == 0
    got, r, n = gpu_run(xf, p, rho0, p.r0, p.h, p.n_steps)
    assert n == p.n_steps and r == pytest.approx(p.r1, rel=1e-14)
    assert np.abs(ref - rho0).max() > 1e-6  # the state actually moved
    assert rel_err(got, ref, n_f) < TOL64


@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
@pytest.mark.parametrize("n_f", [2, 3])
def test_parity_many_ctas_ragged(xf, orc, n_f, stepper):
    """Enough pairs for a multi-CTA grid with a grid barrier; sizes are not
    multiples of any tile (ragged last CTA)."""
    kw = THREE if n_f == 3 else {}
    p = small(n_u=101, n_E=97, stepper=stepper, n_steps=40, r1=50.4, **kw)
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    c = xf.Context(p)
    g, t, b = c.launch_info()
    assert g > 1
    c.set_state(rho0, p.r0)
    c.step(p.n_steps, p.h)
    got, r, n = c.get_state()
    assert rel_err(got, ref, n_f) < TOL64


# ------------------------------------------------------------------ full workloads

def test_parity_c1a_full_run_rk4(xf, orc):
    """Two flavors, 16 x 32 bins, RK4, 20000 steps from 50 to 250 km."""
    p = I.bulb2f_16x32_from_50km()
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    got, r, n = gpu_run(xf, p, rho0, p.r0, p.h, p.n_steps)
    assert n == p.n_steps
    assert rel_err(got, ref, 2) < TOL64


def test_parity_c1_full_run_exph(xf, orc):
    """The literal two-flavor run (10 -> 200 km, 2000 steps) with the paper's
    predictor-corrector and exact propagator."""
    p = I.bulb2f_16x32()
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    got, r, n = gpu_run(xf, p, rho0, p.r0, p.h, p.n_steps)
    assert st == 0 and n == p.n_steps
    assert rel_err(got, ref, 2) < TOL64


@pytest.mark.parametrize("make", [I.bulb3f_1000x200, I.bulb3f_1000x200_from_250km])
def test_parity_three_flavor_full_size(xf, orc, make):
    """400,000 3x3 bins (1000 angles x 200 energies) in the launch shape the
    bench uses (persistent launches of 100 radial steps): 200 steps against
    the oracle on every bin (10 -> 19.9 km for the predictor-corrector run,
    the start of the bench's own range; 250 -> 257.5 km for RK4)."""
    p = make()
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
    assert done == n and r == pytest.approx(p.r0 + n * p.h, rel=1e-13)
    assert np.abs(ref - rho0).max() > 1e-6 * np.abs(rho0).max()
    err = rel_err(got, ref, 3)
    print(f"{make.__name__}: max |d rho| / tr rho after {n} steps = {err:.3e}")
    assert err < TOL64


@pytest.mark.skipif(not os.environ.get("XF_FULL_RUN"), reason="set XF_FULL_RUN=1: about 25 min of oracle time")
def test_parity_three_flavor_full_run(xf, orc):
    """The whole three-flavor bulb run (1000 angles x 200 energies, matter
    r^-3, 20000 predictor-corrector steps from 10 to 1000 km) against the
    oracle, both in chunks of 2000 steps, the error printed at every chunk.
    The device's sine-cosine differs from the host library's by ulps and the
    nonlinear flow amplifies such differences, so the gate applies where the
    flow has not amplified them (max error printed for every radius)."""
    p = I.bulb3f_1000x200()
    rho0 = orc.init_state(p)
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    ref = rho0
    errs = []
    k = 0
    while k < p.n_steps:
        m = min(2000, p.n_steps - k)
        ref, st, _ = orc.evolve(p, ref, p.r0 + k * p.h, p.h, m, n_threads=THREADS)
        assert st == 0
        for _ in range(m // 100):
            c.step_async(100, p.h)
        c.sync()
        k += m
        got, r, done = c.get_state()
        assert done == k
        errs.append((r, rel_err(got, ref, 3)))
        print(f"r = {r:8.3f} km  steps {k:6d}  max |d rho| / tr rho = {errs[-1][1]:.3e}", flush=True)
    c.close()
    assert max(e for _, e in errs) < TOL64


# ------------------------------------------------------------------ status paths

def test_literal_rk4_reports_nonfinite_like_oracle(xf, orc):
    """Explicit RK4 from 10 km at h = 0.095 km diverges; both sides stop and
    keep the last finite state."""
    p = I.bulb2f_16x32().replace(stepper=I.RK4)
    rho0 = orc.init_state(p)
    ref, st, done_o = orc.evolve(p, rho0, p.r0, p.h, 400, n_threads=THREADS)
    assert st == 1
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    with pytest.raises(xf.XFError) as ei:
        c.step(400, p.h)
    assert ei.value.name == "XF_E_NONFINITE"
    got, r, done = c.get_state()
    assert np.isfinite(got).all()
    # past the blow-up the states are ~1e200 and not comparable; the stop
    # step itself must agree to within one step
    assert abs(done - done_o) <= 1


def test_strict_rk4_refuses_unstable_step_sizes(xf, orc):
    """Strict mode: the literal 10 km RK4 step (h = 0.095 km, mu0 = 1e5) is
    refused before any step is taken; the stable 50 km companion
    (h = 0.01 km) runs and matches the oracle."""
    p = I.bulb2f_16x32().replace(stepper=I.RK4, strict=1)
    rho0 = orc.init_state(p)
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    with pytest.raises(xf.XFError) as ei:
        c.step(10, p.h)
    assert ei.value.name == "XF_E_UNSTABLE"
    got, r, done = c.get_state()
    # untouched: only the packing round trip (trace split in FP64) differs
    assert done == 0 and r == p.r0 and np.abs(got - rho0).max() <= 1e-15 * np.abs(rho0).max()
    c.close()
    q = I.bulb2f_16x32_from_50km().replace(strict=1, n_steps=200, r1=52.0)
    rho0 = orc.init_state(q)
    c = xf.Context(q)
    c.set_state(rho0, q.r0)
    c.step(q.n_steps, q.h)
    ref, ok, _ = orc.evolve(q, rho0, q.r0, q.h, q.n_steps, n_threads=THREADS)
    assert rel_err(c.get_state()[0], ref, q.n_f) < 1e-9
    c.close()


def test_step_before_state_and_bad_state(xf):
    p = small()
    c = xf.Context(p)
    with pytest.raises(xf.XFError) as ei:
        c.step(1, 0.01)
    assert ei.value.name == "XF_E_STATE"
    bad = np.zeros(2 * p.n_u * p.n_E * 4)
    bad[5] = np.nan
    with pytest.raises(xf.XFError) as ei:
        c.set_state(bad, p.r0)
    assert ei.value.name == "XF_E_STATE"


def test_deterministic_and_async_chunks_equal(xf, orc):
    p = small(n_u=64, n_E=64, n_steps=60, r1=50.6)
    rho0 = orc.init_state(p)
    a, _, _ = gpu_run(xf, p, rho0, p.r0, p.h, p.n_steps)
    b, _, _ = gpu_run(xf, p, rho0, p.r0, p.h, p.n_steps, allocator="cuda")
    assert np.array_equal(a, b)
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    for _ in range(3):
        c.step_async(20, p.h)
    c.sync()
    d, r, n = c.get_state()
    assert n == 60 and r == pytest.approx(p.r1, rel=1e-14)
    assert np.array_equal(a, d)


def test_outputs_match_state(xf, orc):
    p = small(n_f=3, n_u=5, n_E=11, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72))
    rho0 = orc.init_state(p)
    ref, _, _ = orc.evolve(p, rho0, p.r0, p.h, 50)
    c = xf.Context(p)
    c.set_state(ref, p.r0)
    ps, tr, pur = c.outputs()
    E, uo, phi, Hv = orc.tables(p)
    M = orc.unpack(ref, 3).reshape(2, p.n_u, p.n_E, 3, 3)
    want_tr = np.trace(M, axis1=3, axis2=4).real.reshape(-1)
    T = M - want_tr.reshape(2, p.n_u, p.n_E)[..., None, None] / 3 * np.eye(3)
    want_pur = np.einsum("...ij,...ji->...", T, T).real.reshape(-1)
    pe = np.stack([np.broadcast_to(phi[0], (p.n_u, p.n_E)), np.broadcast_to(phi[1], (p.n_u, p.n_E))])
    px = np.stack([np.broadcast_to(phi[2], (p.n_u, p.n_E)), np.broadcast_to(phi[3], (p.n_u, p.n_E))])
    want_ps = ((M[..., 0, 0].real - px) / (pe - px)).reshape(-1)
    assert np.allclose(tr, want_tr, rtol=1e-14)
    assert np.allclose(pur, want_pur, rtol=1e-10, atol=1e-30)
    assert np.allclose(ps, want_ps, rtol=1e-9)


# ------------------------------------------------------------------ precision variant

def test_fp32_m64_error_vs_fp64_oracle(xf, orc):
    """FP32 per-bin arithmetic with FP64 moments: survival-probability error
    against the FP64 oracle on the stable two-flavor run (50 km on, h = 0.01),
    over bins whose spectra are distinguishable (|phi_e - phi_x| >= 1e-2 max)."""
    p = I.bulb2f_16x32_from_50km().replace(n_steps=5000, r1=100.0)
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    q = p.replace(precision=I.FP32_M64)
    c = xf.Context(q)
    c.set_state(rho0, p.r0)
    c.step(p.n_steps, p.h)
    ps, tr, pur = c.outputs()
    c64 = xf.Context(p)
    c64.set_state(ref, p.r1)
    ps64, _, _ = c64.outputs()
    E, uo, phi, Hv = orc.tables(p)
    sep = np.concatenate([np.tile(np.abs(phi[0] - phi[2]), p.n_u), np.tile(np.abs(phi[1] - phi[3]), p.n_u)])
    mask = sep >= 1e-2 * sep.max()
    err = np.abs(ps - ps64)[mask].max()
    print(f"FP32_M64 max |dP_surv| = {err:.3e}")
    assert err < 1e-3


@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
def test_forced_grid_shapes_match_oracle(xf, orc, stepper):
    """A problem of 8 tiles forced onto 2, 3 and 7 CTAs (grid barrier, several
    tiles per CTA, ragged last tile) agrees with the oracle, is deterministic,
    and gives bitwise the same result for every grid (per-problem tile tree)."""
    p = small(n_u=57, n_E=32, n_steps=100, r1=51.0, stepper=stepper)
    rho0 = orc.init_state(p)
    ref, _, _ = orc.evolve(p, rho0, p.r0, p.h, p.n_steps, n_threads=THREADS)
    first = None
    for g in (2, 3, 7):
        outs = []
        for _ in range(2):
            c = xf.Context(p)
            c.set_option(xf.OPT_TILE_PAIRS, 256)
            c.set_option(xf.OPT_GRID, g)
            assert c.launch_info()[0] == g
            c.set_state(rho0, p.r0)
            c.step(p.n_steps, p.h)
            outs.append(c.get_state()[0])
        assert np.array_equal(outs[0], outs[1])
        assert rel_err(outs[0], ref, 2) < TOL64
        if first is None:
            first = outs[0]
        assert np.array_equal(first, outs[0])


def test_barrier_wait_times_out_with_status(xf, orc):
    """One CTA leaves without arriving: the others' bounded barrier wait runs
    out (short limit), the kernel returns and the host reads
    XF_E_BARRIER_TIMEOUT; the context stays usable after a fresh state."""
    p = small(n_u=40, n_E=32, n_steps=10, r1=50.1)
    rho0 = orc.init_state(p)
    c = xf.Context(p)
    c.set_option(xf.OPT_TILE_PAIRS, 256)
    c.set_option(xf.OPT_GRID, 4)
    assert c.launch_info()[0] == 4
    c.set_option(xf.OPT_BARRIER_TIMEOUT_NS, 50_000_000)
    c.set_option(xf.OPT_TEST_SKIP_ARRIVAL, 2)
    c.set_state(rho0, p.r0)
    with pytest.raises(xf.XFError) as ei:
        c.step(10, p.h)
    assert ei.value.name == "XF_E_BARRIER_TIMEOUT"
    c.set_option(xf.OPT_TEST_SKIP_ARRIVAL, -1)
    c.set_state(rho0, p.r0)
    c.step(10, p.h)
    ref, _, _ = orc.evolve(p, rho0, p.r0, p.h, 10)
    assert rel_err(c.get_state()[0], ref, 2) < TOL64


@pytest.mark.parametrize("make", [I.bulb3f_1000x200, I.bulb3f_1000x200_from_250km])
def test_fp32_three_flavor_error_vs_fp64_oracle(xf, orc, make):
    """FP32 bins with FP64 moments on the full three-flavor workload, 20 steps
    against the FP64 oracle on every bin: the error stays at FP32 rounding
    amplified by the phase per step (A h ~ 3e4 rad at 10 km)."""
    p = make()
    n = 20
    rho0 = orc.init_state(p)
    ref, st, _ = orc.evolve(p, rho0, p.r0, p.h, n, n_threads=THREADS)
    got, r, done = gpu_run(xf, p.replace(precision=I.FP32_M64), rho0, p.r0, p.h, n)
    err = rel_err(got, ref, 3)
    print(f"{make.__name__} FP32_M64 rel err after {n} steps: {err:.3e}")
    assert done == n and err < 1e-4


@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
@pytest.mark.parametrize("n_f", [2, 3])
def test_degenerate_cases(xf, orc, n_f, stepper):
    """Zero steps leave the state bitwise; a vanishing Hamiltonian (no mass
    splitting, no matter, no coupling: lambda = 0 in the rotation, a zero
    matrix for the eigensolver) leaves every bin unchanged to rounding."""
    kw = dict(THREE) if n_f == 3 else {}
    p = small(n_u=5, n_E=9, stepper=stepper, **kw)
    rho0 = orc.init_state(p)
    c = xf.Context(p)
    c.set_state(rho0, p.r0)
    before = c.get_state()[0]
    c.step(0, p.h)
    after, r, n = c.get_state()
    c.close()
    assert n == 0 and r == p.r0 and np.array_equal(before, after)
    q = p.replace(dm2=(0.0, 0.0), mu0=0.0, matter=I.MATTER_NONE)
    got, r, n = gpu_run(xf, q, rho0, q.r0, q.h, 50)
    assert n == 50
    assert np.abs(got - rho0).max() <= 1e-14 * np.abs(rho0).max()  # the pack round trip


def _lepton_invariants(orc, p, rho):
    """tr(Pi_k F) with F = sum_{u,e} (rho_nu - conj rho_nubar) / n_u and Pi_k
    the vacuum mass-basis projectors (the oracle's unpacking and tables)."""
    n = p.n_f
    M = orc.unpack(rho, n).reshape(2, p.n_u, p.n_E, n, n)
    F = (M[0] - M[1].conj()).sum(axis=(0, 1)) / p.n_u
    _, _, _, Hv = orc.tables(p)
    _, V = np.linalg.eigh(orc.unpack(Hv[:1].reshape(-1), n)[0])
    return np.array([(V[:, k].conj() @ F @ V[:, k]).real for k in range(n)]), np.abs(F).max()


@pytest.mark.parametrize("n_f", [2, 3])
def test_lepton_number_moment_conserved(xf, orc, n_f):
    """Without matter the nu-nu terms cancel in d/dr tr(Pi_k F) (Eq. 3.13-3.15:
    sum_u (du/c_u)[M0 - c_u M1, S_u] = [M0, M0] - [M1, M1] = 0); the GPU's RK4
    keeps this linear invariant to rounding while the bins move at O(1)."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72)) if n_f == 3 else {}
    p = I.Problem(n_E=24, n_u=40, n_f=n_f, stepper=I.RK4, mu0=3e4, r0=20.0, r1=22.0, n_steps=400, eps=1e-2,
                  seed=17, **kw)
    rho = orc.init_state(p)
    c = xf.Context(p)
    c.set_state(rho, p.r0)
    c.step(p.n_steps, p.h)
    out = c.get_state()[0]
    c.close()
    I0, scale = _lepton_invariants(orc, p, rho)
    I1, _ = _lepton_invariants(orc, p, out)
    assert np.abs(orc.unpack(out, n_f) - orc.unpack(rho, n_f)).max() > 1e-4
    assert np.abs(I1 - I0).max() < 1e-12 * scale
