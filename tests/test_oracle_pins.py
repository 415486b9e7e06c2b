"""Pins for the FP64 CPU oracle: checks against what the paper and the
mathematics fix, independent of the oracle's own code.

Each test names the passage it pins.  None of them calls the CUDA library.
"""
import math
import os

import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _small(**kw):
    base = dict(n_E=8, n_u=6, n_f=2, stepper=I.RK4, mu0=0.0, r0=50.0, r1=52.0, n_steps=200,
                eps=1e-3, seed=7)
    base.update(kw)
    return I.Problem(**base)


def _trace(rho, n_f):
    x = rho.reshape(-1, n_f * n_f)
    return x[:, :n_f].sum(1)


# ---------------------------------------------------------------- constants

def test_vacuum_coefficient_matches_pdg_phase(orc):
    """Eq. 3.6: Delta = dm^2/(2E); Delta*L/2 is the textbook phase
    1.26693 dm^2[eV^2] L[km] / E[GeV]."""
    ref = float(dict((r[0], r[1]) for r in _golden("constants.txt"))["osc_phase_per_eV2_km_per_GeV"])
    # Delta L / 2 per (eV^2 km / MeV) = coeff / 2 ; per GeV: * 1e-3
    assert orc.vac_coeff() / 2 * 1e-3 == pytest.approx(ref, rel=2e-5)


def test_matter_coefficient_matches_pdg(orc):
    """Eq. 3.7: A = sqrt(2) G_F n_e = 7.63e-14 eV at n_e = N_A cm^-3."""
    ref = float(dict((r[0], r[1]) for r in _golden("constants.txt"))["matter_potential_eV_per_NA_cm3"])
    hbarc_ev_km = 1.973269804e-10
    got_ev = orc.matter_coeff() * 6.02214076e23 * hbarc_ev_km
    assert got_ev == pytest.approx(ref, rel=1e-3)


# ---------------------------------------------------------------- spectra

def test_fd_integrals_closed_form_at_zero(orc):
    """Eq. 4.2 at eta = 0: F_k(0) = (1 - 2^-k) k! zeta(k+1)."""
    zeta3, zeta4 = 1.2020569031595942, math.pi ** 4 / 90
    assert orc.fd_integral(2, 0.0) == pytest.approx(0.75 * 2 * zeta3, rel=1e-14)
    assert orc.fd_integral(3, 0.0) == pytest.approx(0.875 * 6 * zeta4, rel=1e-14)


def test_fd_integrals_match_polylog(orc):
    """Eq. 4.2: F_k(eta) = -k! Li_{k+1}(-e^eta) (library polylog)."""
    mpmath = pytest.importorskip("mpmath")
    for k in (2, 3):
        for eta in (-1.0, 1.5, 3.0):
            ref = float(-math.factorial(k) * mpmath.polylog(k + 1, -mpmath.e ** eta))
            assert orc.fd_integral(k, eta) == pytest.approx(ref, rel=1e-14)


def test_fd_temperatures_reproduce_paper(orc):
    """Sec. 4.5 prints T = 2.76/4.01/6.26 MeV for <E> = 11/16/25 MeV, eta = 3;
    <E> = T F3/F2 (Eq. 4.1-4.2)."""
    for name, meanE, eta, T in _golden("fd_temperatures.txt"):
        ratio = orc.fd_integral(3, float(eta)) / orc.fd_integral(2, float(eta))
        assert round(float(meanE) / ratio, 2) == pytest.approx(float(T), abs=1e-9), name


def test_spectrum_normalised_and_flux_ratios(orc):
    """Eq. 4.1 is a normalised distribution; the number-flux weight of each
    species is L/<E> relative to nu_e, i.e. <E_nue>/<E_a> at equal L."""
    p = I.Problem(n_E=4000, E_min=0.0, E_max=150.0)
    E, u, phi, Hv = orc.tables(p)
    dE = E[1] - E[0]
    ratio = orc.fd_integral(3, 3.0) / orc.fd_integral(2, 3.0)
    meanE = [T * ratio for T in p.T]
    for a in range(4):
        assert phi[a].sum() * dE == pytest.approx(meanE[0] / meanE[a], rel=1e-6)


# ---------------------------------------------------------------- eigen / propagator

def _rand_herm(rng, n, degenerate=False):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = A + A.conj().T
    if degenerate:
        w, V = np.linalg.eigh(H)
        w[1] = w[0]
        H = (V * w) @ V.conj().T
        H = 0.5 * (H + H.conj().T)
    return H


@pytest.mark.parametrize("n", [2, 3])
def test_jacobi_eigh_matches_lapack(orc, n):
    rng = np.random.default_rng(n)
    for trial in range(40):
        H = _rand_herm(rng, n, degenerate=(trial % 5 == 0))
        w, V = orc.eigh(orc.pack(H[None]))
        assert np.allclose(np.sort(w), np.linalg.eigvalsh(H), atol=1e-12 * np.abs(H).max())
        assert np.allclose(V.conj().T @ V, np.eye(n), atol=1e-13)
        assert np.allclose((V * w) @ V.conj().T, H, atol=1e-12 * np.abs(H).max())


@pytest.mark.parametrize("n", [2, 3])
def test_propagator_matches_scipy_expm(orc, n):
    """Eq. 3.10-3.12 (2 flavors) and the spectral form (3 flavors) equal
    exp(-iHt) up to the global phase of tr(H)."""
    expm = pytest.importorskip("scipy.linalg").expm
    rng = np.random.default_rng(10 + n)
    for trial in range(30):
        H = _rand_herm(rng, n, degenerate=(trial % 6 == 0))
        t = rng.uniform(0.01, 3.0)
        U = orc.expm(orc.pack(H[None]), t)
        H0 = H - np.trace(H).real / n * np.eye(n)
        assert np.allclose(U, expm(-1j * H0 * t), atol=1e-12)


# ---------------------------------------------------------------- closed forms

def _path_length(p, r):
    """l(r) - l(r0) with l = r cos(theta) (Eq. 3.3), per angle bin."""
    u = (np.arange(p.n_u) + 0.5) / p.n_u
    l = lambda rr: rr * np.sqrt(1.0 - (p.R_nu / rr) ** 2 * u)
    return l(r) - l(p.r0)


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 2e-8), (I.EXPH, 1e-11)])
def test_vacuum_two_flavor_survival(orc, stepper, tol):
    """P1: mu = A = 0 gives P_ee = 1 - sin^2(2 theta) sin^2(Delta L / 2) along
    each trajectory (Eq. 3.5-3.6, Eq. 3.3); ee entry = phi_x + (phi_e - phi_x) P_ee."""
    p = _small(n_E=12, n_u=5, stepper=stepper, eps=0.0, theta=(0.3, 0, 0), hierarchy=-1,
               E_min=1.0, E_max=13.0, r0=20.0, r1=30.0, n_steps=1000)
    E, u, phi, Hv = orc.tables(p)
    rho = orc.init_state(p)
    out, st, done = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    assert st == 0 and done == p.n_steps
    M = orc.unpack(out, 2).reshape(2, p.n_u, p.n_E, 2, 2)
    Lj = _path_length(p, p.r1)
    Delta = orc.vac_coeff() * p.hierarchy * p.dm2[0] / E
    Pee = 1 - np.sin(2 * 0.3) ** 2 * np.sin(np.outer(Lj, Delta) / 2) ** 2
    for s, (ie, ix) in enumerate([(0, 2), (1, 3)]):
        want = phi[ix] + (phi[ie] - phi[ix]) * Pee
        assert np.abs(M[s, :, :, 0, 0].real - want).max() < tol * phi[0].max()


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 2e-8), (I.EXPH, 1e-11)])
def test_constant_matter_msw(orc, stepper, tol):
    """P2: constant matter.  Textbook two-flavor MSW (Wolfenstein; Mikheyev-
    Smirnov): Delta_m = sqrt((Delta cos2t -+ A)^2 + (Delta sin2t)^2),
    sin 2t_m = Delta sin 2t / Delta_m, with -A for antineutrinos."""
    p = _small(n_E=12, n_u=1, geometry=I.CONST, stepper=stepper, eps=0.0, theta=(0.2, 0, 0),
               hierarchy=+1, E_min=1.0, E_max=25.0, matter=I.MATTER_POWER, ne_ref=2.0e27,
               ne_power=0.0, r0=20.0, r1=24.0, n_steps=800)
    E, u, phi, Hv = orc.tables(p)
    A = orc.matter_A(p, 22.0)
    Delta = orc.vac_coeff() * p.dm2[0] / E
    assert 0.1 < A / Delta.max() and A / Delta.min() < 10  # spans the resonance
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    M = orc.unpack(out, 2).reshape(2, p.n_E, 2, 2)
    L = p.r1 - p.r0
    c2, s2 = math.cos(0.4), math.sin(0.4)
    for s, sgn, (ie, ix) in [(0, +1, (0, 2)), (1, -1, (1, 3))]:
        Dm = np.sqrt((Delta * c2 - sgn * A) ** 2 + (Delta * s2) ** 2)
        sin2m = Delta * s2 / Dm
        Pee = 1 - sin2m ** 2 * np.sin(Dm * L / 2) ** 2
        want = phi[ix] + (phi[ie] - phi[ix]) * Pee
        assert np.abs(M[s, :, 0, 0].real - want).max() < tol * phi[0].max()


@pytest.mark.parametrize("hierarchy", [+1, -1])
def test_constant_matter_three_flavor(orc, hierarchy):
    """P3 with matter: three flavors in constant matter (Eq. 3.4-3.7 with the
    three-flavor vacuum term, delta_CP = 0) is a constant Hamiltonian, so
    rho(L) = exp(-iHL) rho(0) exp(iHL) with the library exponential
    (scipy.linalg.expm).  H_nu = U diag(0, dm21, +-dm31) U^T / 2E + A diag(1, 0, 0),
    H_nubar the same with -A; U the textbook PMNS matrix.  The predictor-
    corrector is exact for a constant H; the density spans the resonances."""
    from scipy.linalg import expm
    p = _small(n_f=3, n_E=6, n_u=1, geometry=I.CONST, stepper=I.EXPH, eps=1e-2, dm2=(7.5e-5, 2.4e-3),
               theta=(0.59, 0.15, 0.72), hierarchy=hierarchy, E_min=2.0, E_max=40.0,
               matter=I.MATTER_POWER, ne_ref=5e26, ne_power=0.0, r0=20.0, r1=24.0, n_steps=200)
    E, u, phi, Hv = orc.tables(p)
    A = 5e26 * orc.matter_coeff()
    K = orc.vac_coeff()
    assert K * 2.4e-3 / E.max() < A < K * 2.4e-3 / E.min()
    s12, c12 = math.sin(0.59), math.cos(0.59)
    s13, c13 = math.sin(0.15), math.cos(0.15)
    s23, c23 = math.sin(0.72), math.cos(0.72)
    U = np.array([[c12 * c13, s12 * c13, s13],
                  [-s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13],
                  [s12 * s23 - c12 * c23 * s13, -c12 * s23 - s12 * c23 * s13, c23 * c13]])
    m2 = np.array([0.0, 7.5e-5, hierarchy * 2.4e-3])
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    assert st == 0
    R0 = orc.unpack(rho, 3).reshape(2, p.n_E, 3, 3)
    R1 = orc.unpack(out, 3).reshape(2, p.n_E, 3, 3)
    L = p.r1 - p.r0
    for s, sgn in ((0, 1.0), (1, -1.0)):
        for e in range(p.n_E):
            H = K * U @ np.diag(m2) @ U.T / E[e] + sgn * A * np.diag([1.0, 0.0, 0.0])
            V = expm(-1j * H * L)
            want = V @ R0[s, e] @ V.conj().T
            assert np.abs(R1[s, e] - want).max() < 1e-11 * np.trace(R0[s, e]).real


# ---------------------------------------------------------------- matter profiles (Eq. 3.7, 4.3, 4.4)
#
# The matter potential A(r) = sqrt(2) G_F Y_e n_b(r) enters only through the
# flavor evolution it drives.  These pins check that evolution against closed
# forms of the two-flavor MSW problem (mu = 0, one radial trajectory), whose
# inputs are the profile's stated shape: n_e = n_ref (r_ref / r)^p (Eq. 4.3,
# p = 3) and n_b' = n_b0 exp(-(r - R) / h_NS) with n_e = Y_e n_b (Eq. 3.7, 4.4).

def _msw(matter, th, n_E, E=(5.0, 45.0), **kw):
    return _small(n_E=n_E, n_u=1, geometry=I.CONST, stepper=I.EXPH, mu0=0.0, eps=0.0,
                  theta=(th, 0, 0), dm2=(2.4e-3, 0), hierarchy=+1, E_min=E[0], E_max=E[1],
                  matter=matter, R_nu=10.0, **kw)


def _pure_nu_e(orc, p):
    """Every neutrino and antineutrino bin in its electron flavor."""
    rho = np.zeros(orc.state_size(p)).reshape(2, p.n_E, 4)
    rho[:, :, 0] = 1.0
    return rho.reshape(-1)


def _populations(orc, rho, p, vecs):
    """<v|rho|v> for each bin, v = vecs[s][e] (a unit 2-vector)."""
    M = orc.unpack(rho, 2).reshape(2, p.n_E, 2, 2)
    return np.einsum("sei,seij,sej->se", vecs.conj(), M, vecs).real


def _mass_basis_nu1(p):
    """The lighter vacuum mass state (cos t, -sin t) of H_vac = (Delta/2)
    [[-cos 2t, sin 2t], [sin 2t, cos 2t]] (Eq. 3.5), normal ordering."""
    th = p.theta[0]
    v = np.array([math.cos(th), -math.sin(th)])
    return np.broadcast_to(v, (2, p.n_E, 2))


def test_exponential_profile_hop_probability_is_exact(orc):
    """Eq. 3.7 with the exponential profile of Eq. 4.4: an electron neutrino
    that starts far above resonance (A >> Delta) and leaves into vacuum ends in
    the lighter mass state with the probability of the exactly solvable
    exponential-density problem (Petcov 1988; Kuo & Pantaleone 1989, the
    double-exponential formula with F = 1 - tan^2 t):
        P_c = (exp(-2 pi Delta h sin^2 t) - exp(-2 pi Delta h)) / (1 - exp(-2 pi Delta h)),
    Delta = dm^2 / 2E, h the scale height h_NS.  Antineutrinos see -A (after
    Eq. 3.4) and cross no resonance; they are the same problem with sin^2 t ->
    cos^2 t, and leave in the lighter state with probability 1 - P_c(cos^2 t).
    The mixing angle is large, so the check is exact, not the Landau-Zener
    limit.  Any error in the sign of the exponent or in the scale height moves
    these numbers; the density normalisation (Y_e n_b0, the offset R) does not
    enter P_c and is pinned by the adiabatic-track test below."""
    th, h_ns, Ye = 0.3, 3.0, 0.5
    p = _msw(I.MATTER_EXP, th, 8, h_ns=h_ns, Ye=Ye)
    E, u, phi, Hv = orc.tables(p)
    Delta = orc.vac_coeff() * p.dm2[0] / E
    A0 = 1e4 * Delta.max()                     # at r = R: far above every resonance
    p = p.replace(nb0=A0 / (orc.matter_coeff() * Ye))
    r0 = p.R_nu
    r1 = r0 + h_ns * math.log(A0 / (1e-5 * Delta.min()))   # A(r1) << Delta sin 2t
    out, st, _ = orc.evolve(p, _pure_nu_e(orc, p), r0, (r1 - r0) / 4000, 4000)
    assert st == 0
    P1 = _populations(orc, out, p, _mass_basis_nu1(p))
    x = 2 * math.pi * Delta * h_ns

    def pc(s2):
        return (np.exp(-x * s2) - np.exp(-x)) / (1 - np.exp(-x))

    assert 0.2 < P1[0].min() and P1[0].max() < 0.8           # the hop is neither 0 nor 1
    assert np.abs(P1[0] - pc(math.sin(th) ** 2)).max() < 5e-5
    assert np.abs(P1[1] - (1 - pc(math.cos(th) ** 2))).max() < 5e-5


def test_power_law_profile_landau_zener(orc):
    """Eq. 3.7 with the r^-3 profile of Eq. 4.3 (the three-flavor workload's
    matter): at small mixing the hop probability across the resonance is the
    Landau-Zener value exp(-pi gamma / 2), gamma = Delta sin^2 2t / (cos 2t
    |d ln A / dr|) = Delta sin^2 2t r_res / (3 cos 2t), with r_res where
    A(r_res) = Delta cos 2t.  For a power-law profile the exact result differs
    from this limit by a relative O(tan^2 t) in the exponent (Kuo &
    Pantaleone 1989), about 2e-3 here, which bounds the tolerance.  The
    energies span gamma = 0.56 ... 1.8, so the profile's direction, exponent
    and normalisation each shift the answer by far more than that."""
    th = 0.03
    p = _msw(I.MATTER_POWER, th, 8, r_ref=10.0, ne_power=3.0)
    E, u, phi, Hv = orc.tables(p)
    Delta = orc.vac_coeff() * p.dm2[0] / E
    C = orc.matter_coeff()
    s2, c2 = math.sin(2 * th), math.cos(2 * th)
    Dmid = math.sqrt(Delta.max() * Delta.min())
    rres_mid = 3 * c2 / (Dmid * s2 * s2)        # gamma = 1 at the middle energy
    ne_ref = Dmid * c2 / C * (rres_mid / p.r_ref) ** 3
    p = p.replace(ne_ref=ne_ref)

    def radius(A):                              # where C ne_ref (r_ref / r)^3 = A
        return p.r_ref * (C * ne_ref / A) ** (1 / 3)

    rres = radius(Delta * c2)
    gamma = Delta * s2 * s2 * rres / (3 * c2)
    rho = _pure_nu_e(orc, p)
    # from A = 100 Delta_max to A = 1e-4 Delta_min, steps growing with r
    rs = np.geomspace(radius(100 * Delta.max()), radius(1e-4 * Delta.min()), 21)
    for a, b in zip(rs[:-1], rs[1:]):
        rho, st, _ = orc.evolve(p, rho, a, (b - a) / 1000, 1000)
        assert st == 0
    P1 = _populations(orc, rho, p, _mass_basis_nu1(p))
    lz = np.exp(-math.pi / 2 * gamma)
    assert 0.5 < gamma.min() and gamma.max() < 2
    assert np.abs(P1[0] - lz).max() < 1.5e-3
    # no resonance for antineutrinos (-A): they stay in the lighter state
    assert np.abs(P1[1] - 1).max() < 1e-4


@pytest.mark.parametrize("profile", ["exp", "power"])
def test_matter_profile_adiabatic_track(orc, profile):
    """Adiabatic MSW (Mikheyev-Smirnov): with a slowly varying profile
    (gamma ~ 130 at resonance) the state keeps its population in each local
    matter eigenstate of H = H_vac + A diag(1, 0) (Eq. 3.5, 3.7), neutrino
    and antineutrino (-A) alike, to O(1/gamma^2).  The eigenstates are taken
    at the density the paper's profile gives at three radii around the
    resonance (A = 3, 1, 1/3 Delta cos 2t at the middle energy).  A wrong
    density there (a dropped Y_e, a missing offset R in Eq. 4.4, a wrong
    n_ref or exponent in Eq. 4.3) turns the basis by up to the full mixing
    and moves the population by far more than the tolerance."""
    th = 0.3
    c2 = math.cos(2 * th)
    p = _msw(I.MATTER_NONE, th, 4, E=(10.0, 30.0))
    E, u, phi, Hv = orc.tables(p)
    Delta = orc.vac_coeff() * p.dm2[0] / E
    Dmid = math.sqrt(Delta.max() * Delta.min())
    C = orc.matter_coeff()
    if profile == "exp":
        Ye, h_ns = 0.5, 1000.0
        nb0 = Dmid * c2 / (C * Ye) * math.exp(5.0)      # resonance at R + 5 h_NS
        p = p.replace(matter=I.MATTER_EXP, Ye=Ye, nb0=nb0, h_ns=h_ns)

        def A(r):
            return C * Ye * nb0 * math.exp(-(r - p.R_nu) / h_ns)
        rres = p.R_nu + 5 * h_ns
        radii = [rres - h_ns * math.log(k) for k in (30.0, 3.0, 1.0, 1 / 3)]
    else:
        rres = 3000.0
        ne_ref = Dmid * c2 / C * (rres / 10.0) ** 3
        p = p.replace(matter=I.MATTER_POWER, ne_ref=ne_ref, r_ref=10.0, ne_power=3.0)

        def A(r):
            return C * ne_ref * (10.0 / r) ** 3
        radii = [rres / k ** (1 / 3) for k in (30.0, 3.0, 1.0, 1 / 3)]

    def local_states(r):
        v = np.zeros((2, p.n_E, 2))
        for s, sgn in ((0, 1.0), (1, -1.0)):
            for e in range(p.n_E):
                H = Delta[e] / 2 * np.array([[-c2, math.sin(2 * th)], [math.sin(2 * th), c2]])
                H[0, 0] += sgn * A(r)
                w, V = np.linalg.eigh(H)
                v[s, e] = V[:, 1] if sgn > 0 else V[:, 0]   # where nu_e / nubar_e start
        return v

    rho = _pure_nu_e(orc, p)
    start = _populations(orc, rho, p, local_states(radii[0]))
    assert start.min() > 0.999
    for a, b in zip(radii[:-1], radii[1:]):
        rho, st, _ = orc.evolve(p, rho, a, (b - a) / 5000, 5000)
        assert st == 0
        pop = _populations(orc, rho, p, local_states(b))
        assert np.abs(pop - start).max() < 5e-4
    # the neutrinos did cross the resonance: their electron content changed
    Pee = orc.unpack(rho, 2).reshape(2, p.n_E, 2, 2)[0, :, 0, 0].real
    assert Pee.max() < 0.7


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 5e-8), (I.EXPH, 1e-11)])
def test_vacuum_three_flavor(orc, stepper, tol):
    """P3: three-flavor vacuum oscillation (textbook, delta_CP = 0):
    P_ab = delta_ab - 4 sum_{j<k} U_aj U_bj U_ak U_bk sin^2(dm2_kj L / 4E)."""
    p = _small(n_f=3, n_E=10, n_u=3, stepper=stepper, eps=0.0, dm2=(7.5e-5, 2.4e-3),
               theta=(0.59, 0.15, 0.72), hierarchy=+1, E_min=2.0, E_max=10.0, r0=20.0,
               r1=30.0, n_steps=4000)
    E, u, phi, Hv = orc.tables(p)
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    M = orc.unpack(out, 3).reshape(2, p.n_u, p.n_E, 3, 3)
    s12, c12 = math.sin(0.59), math.cos(0.59)
    s13, c13 = math.sin(0.15), math.cos(0.15)
    s23, c23 = math.sin(0.72), math.cos(0.72)
    U = np.array([[c12 * c13, s12 * c13, s13],
                  [-s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13],
                  [s12 * s23 - c12 * c23 * s13, -c12 * s23 - s12 * c23 * s13, c23 * c13]])
    m2 = np.array([0.0, 7.5e-5, 2.4e-3])
    K = orc.vac_coeff()
    Lj = _path_length(p, p.r1)
    for beta in (0, 1):  # nu_e -> nu_e and nu_e -> nu_mu
        P = np.full((p.n_u, p.n_E), 1.0 if beta == 0 else 0.0)
        for j in range(3):
            for k in range(j + 1, 3):
                ph = np.outer(Lj, K * (m2[k] - m2[j]) / E) / 2
                P -= 4 * U[0, j] * U[beta, j] * U[0, k] * U[beta, k] * np.sin(ph) ** 2
        want = phi[2] + (phi[0] - phi[2]) * P
        assert np.abs(M[0, :, :, beta, beta].real - want).max() < tol * phi[0].max()


def test_bulb_moments_isotropic_closed_form(orc):
    """Eq. 3.13-3.15 for an angle-independent state: sum_u of the weights
    gives M0 = dE S (1 - sqrt(1 - x^2)), M1 = dE S x^2 / 2, so that the bulb
    potential of a radial trajectory, G(cos=1) = mu dE S (M0 - M1)/(dE S),
    equals the single-angle factor D(r/R) of Eq. 3.17."""
    p = _small(n_E=3, n_u=20000, eps=1e-2)
    rho = orc.init_state(p).reshape(2, p.n_u, p.n_E, 4)
    rho[:, :, :, :] = rho[:, :1, :, :]  # same state on every trajectory
    for r in (12.0, 30.0, 50.0):
        x = p.R_nu / r
        M0, M1 = orc.moments(p, rho.reshape(-1), r)
        E, u, phi, Hv = orc.tables(p)
        dE = E[1] - E[0]
        d = rho[0, 0] - rho[1, 0] * np.array([1, 1, 1, -1])  # rho_nu - conj(rho_nubar), packed
        S = d.sum(0)
        f0 = 1 - math.sqrt(1 - x * x)
        assert np.allclose(M0, dE * S * f0, rtol=2e-5 if r > 12 else 1e-2)
        assert np.allclose(M1, dE * S * x * x / 2, rtol=1e-9)
        D = 0.5 * (1 - math.sqrt(1 - x * x)) ** 2
        assert f0 - x * x / 2 == pytest.approx(D, rel=1e-12)


# ---------------------------------------------------------------- nu-nu coupling's radial dependence

def _precession(orc, geometry, stepper, n_chunks=40, steps_per_chunk=50, mu0=400.0, r0=20.0, r1=24.0):
    """One trajectory (n_u = 1, u = 1/2), three energies, no vacuum or matter
    term, antineutrinos empty: S = sum_E rho_nu is conserved and every bin
    precesses about it.  Returns the accumulated rotation angle of each bin's
    Bloch vector about S (chunks short enough to unwrap), the drift of S, and
    the quantities the closed forms need."""
    p = _small(n_E=3, n_u=1, geometry=geometry, stepper=stepper, mu0=mu0, eps=0.0,
               dm2=(0.0, 0.0), hierarchy=+1, E_min=10.0, E_max=13.0, R_nu=10.0)
    rng = np.random.default_rng(3)
    rho = np.zeros((2, p.n_E, 4))
    for e in range(p.n_E):
        v = rng.normal(size=3)
        v *= 0.4 / np.linalg.norm(v)
        rho[0, e] = [0.5 + v[2] / 2, 0.5 - v[2] / 2, v[0] / 2, -v[1] / 2]
    rho = rho.reshape(-1)

    def bloch(x):
        M = orc.unpack(x, 2).reshape(2, p.n_E, 2, 2)[0]
        return np.stack([2 * M[:, 0, 1].real, -2 * M[:, 0, 1].imag, (M[:, 0, 0] - M[:, 1, 1]).real], 1)

    P = bloch(rho)
    S0 = P.sum(0)
    n = S0 / np.linalg.norm(S0)
    total = np.zeros(p.n_E)
    h = (r1 - r0) / (n_chunks * steps_per_chunk)
    r = r0
    for _ in range(n_chunks):
        rho, st, _ = orc.evolve(p, rho, r, h, steps_per_chunk)
        assert st == 0
        r += h * steps_per_chunk
        Q = bloch(rho)
        for e in range(p.n_E):
            a = P[e] - (P[e] @ n) * n
            b = Q[e] - (Q[e] @ n) * n
            total[e] += math.atan2(np.cross(a, b) @ n, a @ b)
        P = Q
    dE = (p.E_max - p.E_min) / p.n_E
    return total, np.linalg.norm(P.sum(0) - S0), dict(mu0=mu0, dE=dE, sig=np.linalg.norm(S0), u=0.5,
                                                      R=p.R_nu, y0=p.R_nu / r0, y1=p.R_nu / r1)


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 1e-6), (I.EXPH, 1e-3)])
def test_literal_mu_r4_coupling_precession_closed_form(orc, stepper, tol):
    """The literal coupling mode (r-independent weights du, du cos, and
    mu = mu0 (R/r)^4): with one trajectory G = mu0 x^4 dE (1 - cos^2) S and
    1 - cos^2 = x^2 u (Eq. 3.14), so the Bloch vectors turn about S at
    mu0 dE |S| u x^6 / cos per unit radius (dl/dr = 1/cos, Eq. 3.3).  With
    y = R/r and y = sin(t)/sqrt(u):
        angle = mu0 dE |S| u R u^(-5/2) [3t/8 - sin 2t/4 + sin 4t/32] between
    the end points.  A wrong power of x in the coupling changes the angle
    several-fold."""
    ang, dS, q = _precession(orc, I.MU_R4, stepper)

    def F(y):
        t = math.asin(math.sqrt(q["u"]) * y)
        return (3 * t / 8 - math.sin(2 * t) / 4 + math.sin(4 * t) / 32) * q["u"] ** -2.5

    want = q["mu0"] * q["dE"] * q["sig"] * q["u"] * q["R"] * (F(q["y0"]) - F(q["y1"]))
    assert 3 < abs(want) < 30
    assert dS < 1e-12
    assert np.abs(np.abs(ang) - want).max() < tol * want


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 1e-6), (I.EXPH, 1e-3)])
def test_bulb_coupling_precession_closed_form(orc, stepper, tol):
    """The bulb geometry (Eq. 3.13-3.15) on one trajectory: the weights
    x^2 du / (2 cos), x^2 du / 2 give G = mu0 dE (x^2 u / (2 cos)) (1 - cos^2) S
    and, with dl/dr = 1/cos, a precession rate mu0 dE |S| u x^4 / (2 (1 - u x^2));
    with y = R/r the angle is mu0 dE |S| u R / 2 [(atanh(sqrt(u) y)/sqrt(u) - y)/u]
    between the end points."""
    ang, dS, q = _precession(orc, I.BULB, stepper)

    def G(y):
        su = math.sqrt(q["u"])
        return (math.atanh(su * y) / su - y) / q["u"]

    want = q["mu0"] * q["dE"] * q["sig"] * q["u"] / 2 * q["R"] * (G(q["y0"]) - G(q["y1"]))
    assert 3 < abs(want) < 30
    assert dS < 1e-12
    assert np.abs(np.abs(ang) - want).max() < tol * want


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
@pytest.mark.parametrize("n_f", [2, 3])
def test_trace_conserved(orc, stepper, n_f):
    """P4: d(tr rho)/dr = tr(-i[H, rho]) = 0 for every bin."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72)) if n_f == 3 else {}
    p = _small(n_f=n_f, stepper=stepper, mu0=1e5, r0=50.0, r1=51.0, n_steps=100, **kw)
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    t0, t1 = _trace(rho, n_f), _trace(out, n_f)
    assert np.abs(t1 - t0).max() < 1e-13 * np.abs(t0).max()


def _purity_like(rho, n_f):
    M = orc_unpack_cache(rho, n_f)
    t = np.trace(M, axis1=1, axis2=2).real
    M0 = M - t[:, None, None] / n_f * np.eye(n_f)
    return np.einsum("bij,bji->b", M0, M0).real


def orc_unpack_cache(rho, n_f):
    import oracle as O
    return O.unpack(rho, n_f)


@pytest.mark.parametrize("stepper,n_steps,tol", [(I.RK4, 200, 1e-6), (I.EXPH, 800, 1e-5)])
def test_polarization_length_drift_small(orc, stepper, n_steps, tol):
    """P4: tr(rho0^2) of the traceless part (|P|^2 / 2 in two flavors) is
    conserved by the exact flow; the integrators keep it to their truncation
    order.  Pins that the update is a commutator (a wrong sign or a dropped
    term changes it at first order)."""
    p = _small(stepper=stepper, mu0=1e5, r0=50.0, r1=52.0, n_steps=n_steps, eps=1e-2)
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    a, b = _purity_like(rho, 2), _purity_like(out, 2)
    assert np.abs(b - a).max() < tol * np.abs(a).max()


def _lepton_invariants(orc, p, rho):
    """I_k = tr(Pi_k F), F = sum_{u,e} du (rho_nu - conj rho_nubar), Pi_k the
    vacuum mass-basis projectors."""
    n = p.n_f
    M = orc.unpack(rho, n).reshape(2, p.n_u, p.n_E, n, n)
    F = (M[0] - M[1].conj()).sum(axis=(0, 1)) / p.n_u
    E, u, phi, Hv = orc.tables(p)
    Hv0 = orc.unpack(Hv[:1].reshape(-1), n)[0]
    w, V = np.linalg.eigh(Hv0)
    return np.array([(V[:, k].conj() @ F @ V[:, k]).real for k in range(n)]), np.abs(F).max()


@pytest.mark.parametrize("geometry", [I.BULB, I.SINGLE_ANGLE, I.CONST])
@pytest.mark.parametrize("n_f", [2, 3])
def test_lepton_number_moment_conserved(orc, geometry, n_f):
    """P5: with A = 0 the nu-nu terms cancel in d/dr tr(Pi_k F) because
    sum_u (du/c_u)[M0 - c_u M1, S_u] = [M0, M0] - [M1, M1] = 0 (Eq. 3.13-3.15);
    RK4 keeps this linear invariant to rounding."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72)) if n_f == 3 else {}
    n_u = 1 if geometry == I.SINGLE_ANGLE else 6
    mu0 = 100.0 if geometry == I.CONST else 3e4  # keep mu h inside RK4's stable region
    p = _small(n_f=n_f, n_u=n_u, geometry=geometry, mu0=mu0, r0=20.0, r1=22.0, n_steps=400,
               eps=1e-2, **kw)
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    assert st == 0
    I0, scale = _lepton_invariants(orc, p, rho)
    I1, _ = _lepton_invariants(orc, p, out)
    # the individual bins move at O(1): the invariant must not
    assert np.abs(orc.unpack(out, n_f) - orc.unpack(rho, n_f)).max() > 1e-4
    assert np.abs(I1 - I0).max() < 1e-12 * scale


def test_bipolar_energy_conserved(orc):
    """P7: isotropic gas (CONST mode, one angle, A = 0):
    E = sum_e tr(H_vac,e (rho + conj rho_bar)) + (mu dE / 2) tr(D^2),
    D = sum_e (rho - conj rho_bar), is conserved by the flow (derived from
    Eq. 3.4 and the antineutrino rule); RK4 keeps it to O(h^4)."""
    p = _small(n_E=5, n_u=1, geometry=I.CONST, mu0=50.0, eps=0.05, r0=0.0 + 20, r1=25.0,
               n_steps=2000, E_min=5.0, E_max=20.0)
    E, u, phi, Hv = orc.tables(p)
    Hvm = orc.unpack(Hv.reshape(-1), 2)
    dE = E[1] - E[0]

    def energy(rho):
        M = orc.unpack(rho, 2).reshape(2, p.n_E, 2, 2)
        S = M[0] + M[1].conj()
        D = (M[0] - M[1].conj()).sum(0)
        return (np.einsum("eij,eji->", Hvm, S).real + p.mu0 * dE / 2 * np.trace(D @ D).real)

    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    moved = np.abs(orc.unpack(out, 2) - orc.unpack(rho, 2)).max()
    assert moved > 1e-2
    assert abs(energy(out) - energy(rho)) < 1e-9 * abs(energy(rho))


def test_bipolar_instability_only_in_inverted_hierarchy(orc):
    """Sign of the nu-nu term relative to H_vac: in an isotropic gas with a
    nu_e excess and mu of the order of the vacuum frequency, the bipolar
    (pendulum) mode is unstable for the inverted hierarchy only (Hannestad,
    Raffelt, Sigl, Wong 2006; Duan, Fuller, Carlson, Qian 2006): rho_ee moves
    at O(10%) in IH and only at the vacuum amplitude sin^2(2 theta) in NH."""
    def max_change(hier):
        p = _small(n_E=1, n_u=1, geometry=I.CONST, mu0=20.0, eps=1e-6, theta=(0.01, 0, 0),
                   hierarchy=hier, E_min=9.0, E_max=11.0, r0=20.0, r1=120.0, n_steps=20000)
        rho = orc.init_state(p)
        ee0 = orc.unpack(rho, 2)[:, 0, 0].real
        r, worst = p.r0, 0.0
        for _ in range(20):
            rho, st, _ = orc.evolve(p, rho, r, p.h, 1000)
            r += 1000 * p.h
            worst = max(worst, np.abs(orc.unpack(rho, 2)[:, 0, 0].real - ee0).max() / ee0[0])
        return worst
    assert max_change(-1) > 0.1
    assert max_change(+1) < 2 * math.sin(0.02) ** 2


def test_nu_nubar_symmetric_in_vacuum(orc):
    """P9: with A = mu = 0 the antineutrino Hamiltonian equals H_vac (after
    Eq. 3.4), so equal initial states stay equal."""
    p = _small(mu0=0.0, eps=1e-2, r0=20.0, r1=30.0, n_steps=300)
    rho = orc.init_state(p).reshape(2, -1)
    rho[1] = rho[0]
    for stepper in (I.RK4, I.EXPH):
        out, st, _ = orc.evolve(p.replace(stepper=stepper), rho.reshape(-1), p.r0, p.h, p.n_steps)
        out = out.reshape(2, -1)
        assert np.array_equal(out[0], out[1])


# ---------------------------------------------------------------- independent SA integrator

def _sa_bloch_rk4(orc, p, rho):
    """Single-angle model (Eq. 3.16-3.17) written independently in
    polarization-vector form: rho = (P0 + P.sigma)/2, H = (h0 + h.sigma)/2,
    dP/dr = h x P.  h_vac = Delta (sin2t, 0, -cos2t) (Eq. 3.5), matter
    (0, 0, A) (Eq. 3.7), nu-nu mu D(x) dE sum_e (P - P_bar*), with
    P* = (Px, -Py, Pz) the Bloch vector of the complex conjugate."""
    E, u, phi, Hv = orc.tables(p)
    dE = E[1] - E[0]
    Delta = orc.vac_coeff() * p.hierarchy * p.dm2[0] / E
    th = p.theta[0]
    hv = np.stack([Delta * math.sin(2 * th), 0 * Delta, -Delta * math.cos(2 * th)], 1)
    x = rho.reshape(2, p.n_E, 4)
    P = np.stack([2 * x[:, :, 2], -2 * x[:, :, 3], x[:, :, 0] - x[:, :, 1]], 2)  # [s][e][3]
    P0 = x[:, :, 0] + x[:, :, 1]
    cj = np.array([1.0, -1.0, 1.0])

    def f(r, P):
        xx = p.R_nu / r
        mu = p.mu0 * 0.5 * (1 - math.sqrt(1 - xx * xx)) ** 2
        hG = mu * dE * (P[0] - P[1] * cj).sum(0)
        h_nu = hv + hG
        h_nb = hv - hG * cj
        return np.stack([np.cross(h_nu, P[0]), np.cross(h_nb, P[1])])

    h = p.h
    for n in range(p.n_steps):
        r = p.r0 + n * h
        k1 = f(r, P)
        k2 = f(r + h / 2, P + h / 2 * k1)
        k3 = f(r + h / 2, P + h / 2 * k2)
        k4 = f(r + h, P + h * k3)
        P = P + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    out = np.stack([(P0 + P[:, :, 2]) / 2, (P0 - P[:, :, 2]) / 2, P[:, :, 0] / 2, -P[:, :, 1] / 2], 2)
    return out.reshape(-1)


def test_single_angle_matches_bloch_brute_force(orc):
    """P6: the oracle's multi-angle integrator in single-angle mode with one
    angle bin equals an independently written Bloch-vector integrator."""
    p = _small(n_E=9, n_u=1, geometry=I.SINGLE_ANGLE, mu0=1e5, eps=1e-2, r0=40.0, r1=42.0,
               n_steps=400)
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    assert st == 0
    ref = _sa_bloch_rk4(orc, p, rho)
    assert np.abs(orc.unpack(out, 2) - orc.unpack(rho, 2)).max() > 1e-3
    assert np.abs(out - ref).max() < 1e-12 * np.abs(rho).max()


# ---------------------------------------------------------------- convergence

def test_convergence_orders(orc):
    """P8: halving h cuts the RK4 error ~16x and the predictor-corrector
    error ~4x (second order, Sec. 4.2.3)."""
    base = _small(n_E=6, n_u=4, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0)
    rho = orc.init_state(base)
    ref, _, _ = orc.evolve(base, rho, 50.0, 1.0 / 3200, 3200)

    def err(stepper, n):
        out, _, _ = orc.evolve(base.replace(stepper=stepper), rho, 50.0, 1.0 / n, n)
        return np.abs(out - ref).max()

    e = [err(I.RK4, n) for n in (25, 50, 100)]
    assert 12 < e[0] / e[1] < 20 and 12 < e[1] / e[2] < 20
    e = [err(I.EXPH, n) for n in (50, 100, 200)]
    assert 3.2 < e[0] / e[1] < 4.8 and 3.2 < e[1] / e[2] < 4.8


# ---------------------------------------------------------------- state / status

def test_initial_state_structure(orc):
    """Seeded start: flavor-diagonal phi_a(E) with |rho_ij| = eps sqrt(rho_ii rho_jj)."""
    p = _small(n_f=3, eps=1e-6, seed=3)
    rho = orc.init_state(p)
    M = orc.unpack(rho, 3).reshape(2, p.n_u, p.n_E, 3, 3)
    E, u, phi, Hv = orc.tables(p)
    assert np.allclose(M[0, :, :, 0, 0].real, phi[0][None])
    assert np.allclose(M[1, :, :, 2, 2].real, phi[3][None])
    amp = np.abs(M[0, :, :, 0, 1])
    assert np.allclose(amp, 1e-6 * np.sqrt(phi[0] * phi[2])[None], rtol=1e-12)
    ph = np.angle(M[:, :, :, 0, 1]).ravel()
    assert ph.std() > 1.0  # phases spread over the circle
    assert not np.array_equal(orc.init_state(p.replace(seed=4)), rho)


def test_literal_rk4_config_reports_nonfinite(orc):
    """Explicit RK4 at h = 0.095 km from 10 km (mu0 = 1e5) is far outside its
    stability region; the oracle reports it and keeps the last finite state."""
    p = I.bulb2f_16x32().replace(stepper=I.RK4)
    rho = orc.init_state(p)
    out, st, done = orc.evolve(p, rho, p.r0, p.h, 400)
    assert st == 1 and done < 400
    assert np.isfinite(out).all()


def test_literal_mu_r4_breaks_lepton_number(orc):
    """The literal reading (r-independent angle weights, mu0 (R/r)^4) loses the
    cancellation of P5: its weights lack the 1/cos factor of Eq. 3.15 that
    matches the path factor dl/dr = 1/cos of Eq. 3.3.  This is why the bulb
    geometry is the default mode."""
    p = _small(n_u=6, geometry=I.MU_R4, mu0=3e4, r0=20.0, r1=22.0, n_steps=400, eps=1e-2)
    rho = orc.init_state(p)
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    I0, scale = _lepton_invariants(orc, p, rho)
    I1, _ = _lepton_invariants(orc, p, out)
    assert np.abs(I1 - I0).max() > 1e-6 * scale


# ---------------------------------------------------------------- renormalised method

@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
@pytest.mark.parametrize("n_f", [2, 3])
def test_renormalised_method_keeps_purity_and_trace(orc, stepper, n_f):
    """The renormalised method holds each bin's tr(T^2) (a constant of the
    exact flow, Eq. 3.10) and its trace, in a regime where the plain method
    visibly loses tr(T^2) (strong coupling, coarse step)."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72)) if n_f == 3 else {}
    p = _small(n_f=n_f, stepper=stepper, mu0=3e4, eps=1e-2, r0=50.0, r1=52.0, n_steps=100, **kw)
    rho = orc.init_state(p)
    plain, st0, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    ren, st1, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps, renorm=True)
    assert st0 == 0 and st1 == 0
    q0, qp, qr = _purity_like(rho, n_f), _purity_like(plain, n_f), _purity_like(ren, n_f)
    assert np.abs(qp / q0 - 1).max() > 1e-6      # the plain method drifts here
    assert np.abs(qr / q0 - 1).max() < 1e-13     # the renormalised one does not
    assert np.abs(_trace(ren, n_f) - _trace(rho, n_f)).max() < 1e-13 * np.abs(_trace(rho, n_f)).max()


def test_renormalised_method_is_exact_in_vacuum(orc):
    """In vacuum the predictor-corrector is exact (P1), so it keeps tr(T^2) by
    itself and the renormalisation must not change anything; the result is
    the textbook survival probability."""
    p = _small(n_E=12, n_u=5, stepper=I.EXPH, eps=0.0, theta=(0.3, 0, 0), hierarchy=-1,
               E_min=1.0, E_max=13.0, r0=20.0, r1=30.0, n_steps=1000)
    rho = orc.init_state(p)
    plain, _, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    ren, _, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps, renorm=True)
    assert np.abs(ren - plain).max() < 1e-13 * np.abs(plain).max()


def test_renormalised_rk4_converges_to_the_same_flow(orc):
    """On an oscillation RK4's amplification factor has modulus
    sqrt(1 - z^6/72 + ...) (z = lambda h), so plain RK4 loses tr(T^2) by
    O(h^6) per step, O(h^5) over a fixed interval; the renormalisation
    removes just that, so halving h shrinks the plain-vs-renormalised gap
    about 32x and both approach the same exact flow.  A renormalisation that
    rescaled anything but the traceless part would leave an O(1) gap."""
    base = _small(n_E=6, n_u=4, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0)
    rho = orc.init_state(base)

    def gap(n):
        a, _, _ = orc.evolve(base, rho, 50.0, 1.0 / n, n)
        b, _, _ = orc.evolve(base, rho, 50.0, 1.0 / n, n, renorm=True)
        return np.abs(a - b).max()

    g = [gap(n) for n in (25, 50, 100)]
    assert 26 < g[0] / g[1] < 38 and 26 < g[1] / g[2] < 38


# ---------------------------------------------------------------- error-controlled step

def test_adaptive_error_estimate_scales_as_h_squared(orc):
    """The coarse path of an attempt is the second-order predictor-corrector;
    the fine path (two exponential half steps averaged with a full step under
    the end-point Hamiltonian) is first order, so their difference, the
    error estimate, falls 4x per halving of h.  This fixes the exponent 1/2
    of the step-size update."""
    p = _small(stepper=I.EXPH, mu0=1e5, eps=1e-2, n_E=6, n_u=4)
    rho = orc.init_state(p)
    e = [orc.attempt_adaptive(p, rho, 50.0, h)[2] for h in (0.02, 0.01, 0.005)]
    assert 3.6 < e[0] / e[1] < 4.6 and 3.6 < e[1] / e[2] < 4.6


def test_adaptive_coarse_result_is_the_fixed_step(orc):
    """With a tolerance no attempt can miss and h0 = dr_max, every attempt is
    accepted at the same h, and the result is the fixed-step
    predictor-corrector (pinned against the textbook cases P1-P3)."""
    p = _small(stepper=I.EXPH, mu0=1e5, eps=1e-2, n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72),
               matter=I.MATTER_POWER, ne_ref=1e31, eps0=1e300, dr_max=0.01, r0=50.0, r1=50.5, n_steps=50)
    rho = orc.init_state(p)
    fixed, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    out, st, r, h, na, nr = orc.evolve_adaptive(p, rho, p.r0, p.r1, p.h)
    assert st == 0 and r == p.r1 and nr == 0 and na == p.n_steps
    assert np.abs(out - fixed).max() < 1e-13 * np.abs(fixed).max()


def test_adaptive_is_exact_in_vacuum(orc):
    """In vacuum both paths are exact (the propagator composes along the
    trajectory), the error estimate is rounding, every step is dr_max and the
    result is the textbook two-flavor survival probability (P1)."""
    p = _small(n_E=12, n_u=5, stepper=I.EXPH, eps=0.0, theta=(0.3, 0, 0), hierarchy=-1,
               E_min=1.0, E_max=13.0, r0=20.0, r1=30.0, eps0=1e-10, dr_max=0.25)
    E, u, phi, Hv = orc.tables(p)
    rho = orc.init_state(p)
    out, st, r, h, na, nr = orc.evolve_adaptive(p, rho, p.r0, p.r1, 0.01)
    assert st == 0 and r == p.r1 and nr == 0
    assert na <= 2 + int(np.ceil((p.r1 - p.r0) / p.dr_max))  # one short start, then dr_max
    M = orc.unpack(out, 2).reshape(2, p.n_u, p.n_E, 2, 2)
    Lj = _path_length(p, p.r1)
    Delta = orc.vac_coeff() * p.hierarchy * p.dm2[0] / E
    Pee = 1 - np.sin(2 * 0.3) ** 2 * np.sin(np.outer(Lj, Delta) / 2) ** 2
    for s, (ie, ix) in enumerate([(0, 2), (1, 3)]):
        want = phi[ix] + (phi[ie] - phi[ix]) * Pee
        assert np.abs(M[s, :, :, 0, 0].real - want).max() < 1e-11 * phi[0].max()


def test_adaptive_converges_with_tolerance(orc):
    """Single-angle model against the independent Bloch-vector integrator
    (P6, at a step far below any adaptive one): tightening eps0 tightens the
    result, the step sequence adapts (some attempts rejected from a large
    h0), and the run ends exactly on r_end."""
    p = _small(n_E=9, n_u=1, geometry=I.SINGLE_ANGLE, stepper=I.EXPH, mu0=1e5, eps=1e-2, r0=40.0,
               r1=42.0, n_steps=4000, dr_max=0.5)
    rho = orc.init_state(p)
    ref = _sa_bloch_rk4(orc, p, rho)
    errs = []
    for eps0 in (1e-4, 1e-5, 1e-6):
        out, st, r, h, na, nr = orc.evolve_adaptive(p.replace(eps0=eps0), rho, p.r0, p.r1, 0.5)
        assert st == 0 and r == p.r1 and nr >= 1
        errs.append(np.abs(out - ref).max() / np.abs(rho).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


def test_adaptive_budget_and_status(orc):
    p = _small(stepper=I.EXPH, mu0=1e5, eps=1e-2, eps0=1e-8, dr_max=0.1)
    rho = orc.init_state(p)
    out, st, r, h, na, nr = orc.evolve_adaptive(p, rho, 50.0, 60.0, 0.1, max_iters=3)
    assert st == 2 and na + nr == 3 and 50.0 <= r < 60.0


# ---------------------------------------------------------------- extended bulb (Eq. 3.18)

def _maa(**kw):
    base = dict(n_E=6, n_u=5, n_phi=6, n_f=2, stepper=I.EXPH, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0,
                n_steps=100, seed=9)
    base.update(kw)
    return I.Problem(**base)


def _replicate_over_azimuths(rho_ma, p):
    x = rho_ma.reshape(2, p.n_u, 1, p.n_E, -1)
    return np.ascontiguousarray(np.broadcast_to(x, (2, p.n_u, p.n_phi, p.n_E, x.shape[-1]))).reshape(-1)


@pytest.mark.parametrize("n_f,stepper", [(2, I.EXPH), (2, I.RK4), (3, I.EXPH)])
def test_extended_bulb_with_symmetric_azimuths_is_the_bulb(orc, n_f, stepper):
    """Integrating 1 - cos(gamma) over the azimuth of an azimuthally symmetric
    state leaves the bulb model's 1 - cos(th) cos(th') (Eq. 3.18 -> 3.13): a
    state equal in every azimuth bin evolves exactly like the bulb model, in
    every bin, and its azimuthal moments M2, M3 vanish."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1, mu0=1e4) if n_f == 3 else {}
    p = _maa(n_f=n_f, stepper=stepper, **kw)
    ma = p.replace(n_phi=1)
    rho_ma = orc.init_state(ma)
    rho = _replicate_over_azimuths(rho_ma, p)
    M = orc.moments_ex(p, rho, p.r0)
    M_ma = orc.moments_ex(ma, rho_ma, p.r0)
    scale = np.abs(M[0]).max()
    assert np.abs(M[2:]).max() < 1e-15 * scale
    assert np.abs(M[:2] - M_ma[:2]).max() < 1e-14 * scale
    out, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    out_ma, st_ma, _ = orc.evolve(ma, rho_ma, p.r0, p.h, p.n_steps)
    assert st == 0 and st_ma == 0
    assert np.abs(orc.unpack(out_ma, n_f) - orc.unpack(rho_ma, n_f)).max() > 1e-6  # it moved
    want = _replicate_over_azimuths(out_ma, p)
    assert np.abs(out - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("n_f", [2, 3])
def test_extended_bulb_is_azimuth_rotation_equivariant(orc, n_f):
    """The azimuth grid is uniform, so rotating every state by one azimuth bin
    and evolving equals evolving and then rotating (the moments M2, M3 rotate
    with the state and G follows): an inconsistent sign or weight between the
    cos(ph) / sin(ph) moments and their factors in G breaks it."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1, mu0=1e4) if n_f == 3 else {}
    p = _maa(n_f=n_f, n_phi=7, **kw)
    rho = orc.init_state(p)
    shape = (2, p.n_u, p.n_phi, p.n_E, n_f * n_f)
    shift = lambda x: np.roll(x.reshape(shape), 1, axis=2).reshape(-1)
    a, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    b, st2, _ = orc.evolve(p, shift(rho), p.r0, p.h, p.n_steps)
    assert st == 0 and st2 == 0
    assert np.abs(shift(a) - b).max() < 1e-12 * np.abs(a).max()
    # and the azimuthal structure matters: the unshifted result differs
    assert np.abs(shift(a) - a).max() > 1e-9 * np.abs(a).max()


def test_extended_bulb_moment_weights_give_the_trajectory_direction(orc):
    """With the difference nu - conj(nubar) carried by one trajectory (zenith u,
    azimuth ph) only, the moment ratios are that trajectory's unit direction
    (cos th, sin th cos ph, sin th sin ph) at radius r, with cos th from
    Eq. 3.14 and sin^2 + cos^2 = 1 (so 1 - cos(gamma) of Eq. 3.18 is one minus
    a dot product of unit vectors)."""
    p = _maa(n_phi=8, eps=0.0)
    r = 23.0
    rho = np.zeros(orc.state_size(p)).reshape(2, p.n_u, p.n_phi, p.n_E, 4)
    j, k = 3, 5
    rho[0, j, k, 2, 2] = 1.0  # Re rho_12 of one nu bin
    M = orc.moments_ex(p, rho.reshape(-1), r)
    u = (j + 0.5) / p.n_u
    x = p.R_nu / r
    cth = math.sqrt(1 - x * x * u)
    ph = (k + 0.5) * 2 * math.pi / p.n_phi
    n_hat = np.array([cth, math.sqrt(1 - cth * cth) * math.cos(ph), math.sqrt(1 - cth * cth) * math.sin(ph)])
    ratios = M[1:, 2] / M[0, 2]
    assert np.abs(ratios - n_hat).max() < 1e-14
    assert abs(np.linalg.norm(ratios) - 1.0) < 1e-14


# ---------------------------------------------------------------- wavefunction form

def _psi_norms(psi, n_f):
    v = psi.reshape(-1, n_f, n_f, 2)
    return (v ** 2).sum(axis=(2, 3))  # [bin][flavor]


@pytest.mark.parametrize("n_f", [2, 3])
def test_psi_initial_state_gives_a_physical_rho(orc, n_f):
    """rho = sum_a phi_a psi_a psi_a^+ of the seeded unit wavefunctions: trace
    phi_e + (n_f - 1) phi_x per bin, Hermitian and positive semidefinite,
    off-diagonal of order eps."""
    kw = dict(dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72)) if n_f == 3 else {}
    p = _small(n_f=n_f, eps=1e-3, **kw)
    psi = orc.init_psi(p)
    assert np.abs(_psi_norms(psi, n_f) - 1).max() < 1e-15
    rho = orc.psi_to_rho(p, psi)
    E, u, phi, Hv = orc.tables(p)
    M = orc.unpack(rho, n_f).reshape(2, p.n_u, p.n_E, n_f, n_f)
    for s, (ie, ix) in enumerate([(0, 2), (1, 3)]):
        tr = np.trace(M[s], axis1=-2, axis2=-1).real
        assert np.abs(tr - (phi[ie] + (n_f - 1) * phi[ix])).max() < 1e-14 * phi[0].max()
    w = np.linalg.eigvalsh(orc.unpack(rho, n_f))
    assert w.min() > -1e-15
    off = np.abs(orc.unpack(rho, n_f)[:, 0, 1])
    assert 1e-5 * phi.max() < off.max() < 3e-3 * phi.max()


def test_psi_form_is_exact_in_vacuum(orc):
    """P1 in the wavefunction form: the predictor and corrector rotations
    coincide in vacuum, so the average is the exact rotation."""
    p = _small(n_E=12, n_u=5, stepper=I.EXPH, eps=0.0, theta=(0.3, 0, 0), hierarchy=-1,
               E_min=1.0, E_max=13.0, r0=20.0, r1=30.0, n_steps=1000)
    E, u, phi, Hv = orc.tables(p)
    psi = orc.init_psi(p)
    out, st, done = orc.evolve_psi(p, psi, p.r0, p.h, p.n_steps)
    assert st == 0 and done == p.n_steps
    M = orc.unpack(orc.psi_to_rho(p, out), 2).reshape(2, p.n_u, p.n_E, 2, 2)
    Lj = _path_length(p, p.r1)
    Delta = orc.vac_coeff() * p.hierarchy * p.dm2[0] / E
    Pee = 1 - np.sin(2 * 0.3) ** 2 * np.sin(np.outer(Lj, Delta) / 2) ** 2
    for s, (ie, ix) in enumerate([(0, 2), (1, 3)]):
        want = phi[ix] + (phi[ie] - phi[ix]) * Pee
        assert np.abs(M[s, :, :, 0, 0].real - want).max() < 1e-11 * phi[0].max()


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 1e-7), (I.EXPH, 1e-11)])
def test_psi_amplitudes_in_vacuum(orc, stepper, tol):
    """The textbook two-flavor amplitudes (P1 before squaring): with the
    traceless H0 = (Delta/2)[[-cos 2theta, sin 2theta], [sin 2theta, cos 2theta]]
    (Eq. 3.5-3.6), U = exp(-i H0 L) = cos(Delta L/2) - i sin(Delta L/2) H0/(Delta/2),
    so psi_e(L) = (cos + i cos2theta sin, -i sin2theta sin) and psi_x(L) =
    (-i sin2theta sin, cos - i cos2theta sin).  Fixes the phase of every psi,
    which rho does not: a stepper that kept the trace of H would turn them."""
    th = 0.3
    p = _small(n_E=12, n_u=5, stepper=stepper, eps=0.0, theta=(th, 0, 0), hierarchy=-1,
               E_min=1.0, E_max=13.0, r0=20.0, r1=30.0, n_steps=1000)
    E, u, phi, Hv = orc.tables(p)
    out, st, done = orc.evolve_psi(p, orc.init_psi(p), p.r0, p.h, p.n_steps)
    assert st == 0 and done == p.n_steps
    psi = out.reshape(2, p.n_u, p.n_E, 2, 2, 2)
    psi = psi[..., 0] + 1j * psi[..., 1]  # [s][u][E][a][i]
    Delta = orc.vac_coeff() * p.hierarchy * p.dm2[0] / E
    ph = np.outer(_path_length(p, p.r1), Delta) / 2
    c2, s2 = np.cos(2 * th), np.sin(2 * th)
    want = np.empty((p.n_u, p.n_E, 2, 2), dtype=complex)
    want[..., 0, 0] = np.cos(ph) + 1j * c2 * np.sin(ph)
    want[..., 0, 1] = -1j * s2 * np.sin(ph)
    want[..., 1, 0] = -1j * s2 * np.sin(ph)
    want[..., 1, 1] = np.cos(ph) - 1j * c2 * np.sin(ph)
    for s in range(2):  # the vacuum term is the same for nu and nubar
        assert np.abs(psi[s] - want).max() < tol


@pytest.mark.parametrize("stepper,ratio", [(I.RK4, 16.0), (I.EXPH, 8.0)])
def test_psi_form_and_rho_form_converge_to_one_flow(orc, stepper, ratio):
    """Both forms integrate the same flow (rho = sum phi psi psi^+ evolves as
    U rho U^+), so from the same initial rho they converge together.  RK4:
    the gap is the methods' truncation error, ~16x smaller per halving of h.
    Predictor-corrector: averaging density matrices or wavefunctions differs
    per step by (1/4) phi (U0 psi - U1 psi)(U0 psi - U1 psi)^+ = O(h^4) (the
    two rotations differ by (H1 - H0) h = O(h^2)), O(h^3) over the run: ~8x."""
    base = _small(n_E=6, n_u=4, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0, stepper=stepper)
    psi = orc.init_psi(base)
    rho = orc.psi_to_rho(base, psi)

    def gap(n):
        a, st, _ = orc.evolve_psi(base, psi, 50.0, 1.0 / n, n)
        b, st2, _ = orc.evolve(base, rho, 50.0, 1.0 / n, n)
        assert st == 0 and st2 == 0
        return np.abs(orc.psi_to_rho(base, a) - b).max()

    g = [gap(n) for n in (50, 100, 200)]
    assert 0.7 * ratio < g[0] / g[1] < 1.4 * ratio and 0.7 * ratio < g[1] / g[2] < 1.4 * ratio


def test_psi_norms_under_the_two_steppers(orc):
    """RK4 keeps |psi| to its truncation order: O(h^5) per step from the change
    of H within the step, O(h^4) over the run (the z^6/72 loss on a pure
    oscillation is one order higher), so the drift falls 16-32x per halving of
    h, nearing 16 as h falls.  The averaged predictor-corrector shortens psi:
    |(U0 psi + U1 psi)/2|^2 = 1 - |U0 psi - U1 psi|^2/4 = 1 - O(h^4) per step,
    O(h^3) over the run, ~8x less per halving of h."""
    base = _small(n_E=6, n_u=4, mu0=1e5, eps=1e-2, r0=50.0, r1=51.0)
    psi = orc.init_psi(base)
    loss = []
    for n in (50, 100):
        a, _, _ = orc.evolve_psi(base.replace(stepper=I.EXPH), psi, 50.0, 1.0 / n, n)
        loss.append(np.abs(_psi_norms(a, 2) - 1).max())
    assert 6.0 < loss[0] / loss[1] < 10.0
    drift = []
    for n in (100, 200, 400):
        r, _, _ = orc.evolve_psi(base.replace(stepper=I.RK4), psi, 50.0, 1.0 / n, n)
        drift.append(np.abs(_psi_norms(r, 2) - 1).max())
    assert 14.0 < drift[1] / drift[2] < drift[0] / drift[1] < 34.0


# ------------------------------------------------------------ cylinder / line model (Sec. 3.2.5)

def _cyl(**kw):
    base = dict(n_E=6, n_u=8, n_phi=5, n_f=2, geometry=I.CYLINDER, stepper=I.EXPH, mu0=1e3, eps=1e-2,
                r0=20.0, r1=21.0, n_steps=50, seed=17)
    base.update(kw)
    return I.Problem(**base)


def _ray_point(R, r, lat, th):
    """Where the ray that leaves the circle of radius R at latitude `lat`, at
    angle `th` from the outward normal (positive clockwise), reaches radius r,
    and its direction there (plane geometry, written from scratch)."""
    e = R * np.array([np.cos(lat), np.sin(lat)])
    d = np.array([np.cos(lat - th), np.sin(lat - th)])
    s = -R * np.cos(th) + np.sqrt(r * r - (R * np.sin(th)) ** 2)
    return e + s * d, d


def test_cylinder_latitude_map_by_ray_tracing(orc):
    """Eq. 3.20's Phi' = Phi + theta' - theta + asin(x sin theta) - asin(x sin theta')
    is the latitude from which the background ray of angle theta' left to
    cross the point that the ray (Phi, theta) reaches at radius r, with theta
    measured clockwise from the outward normal; and 1 - cos(alpha - alpha') is
    one minus the dot product of the two rays' directions there.  Both
    checked against plane ray tracing."""
    p = _cyl(n_u=12)
    rng = np.random.default_rng(3)
    th = -np.pi / 2 + (np.arange(p.n_u) + 0.5) * np.pi / p.n_u
    for _ in range(40):
        r = p.R_nu * (1.0 + 4.0 * rng.random())
        j, jp = rng.integers(0, p.n_u, 2)
        lat = 2 * np.pi * rng.random()
        P, d = _ray_point(p.R_nu, r, lat, th[j])
        # the background ray from latitude 0, rotated onto the point P
        P0, d0 = _ray_point(p.R_nu, r, 0.0, th[jp])
        rot = np.arctan2(P[1], P[0]) - np.arctan2(P0[1], P0[0])
        dp = np.array([np.cos(rot) * d0[0] - np.sin(rot) * d0[1], np.sin(rot) * d0[0] + np.cos(rot) * d0[1]])
        shift, weight = orc.cyl_pair(p, r, int(j), int(jp))
        assert abs(np.angle(np.exp(1j * (rot - lat - shift)))) < 1e-12  # Phi' - Phi, mod 2 pi
        x = p.R_nu / r
        wc = np.cos(th[jp]) / np.sqrt(1 - (x * np.sin(th[jp])) ** 2) * np.pi / p.n_u
        assert weight == pytest.approx(wc * (1.0 - d @ dp), rel=1e-12, abs=1e-15)


def test_cylinder_weights_cover_the_visible_arc(orc):
    """For a state equal on every trajectory the moments are closed forms:
    sum_j cos(theta_j)/cos(alpha_j) dtheta -> int cos th / sqrt(1 - x^2 sin^2 th)
    dth = (2/x) asin(x) (so mu0 x M0 / S is the arc 2 asin(x) the cylinder
    fills in the sky of the point); the cos(alpha) moment -> int cos th dth = 2;
    the sin(alpha) moment vanishes (theta -> -theta)."""
    p = _cyl(n_u=4000, n_phi=1, n_E=1, eps=0.0)
    rho = orc.init_state(p)
    r = 15.0
    x = p.R_nu / r
    M = orc.moments_ex(p, rho, r).reshape(4, 4)
    R = orc.unpack(rho, 2).reshape(2, p.n_u, 2, 2)
    S = (R[0, 0] - np.conj(R[1, 0])) * (p.E_max - p.E_min)  # dE times the one energy bin, any trajectory
    assert M[0, 0] == pytest.approx(S[0, 0].real * 2 * np.arcsin(x) / x, rel=1e-6)
    assert M[1, 0] == pytest.approx(S[0, 0].real * 2.0, rel=1e-6)
    assert abs(M[2, 0]) < 1e-12 * abs(M[0, 0])


@pytest.mark.parametrize("stepper", [I.RK4, I.EXPH])
def test_cylinder_uniform_latitudes_equal_one_latitude(orc, stepper):
    """A state the same at every latitude stays so, and equals the model with
    one latitude bin, where G = mu (M0 - cos(alpha) M1 - sin(alpha) M2) from
    three moments: the interpolated pair sum and the moment sum agree."""
    p = _cyl(stepper=stepper, n_steps=40)
    one = p.replace(n_phi=1)
    rho1 = orc.init_state(one)
    rho = np.ascontiguousarray(np.broadcast_to(rho1.reshape(2, p.n_u, 1, p.n_E, 4),
                                               (2, p.n_u, p.n_phi, p.n_E, 4))).reshape(-1)
    a, st, _ = orc.evolve(p, rho, p.r0, p.h, p.n_steps)
    b, st1, _ = orc.evolve(one, rho1, p.r0, p.h, p.n_steps)
    assert st == 0 and st1 == 0
    a = a.reshape(2, p.n_u, p.n_phi, p.n_E, 4)
    assert np.abs(b - rho1).max() > 1e-4
    for k in range(p.n_phi):
        assert np.abs(a[:, :, k] - b.reshape(2, p.n_u, p.n_E, 4)).max() < 1e-12


def test_cylinder_rotation_and_mirror(orc):
    """The model is invariant under a rotation by one latitude bin and under
    the mirror (Phi, theta) -> (-Phi, -theta): evolving the rotated or
    mirrored state gives the rotated or mirrored result."""
    p = _cyl(n_steps=30)
    rho = orc.init_state(p).reshape(2, p.n_u, p.n_phi, p.n_E, 4)
    out, st, _ = orc.evolve(p, rho.reshape(-1), p.r0, p.h, p.n_steps)
    out = out.reshape(rho.shape)
    rot, _, _ = orc.evolve(p, np.roll(rho, 1, axis=2).reshape(-1), p.r0, p.h, p.n_steps)
    assert np.abs(rot.reshape(rho.shape) - np.roll(out, 1, axis=2)).max() < 1e-14
    mir = rho[:, ::-1, ::-1]
    m, _, _ = orc.evolve(p, np.ascontiguousarray(mir).reshape(-1), p.r0, p.h, p.n_steps)
    assert np.abs(m.reshape(rho.shape) - out[:, ::-1, ::-1]).max() < 1e-12
    assert np.abs(out - rho).max() > 1e-4


@pytest.mark.parametrize("stepper,tol", [(I.RK4, 2e-8), (I.EXPH, 1e-11)])
def test_cylinder_vacuum_survival(orc, stepper, tol):
    """P1 on the cylinder's trajectories: mu = A = 0 gives P_ee = 1 -
    sin^2(2 theta) sin^2(Delta L/2) with L = sqrt(r^2 - R^2 sin^2 th) between
    r0 and r1 (the chord of a straight ray whose impact parameter is R sin th)."""
    p = _cyl(n_E=12, n_u=7, n_phi=3, stepper=stepper, mu0=0.0, eps=0.0, theta=(0.3, 0, 0), hierarchy=-1,
             E_min=1.0, E_max=13.0, r0=20.0, r1=30.0, n_steps=1000)
    E, u, phi, Hv = orc.tables(p)
    out, st, _ = orc.evolve(p, orc.init_state(p), p.r0, p.h, p.n_steps)
    assert st == 0
    M = orc.unpack(out, 2).reshape(2, p.n_u, p.n_phi, p.n_E, 2, 2)
    th = -np.pi / 2 + (np.arange(p.n_u) + 0.5) * np.pi / p.n_u
    b2 = (p.R_nu * np.sin(th)) ** 2
    L = np.sqrt(p.r1 ** 2 - b2) - np.sqrt(p.r0 ** 2 - b2)
    Delta = orc.vac_coeff() * p.hierarchy * p.dm2[0] / E
    Pee = 1 - np.sin(2 * 0.3) ** 2 * np.sin(np.outer(L, Delta) / 2) ** 2
    for s, (ie, ix) in enumerate([(0, 2), (1, 3)]):
        want = phi[ix] + (phi[ie] - phi[ix]) * Pee
        for k in range(p.n_phi):
            assert np.abs(M[s, :, k, :, 0, 0].real - want).max() < tol * phi[0].max()
