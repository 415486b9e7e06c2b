"""Seeded synthetic workloads for the bulb-model flavor-evolution path.

This module only states parameter sets and draws seeded random numbers.  It
holds none of the method's arithmetic, so both the CUDA path and the CPU
oracle may take their inputs from it.

The physical parameters follow the paper's bulb-model runs (Sec. 4.5): Fermi-
Dirac spectra with degeneracy eta = 3 and temperatures 2.76 / 4.01 / 6.26 MeV
for nu_e / nubar_e / nu_x, equal luminosities, neutrinosphere radius 10 km,
mixing angle 0.1.  The workloads below are the five run shapes the library is
measured on (two- and three-flavor single instances, a precision study, a
batched ensemble, and a served job stream), plus stable companions that start
at 50 km, the start radius of the paper's validation runs (Sec. 4.5).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Tuple

# stepper / geometry / matter / precision enums (values fixed by include/xf.h)
RK4, EXPH, EXPH_ADAPTIVE = 0, 1, 2
BULB, MU_R4, SINGLE_ANGLE, CONST, CYLINDER = 0, 1, 2, 3, 4
MATTER_NONE, MATTER_POWER, MATTER_EXP = 0, 1, 2
FP64, FP32_M64, FP32_COMP, FP32_M64_RENORM, FP32X2 = 0, 1, 2, 3, 4
FORM_RHO, FORM_PSI = 0, 1  # state: density matrices, or one wavefunction per initial flavor


@dataclass
class Problem:
    """One flavor-evolution problem (the paper's configuration keywords)."""

    n_E: int = 32                     # Ebins
    n_u: int = 16                     # Abins
    n_f: int = 2                      # Flvs
    n_phi: int = 1                    # Pbins: azimuth bins of the extended bulb model (1: none)
    stepper: int = RK4
    geometry: int = BULB
    precision: int = FP64
    strict: int = 0                   # 1: refuse RK4 steps outside the stable region
    form: int = FORM_RHO              # FORM_PSI: the wavefunction form (Eq. 3.9-3.11)
    R_nu: float = 10.0                # km, neutrinosphere radius
    mu0: float = 1.0e5                # km^-1
    E_min: float = 1.0                # MeV
    E_max: float = 60.0               # MeV
    dm2: Tuple[float, float] = (2.4e-3, 0.0)       # eV^2 magnitudes
    theta: Tuple[float, float, float] = (0.1, 0.0, 0.0)
    hierarchy: int = -1               # +1 normal, -1 inverted
    matter: int = MATTER_NONE
    ne_ref: float = 0.0               # cm^-3 at r_ref
    r_ref: float = 10.0               # km
    ne_power: float = 3.0
    nb0: float = 0.0
    h_ns: float = 1.0
    Ye: float = 0.5
    T: Tuple[float, float, float, float] = (2.76, 4.01, 6.26, 6.26)
    eta: Tuple[float, float, float, float] = (3.0, 3.0, 3.0, 3.0)
    L: Tuple[float, float, float, float] = (1.0, 1.0, 1.0, 1.0)
    eps: float = 1.0e-6
    seed: int = 1
    eps0: float = 1.0e-6              # error-controlled step: tolerance
    ksi: float = 0.9                  # error-controlled step: safety factor
    dr_max: float = 1.0               # error-controlled step: largest step, km
    r0: float = 10.0                  # km, start radius
    r1: float = 200.0                 # km, end radius
    n_steps: int = 2000

    @property
    def h(self) -> float:
        return (self.r1 - self.r0) / self.n_steps

    @property
    def n_bins(self) -> int:
        return 2 * self.n_u * self.n_phi * self.n_E

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---- the measured run shapes --------------------------------------------

def bulb2f_16x32() -> Problem:
    """Two flavors, 16 angles x 32 energies (1-60 MeV), inverted hierarchy,
    mu0 = 1e5 km^-1, no matter, 2000 steps from 10 to 200 km."""
    return Problem(n_E=32, n_u=16, n_f=2, stepper=EXPH, mu0=1.0e5, r0=10.0, r1=200.0,
                   n_steps=2000, seed=1)


def bulb2f_16x32_from_50km() -> Problem:
    """The two-flavor 16 x 32 physics from 50 to 250 km in 20000 steps (h = 0.01 km), where
    explicit RK4 is stable."""
    return bulb2f_16x32().replace(stepper=RK4, r0=50.0, r1=250.0, n_steps=20000)


def bulb3f_1000x200() -> Problem:
    """Three flavors, 1000 angles x 200 energies (400,000 3x3 bins),
    dm21 = 7.5e-5, dm31 = 2.4e-3 eV^2 (normal), angles 0.59/0.15/0.72,
    n_e = 1e33 (10 km / r)^3 cm^-3, 20000 steps from 10 to 1000 km."""
    return Problem(n_E=200, n_u=1000, n_f=3, stepper=EXPH, mu0=1.0e5,
                   dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1,
                   matter=MATTER_POWER, ne_ref=1.0e33, r_ref=10.0, ne_power=3.0,
                   r0=10.0, r1=1000.0, n_steps=20000, seed=2)


def bulb3f_1000x200_from_250km() -> Problem:
    """The three-flavor 1000 x 200 physics from 250 to 1000 km in 20000 steps, stable for RK4."""
    return bulb3f_1000x200().replace(stepper=RK4, r0=250.0, r1=1000.0, n_steps=20000)


def bulb2f_16x32_coarse(precision: int = FP32_M64) -> Problem:
    """The two-flavor 16 x 32 physics from 10 km with h = 0.1 km (precision study; checkpoints at
    100, 300 and 1000 km)."""
    return bulb2f_16x32().replace(stepper=EXPH, precision=precision, r0=10.0, r1=1000.0, n_steps=9900)


def bulb2f_16x32_fine(precision: int = FP32_M64, stepper: int = RK4) -> Problem:
    """The precision-study physics (two flavors, 16 x 32) from 50 km with h = 0.01 km."""
    return bulb2f_16x32().replace(stepper=stepper, precision=precision, r0=50.0, r1=1000.0, n_steps=95000)


# ---- seeded generators ----------------------------------------------------

class SplitMix64:
    """Sequential SplitMix64 (Steele, Lea & Flood 2014) for drawing workload
    parameters.  Not used for anything inside the integrator."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


def ensemble_problems(n_instances: int = 256, seed: int = 4, n_steps: int = 1000) -> List[Problem]:
    """Batched ensemble: n_u ~ U{64..1024}, n_E ~ U{32..256}, 2 or 3 flavors,
    mu0 log-uniform in [1e3, 1e6] km^-1, either hierarchy, theta_v ~ U[0.01, 0.6]
    (2 flavors; 3 flavors use the 1000-angle problem's), r 50 -> 250 km."""
    g = SplitMix64(seed)
    out = []
    for i in range(n_instances):
        n_u = g.randint(64, 1024)
        n_E = g.randint(32, 256)
        n_f = 2 if g.uniform() < 0.5 else 3
        mu0 = 10.0 ** (3.0 + 3.0 * g.uniform())
        hier = 1 if g.uniform() < 0.5 else -1
        th = 0.01 + 0.59 * g.uniform()
        if n_f == 2:
            p = Problem(n_E=n_E, n_u=n_u, n_f=2, dm2=(2.4e-3, 0.0), theta=(th, 0.0, 0.0))
        else:
            p = Problem(n_E=n_E, n_u=n_u, n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72))
        out.append(p.replace(mu0=mu0, hierarchy=hier, stepper=EXPH, precision=FP32_M64,
                             r0=50.0, r1=250.0, n_steps=n_steps, seed=1000 + i))
    return out


def job_arrivals(rate_per_s: float = 200.0, window_s: float = 60.0, seed: int = 5,
                size_scale: float = 1.0) -> List[Tuple[float, Problem]]:
    """Served job stream: Poisson arrivals at `rate_per_s` over `window_s`;
    two-flavor jobs with the batched ensemble's size distribution (scaled by size_scale),
    1000-20000 steps of h = 0.01 km from 50 km, FP32 with FP64 moments."""
    g = SplitMix64(seed)
    t = 0.0
    out = []
    k = 0
    while True:
        t += -math.log(1.0 - g.uniform()) / rate_per_s
        if t >= window_s:
            break
        n_u = max(1, int(g.randint(64, 1024) * size_scale))
        n_E = max(1, int(g.randint(32, 256) * size_scale))
        steps = g.randint(1000, 20000)
        mu0 = 10.0 ** (3.0 + 3.0 * g.uniform())
        hier = 1 if g.uniform() < 0.5 else -1
        th = 0.01 + 0.59 * g.uniform()
        p = Problem(n_E=n_E, n_u=n_u, n_f=2, mu0=mu0, hierarchy=hier, theta=(th, 0.0, 0.0),
                    stepper=EXPH, precision=FP32_M64, r0=50.0, r1=50.0 + 0.01 * steps,
                    n_steps=steps, seed=5000 + k)
        out.append((t, p))
        k += 1
    return out
