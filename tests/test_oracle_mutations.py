"""The oracle's pins are tight enough to catch plausible mistakes.

Each case below plants one mistake in a scratch copy of the oracle's C source
(a reversed profile, a dropped factor, a wrong power of R/r, a misplaced or
mis-signed matter term, a wrong angle weight), builds it into a temporary
library and runs the pins that should notice it against that library, in a
child process.  The case passes when at least one of those pins fails.  The
repository's oracle itself is untouched; every mistake lives only in the
temporary copy, on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "xf_oracle.c")

# (name, text in the oracle, planted replacement, pins expected to notice)
MUTATIONS = [
    ("power law turned upside down (Eq. 4.3)",
     "pow(p->r_ref / r, p->ne_power)", "pow(r / p->r_ref, p->ne_power)",
     "landau_zener or adiabatic_track"),
    ("power-law exponent off by one (Eq. 4.3)",
     "pow(p->r_ref / r, p->ne_power)", "pow(p->r_ref / r, p->ne_power - 1.0)",
     "landau_zener or adiabatic_track"),
    ("electron fraction dropped (Eq. 3.7, 4.4)",
     "p->Ye * p->nb0 * exp", "p->nb0 * exp",
     "adiabatic_track or hop_probability"),
    ("exponential profile growing outward (Eq. 4.4)",
     "exp(-(r - p->R_nu) / p->h_ns)", "exp((r - p->R_nu) / p->h_ns)",
     "adiabatic_track or hop_probability"),
    ("offset R dropped from the exponential profile (Eq. 4.4)",
     "exp(-(r - p->R_nu) / p->h_ns)", "exp(-r / p->h_ns)",
     "adiabatic_track or hop_probability"),
    ("literal coupling with (R/r)^2 instead of (R/r)^4",
     "p->mu0 * x2 * x2", "p->mu0 * x2",
     "mu_r4_coupling_precession"),
    ("literal coupling without the cosine weight of M1",
     "g->w[1][t] = c->du * cth;", "g->w[1][t] = c->du;",
     "mu_r4_coupling_precession"),
    ("bulb weight of M1 without its cosine (Eq. 3.13-3.15)",
     "g->w[1][t] = a * cth / c->nphi;", "g->w[1][t] = a / c->nphi;",
     "bulb_coupling_precession or isotropic_closed_form"),
    ("matter term on the last flavor instead of nu_e",
     "H[0] += (s == 0 ? A : -A);", "H[n * n - 1] += (s == 0 ? A : -A);",
     "constant_matter"),
    ("antineutrinos see +A (after Eq. 3.4)",
     "H[0] += (s == 0 ? A : -A);", "H[0] += A;",
     "constant_matter or hop_probability"),
    ("three-flavor matter potential halved",
     "H[0] += (s == 0 ? A : -A);", "H[0] += (s == 0 ? A : -A) * (n == 3 ? 0.5 : 1.0);",
     "constant_matter_three_flavor"),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, pins):
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    text = open(SRC).read()
    assert text.count(old) == 1, f"the text to mutate is not unique in the oracle: {old!r}"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    lib = str(tmp_path / "libmutant.so")
    O.compile_to(str(src), lib)
    env = dict(os.environ, XF_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode == 1 and " failed" in r.stdout, \
        f"no pin noticed the planted mistake ({name}):\n{r.stdout[-2000:]}"
