"""Checkpoints and reduced outputs (the paper's I/O module, Sec. 4.2.4):
a run stopped, saved, loaded into a fresh context and continued gives bitwise
the state of the run that never stopped; the asynchronous save copies the
state of the moment it was called while later steps run; dump mode 2 (the
energy average of each trajectory) equals the average of the full state."""
import numpy as np
import pytest

from paper_1907_05560_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05560_gb300 import build, xf as X
    build.build()
    X.load()
    return X


THREE = dict(n_f=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.72), hierarchy=+1, matter=I.MATTER_POWER,
             ne_ref=1e31)
CASES = {
    "2f-exph-fp64": I.Problem(n_E=24, n_u=20, stepper=I.EXPH, r0=50.0, r1=51.0, n_steps=100, eps=1e-3, seed=3),
    "3f-exph-fp64": I.Problem(n_E=20, n_u=17, stepper=I.EXPH, r0=60.0, r1=60.8, n_steps=80, eps=1e-3, seed=4,
                              mu0=1e4, **THREE),
    "2f-rk4-fp32": I.Problem(n_E=24, n_u=20, stepper=I.RK4, precision=I.FP32_M64, r0=50.0, r1=51.0, n_steps=100,
                             eps=1e-3, seed=5),
    "3f-exph-renorm": I.Problem(n_E=20, n_u=17, stepper=I.EXPH, precision=I.FP32_M64_RENORM, r0=60.0, r1=60.8,
                                n_steps=80, eps=1e-3, seed=6, mu0=1e4, **THREE),
    "3f-exph-fp32x2": I.Problem(n_E=20, n_u=17, stepper=I.EXPH, precision=I.FP32X2, r0=60.0, r1=60.8,
                                n_steps=80, eps=1e-3, seed=7, mu0=1e4, **THREE),
}


@pytest.mark.parametrize("name", list(CASES))
def test_resume_from_checkpoint_is_bitwise(xf, name):
    p = CASES[name]
    k = 37
    a = xf.Context(p)
    a.init_state(p.r0)
    a.step(p.n_steps, p.h)
    want, r_want, n_want = a.get_state()
    a.close()
    b = xf.Context(p)
    b.init_state(p.r0)
    b.step(k, p.h)
    ck = b.checkpoint_save()
    b.close()
    c = xf.Context(p)
    c.checkpoint_load(ck)
    got0, r0, n0 = c.get_state()
    assert n0 == k and r0 == pytest.approx(p.r0 + k * p.h, rel=1e-14)
    c.step(p.n_steps - k, p.h)
    got, r, n = c.get_state()
    c.close()
    assert np.array_equal(got, want) and r == r_want and n == n_want


def test_async_checkpoint_captures_the_moment_of_the_call(xf):
    p = CASES["3f-exph-fp64"]
    c = xf.Context(p)
    c.init_state(p.r0)
    c.step(20, p.h)
    sync = c.checkpoint_save()
    buf = np.zeros(c.checkpoint_bytes(), dtype=np.uint8)
    c.checkpoint_save_async(buf)
    c.step_async(30, p.h)  # runs while the copy is in flight
    with pytest.raises(xf.XFError) as ei:
        c.checkpoint_save_async(np.zeros_like(buf))
    assert ei.value.name == "XF_E_BUSY"
    c.checkpoint_wait()
    c.sync()
    assert np.array_equal(buf, sync)
    assert c.get_state()[2] == 50
    c.close()


def test_adaptive_resume_is_bitwise(xf, orc):
    p = I.Problem(n_E=24, n_u=12, mu0=1e5, eps=1e-3, seed=11, r0=50.0, eps0=1e-6, dr_max=0.2,
                  stepper=I.EXPH_ADAPTIVE)
    a = xf.Context(p)
    a.init_state(p.r0)
    with pytest.raises(xf.XFError):
        a.evolve(52.0, 400, 0.1)  # stops on the budget
    ck = a.checkpoint_save()
    s_mid = a.adapt_status()
    a.evolve(52.0, 1 << 40, 0.0)
    want = a.get_state()[0]
    s_a = a.adapt_status()
    a.close()
    b = xf.Context(p)
    b.checkpoint_load(ck)
    s_b0 = b.adapt_status()
    assert s_b0["r"] == s_mid["r"] and s_b0["h_next"] == s_mid["h_next"]
    b.evolve(52.0, 1 << 40, 0.0)
    s_b = b.adapt_status()
    assert np.array_equal(b.get_state()[0], want)
    assert (s_b["n_accepted"], s_b["n_rejected"], s_b["r"]) == (s_a["n_accepted"], s_a["n_rejected"], s_a["r"])
    b.close()


def test_checkpoint_rejects_other_problems(xf):
    p = CASES["2f-exph-fp64"]
    c = xf.Context(p)
    c.init_state(p.r0)
    ck = c.checkpoint_save()
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(xf.XFError) as ei:
        c.checkpoint_load(bad)
    assert ei.value.name == "XF_E_ARG"
    other = xf.Context(p.replace(stepper=I.RK4))
    with pytest.raises(xf.XFError) as ei:
        other.checkpoint_load(ck)
    assert ei.value.name == "XF_E_ARG"
    other.close()
    c.close()


@pytest.mark.parametrize("name", ["2f-exph-fp64", "3f-exph-fp64", "2f-rk4-fp32"])
def test_angle_average_is_the_energy_mean(xf, name):
    p = CASES[name]
    c = xf.Context(p)
    c.init_state(p.r0)
    c.step(10, p.h)
    rho = c.get_state()[0].reshape(2, p.n_u, p.n_E, p.n_f * p.n_f)
    avg = c.angle_average().reshape(2, p.n_u, p.n_f * p.n_f)
    c.close()
    want = rho.mean(axis=2)
    assert np.abs(avg - want).max() <= 1e-14 * np.abs(want).max()
