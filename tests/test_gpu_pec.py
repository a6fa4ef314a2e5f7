"""The iterated Hermite corrector P(EC)^n (nb_config.n_corr) on the GPU against the oracle's
P(EC)^n: shared and block steps, FP64 and double-single pairs, and the time symmetry the
iterations buy."""
import math

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu


def _two_body_kepler(nper):
    e, d = 0.5, 0.5
    a = d / (1 - e)
    vrel = math.sqrt((1 + e) / (a * (1 - e)))
    pos = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    vel = np.array([[0, -vrel / 2, 0], [0, vrel / 2, 0]])
    return np.array([0.5, 0.5]), pos, vel, 2 * math.pi * a ** 1.5 / nper


def test_one_iteration_is_pec(nb):
    p = ic.plummer(600, 70)
    kw = dict(variant="f32ds", eps=0.01, eta=0.02, device=0)
    with nb.System(p.m, p.pos, p.vel, flags=nb.NB_FLAG_NO_FUSED, **kw) as a:
        a.step(1.0 / 16)
        ga = a.state()
    with nb.System(p.m, p.pos, p.vel, flags=nb.NB_FLAG_NO_FUSED, n_corr=1, **kw) as b:
        b.step(1.0 / 16)
        gb = b.state()
    for k in ("pos", "vel", "acc", "jerk", "dt"):
        np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("n_corr", [2, 3])
def test_shared_steps_fp64_vs_oracle(nb, n_corr):
    """N = 256, FP64 pairs, 32 shared steps: the oracle's P(EC)^n state to 1e-11."""
    p = ic.plummer(256, 71)
    eps, dt = 1.0 / 64, 1.0 / 256
    st = oracle.State(p.m, p.pos, p.vel)
    _, o_inter = oracle.hermite_run(st, 32 * dt, eps * eps, dt_shared=dt, n_corr=n_corr)
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=eps, shared_dt=dt, n_corr=n_corr,
                   device=0) as s:
        stats = s.step(32 * dt)
        g = s.state()
    assert stats["interactions"] == o_inter
    assert np.abs(g["pos"].T - st.pos).max() < 1e-11
    assert np.abs(g["vel"].T - st.vel).max() < 1e-10


@pytest.mark.parametrize("variant", ["f64", "f32ds"])
def test_block_steps_vs_oracle(nb, variant):
    """Block steps (eta = 0.02) over 1/16 time unit with P(EC)^2: the oracle's schedule and
    state (FP64 pairs: the same schedule exactly)."""
    p = ic.plummer(512, 72)
    eps = 0.01
    st = oracle.State(p.m, p.pos, p.vel)
    o_steps, o_inter = oracle.hermite_run(st, 1.0 / 16, eps * eps, eta=0.02, dt_max=1.0 / 16,
                                          n_corr=2)
    with nb.System(p.m, p.pos, p.vel, variant=variant, eps=eps, eta=0.02, dt_max=1.0 / 16,
                   n_corr=2, device=0) as s:
        stats = s.step(1.0 / 16)
        g = s.state()
    assert stats["fused_steps"] == 0
    np.testing.assert_array_equal(g["t"], 1.0 / 16)
    if variant == "f64":
        assert stats["block_steps"] == o_steps
        assert abs(stats["interactions"] - o_inter) <= 1e-3 * o_inter
        assert np.abs(g["pos"].T - st.pos).max() < 1e-8
    else:
        assert abs(stats["block_steps"] - o_steps) <= 0.05 * o_steps
        assert np.abs(g["pos"].T - st.pos).max() < 1e-5


def _reversal(nb, n_corr, nper=256, periods=3):
    m, pos, vel, dt = _two_body_kepler(nper)
    t = nper * periods * dt
    kw = dict(variant="f64", eps=0.0, shared_dt=dt, n_corr=n_corr, device=0)
    with nb.System(m, pos, vel, **kw) as s:
        s.step(t)
        g = s.state()
    with nb.System(m, g["pos"].T, -g["vel"].T, **kw) as s:
        s.step(t)
        b = s.state()
    return np.abs(b["pos"].T - pos).max()


def test_iterations_approach_time_symmetry(nb):
    r1, r2 = _reversal(nb, 1), _reversal(nb, 2)
    assert r1 > 1e-5
    assert r2 < 1e-3 * r1


def test_n_corr_limits(nb):
    p = ic.plummer(64, 73)
    with pytest.raises(nb.NBodyError) as e:
        nb.System(p.m, p.pos, p.vel, n_corr=nb.NB_MAX_CORR + 1, device=0)
    assert e.value.status == nb.NB_ERR_ARG
