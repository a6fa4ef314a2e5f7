"""Pins of the oracle's Hermite integrator, step criterion and block scheduler.

Facts used (none of them is the oracle's own formula typed again):
- the predictor is exact for cubic trajectories, the corrector for quintic ones
  (Hermite interpolation through a, jerk at both ends is exact for cubic a(t));
- hand-evaluated step criterion and block quantization cases;
- two-body orbits: Kepler's equation (no softening) and the softened circular
  orbit omega^2 = M / (d^2 + eps^2)^(3/2);
- 4th-order convergence: halving dt divides the position error by ~16 and
  the energy error by at least 14;
- shared-step Hermite conserves linear momentum to rounding;
- block times are dyadic, every dt is a power of two that divides t;
- a block run whose steps are all forced equal is bit-identical to a
  shared-step run;
- energy drift of the N = 1024 Plummer test case over one time unit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic


def test_predictor_exact_for_cubic():
    # x(t) = 1 + 2t + 3t^2 + 2t^3 : v = 2 + 6t + 6t^2, a = 6 + 12t, jerk = 12
    pos = np.array([[1.0, -1.0, 0.5]])
    vel = np.array([[2.0, -2.0, 1.0]])
    acc = np.array([[6.0, -6.0, 3.0]])
    jerk = np.array([[12.0, -12.0, 6.0]])
    pp, vp = oracle.predict(0.5, [0.0], pos, vel, acc, jerk)
    np.testing.assert_array_equal(pp, [[3.0, -3.0, 1.5]])
    np.testing.assert_array_equal(vp, [[6.5, -6.5, 3.25]])
    # from a later own time: prediction from t_j = 0.25 to 0.75 of the same curve
    t0 = 0.25
    x0 = 1 + 2 * t0 + 3 * t0 ** 2 + 2 * t0 ** 3
    v0 = 2 + 6 * t0 + 6 * t0 ** 2
    a0 = 6 + 12 * t0
    pp, vp = oracle.predict(0.75, [t0], [[x0] * 3], [[v0] * 3], [[a0] * 3], [[12.0] * 3])
    t1 = 0.75
    np.testing.assert_allclose(pp, [[1 + 2 * t1 + 3 * t1 ** 2 + 2 * t1 ** 3] * 3], rtol=1e-15)
    np.testing.assert_allclose(vp, [[2 + 6 * t1 + 6 * t1 ** 2] * 3], rtol=1e-15)


def test_corrector_exact_for_quintic():
    """x(t) = sum c_k t^k, k <= 5: a is cubic, so a2, a3 from (a0, j0, a1, j1) are exact
    and the corrected x1, v1 equal the polynomial at t = dt."""
    c = np.array([0.3, -1.1, 0.7, 2.0, -1.5, 0.9])

    def deriv(t, d):
        out = 0.0
        for k in range(d, 6):
            out += c[k] * math.factorial(k) / math.factorial(k - d) * t ** (k - d)
        return out

    dt = 0.125
    x0, v0, a0, j0 = (np.full(3, deriv(0.0, d)) for d in range(4))
    xp, vp = oracle.predict(dt, [0.0], x0[None], v0[None], a0[None], j0[None])
    a1, j1 = np.full(3, deriv(dt, 2)), np.full(3, deriv(dt, 3))
    x1, v1, a2e, a3e = oracle.correct_one(dt, xp[0], vp[0], a0, j0, a1, j1)
    np.testing.assert_allclose(x1, deriv(dt, 0), rtol=1e-14)
    np.testing.assert_allclose(v1, deriv(dt, 1), rtol=1e-14)
    np.testing.assert_allclose(a2e, deriv(dt, 4), rtol=1e-12)
    np.testing.assert_allclose(a3e, deriv(dt, 5), rtol=1e-12)


def test_aarseth_criterion_hand_values():
    # |a|=|j|=|a2|=|a3|=1: dt = sqrt(eta * 2 / 2)
    assert oracle.aarseth_dt([1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 0], 0.04) == pytest.approx(
        0.2, rel=1e-15)
    # |a|=2, |j|=1, |a2|=3, |a3|=4: dt = sqrt(eta (2*3 + 1) / (1*4 + 9)) = sqrt(7 eta / 13)
    assert oracle.aarseth_dt([0, 2, 0], [1, 0, 0], [0, 0, 3], [0, 4, 0], 0.01) == pytest.approx(
        math.sqrt(0.07 / 13), rel=1e-15)
    assert oracle.aarseth_dt([0, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0], 0.01) == math.inf
    assert oracle.initial_dt([3, 4, 0], [0, 0, 2], 0.01) == pytest.approx(0.025, rel=1e-15)
    assert oracle.initial_dt([1, 0, 0], [0, 0, 0], 0.01) == math.inf


def test_quantize_cases():
    dmin, dmax = 2.0 ** -30, 1.0 / 16
    q = oracle.quantize
    assert q(0.3, 0.0, 0.0, dmin, dmax) == dmax            # clamp to dt_max
    assert q(0.02, 0.0, 0.0, dmin, dmax) == 1.0 / 64       # 1/64 <= 0.02 < 1/32
    assert q(1.0 / 64, 0.0, 0.0, dmin, dmax) == 1.0 / 64   # exact power of two kept
    assert q(math.inf, 1.0 / 64, 1.0 / 32, dmin, dmax) == 1.0 / 32   # growth limited to x2
    # growth only where the new time is a multiple of the doubled step
    assert q(1.0, 1.0 / 64, 3.0 / 64, dmin, dmax) == 1.0 / 64
    assert q(1.0, 1.0 / 64, 4.0 / 64, dmin, dmax) == 1.0 / 32
    # shrinking is free: 1e-5 -> 2^-17 (7.6e-6 <= 1e-5 < 1.5e-5)
    assert q(1e-5, 1.0 / 64, 3.0 / 64, dmin, dmax) == 2.0 ** -17
    assert q(1e-12, 1.0 / 64, 3.0 / 64, dmin, dmax) == dmin  # clamp to dt_min
    # a step must divide the particle's time: at t = 3/8, 1/4 does not (3/8 = 1.5 * 1/4)
    assert q(0.3, 0.0, 3.0 / 8, dmin, 0.25) == 1.0 / 8
    assert q(0.07, 0.0, 3.0 / 8, dmin, 0.25) == 1.0 / 16   # 1/16 <= 0.07 and 3/8 = 6/16


def _two_body(d, e_frac=0.0, eps=0.0):
    """Equal masses 1/2 (M=1) on a relative orbit starting at pericentre d with
    eccentricity e (e = 0: circular, softened when eps > 0). Centre-of-mass frame."""
    if e_frac == 0.0:
        omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
        vrel = omega * d
    else:
        a = d / (1 - e_frac)
        vrel = math.sqrt((1 + e_frac) / (a * (1 - e_frac)))
    pos = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    vel = np.array([[0, -vrel / 2, 0], [0, vrel / 2, 0]])
    return np.array([0.5, 0.5]), pos, vel


def _run_shared(m, pos, vel, eps2, dt, nsteps):
    st = oracle.State(m, pos, vel)
    steps, _ = oracle.hermite_run(st, math.inf, eps2, dt_shared=dt, max_steps=nsteps)
    assert steps == nsteps
    return st


def _circular_error(nsteps):
    d, eps = 1.0, 0.3
    m, pos, vel = _two_body(d, eps=eps)
    omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
    period = 2 * math.pi / omega
    st = _run_shared(m, pos, vel, eps * eps, period / nsteps, nsteps)
    return np.abs(st.pos - pos).max()


def test_softened_circular_orbit_and_convergence():
    e1 = _circular_error(128)
    e2 = _circular_error(256)
    assert e2 < 2e-7
    assert 12.0 < e1 / e2 < 20.0   # 4th order: error / 16


def _kepler_position(t, a, e):
    """Relative position at time t after pericentre (M = 1) from Kepler's equation."""
    mean = t / a ** 1.5
    ea = mean
    for _ in range(50):
        ea -= (ea - e * math.sin(ea) - mean) / (1 - e * math.cos(ea))
    return np.array([a * (math.cos(ea) - e), a * math.sqrt(1 - e * e) * math.sin(ea), 0.0])


def _kepler_error(nsteps_per_period):
    e, d = 0.5, 0.5
    a = d / (1 - e)
    m, pos, vel = _two_body(d, e_frac=e)
    period = 2 * math.pi * a ** 1.5
    n = nsteps_per_period // 3
    dt = period / nsteps_per_period
    st = _run_shared(m, pos, vel, 0.0, dt, n)
    rel = st.pos[1] - st.pos[0]
    return np.abs(rel - _kepler_position(n * dt, a, e)).max()


def test_kepler_ellipse_and_convergence():
    e1 = _kepler_error(768)
    e2 = _kepler_error(1536)
    assert e2 < 1e-7
    assert 12.0 < e1 / e2 < 20.0


def test_shared_step_momentum_conservation():
    p = ic.plummer(64, 21, masses="lognormal")
    st = _run_shared(p.m, p.pos, p.vel, 1e-2, 1.0 / 256, 32)
    mom = (p.m[:, None] * st.vel).sum(axis=0)
    assert np.abs(mom).max() < 1e-15


def make_block_run():
    p = ic.plummer(128, 22)
    st = oracle.State(p.m, p.pos, p.vel)
    steps, inter = oracle.hermite_run(st, 0.25, (1.0 / 64) ** 2, eta=0.02, dt_max=1.0 / 16)
    return p, st, steps, inter


@pytest.fixture(scope="module")
def block_run():
    return make_block_run()


def test_block_times_are_dyadic(block_run):
    p, st, steps, inter = block_run
    np.testing.assert_array_equal(st.t, 0.25)        # every particle reached t_end exactly
    lg = np.log2(st.dt)
    np.testing.assert_array_equal(lg, np.round(lg))    # powers of two
    assert (st.dt <= 1.0 / 16).all()
    np.testing.assert_array_equal(np.fmod(st.t, st.dt), 0.0)
    assert steps > 4 and inter > 128 * 128
    assert len(np.unique(st.dt)) > 1                   # steps really are individual


def test_block_steps_resume_equals_uninterrupted():
    p = ic.plummer(64, 23)
    a = oracle.State(p.m, p.pos, p.vel)
    oracle.hermite_run(a, 0.125, 1e-3, eta=0.02)
    b = oracle.State(p.m, p.pos, p.vel)
    oracle.hermite_run(b, 1.0 / 16, 1e-3, eta=0.02)
    c = oracle.State(b.m, b.pos, b.vel, acc=b.acc, jerk=b.jerk, t=b.t, dt=b.dt)
    oracle.hermite_run(c, 0.125, 1e-3, eta=0.02)
    np.testing.assert_array_equal(a.pos, c.pos)
    np.testing.assert_array_equal(a.vel, c.vel)


def test_equal_block_steps_equal_shared_steps():
    p = ic.plummer(64, 24)
    dt = 1.0 / 256
    a = _run_shared(p.m, p.pos, p.vel, 1e-3, dt, 16)
    b = oracle.State(p.m, p.pos, p.vel)
    steps, _ = oracle.hermite_run(b, 16 * dt, 1e-3, eta=0.01, dt_min=dt, dt_max=dt)
    assert steps == 16
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.vel, b.vel)


def _energy(st, eps2):
    k, w = oracle.energy(st.m, st.pos, st.vel, eps2)
    return k + w


def test_energy_convergence_order():
    """Energy error over a fixed interval falls at least as fast as dt^4 (here it is
    close to dt^5, a ratio near 32); a dropped corrector term gives a ratio of 8 or less."""
    p = ic.plummer(16, 25)
    eps2 = 0.05 ** 2
    e0 = _energy(oracle.State(p.m, p.pos, p.vel), eps2)
    errs = []
    for nsteps in (128, 256):
        st = _run_shared(p.m, p.pos, p.vel, eps2, 0.5 / nsteps, nsteps)
        errs.append(abs(_energy(st, eps2) - e0))
    assert 14.0 < errs[0] / errs[1] < 40.0


@pytest.mark.slow
def test_plummer_1024_energy_drift():
    """The small test case: N = 1024 Plummer, eps = 1/64, shared dt = 1/256, one time unit."""
    p = ic.plummer(1024)
    eps2 = (1.0 / 64) ** 2
    st = oracle.State(p.m, p.pos, p.vel)
    e0 = _energy(st, eps2)
    steps, inter = oracle.hermite_run(st, 1.0, eps2, dt_shared=1.0 / 256)
    assert steps == 256
    assert inter == 257 * 1024 * 1024
    e1 = _energy(st, eps2)
    assert abs((e1 - e0) / e0) < 1e-6


def _two_binaries():
    """Two circular binaries (masses 1/4, separations 0.01 and 0.04) ten units apart.
    For uniform circular motion |a|, |jerk|, |a2|, |a3| are omega^k r, so the step
    criterion gives dt = sqrt(eta) / omega for the whole orbit, and with eta_s =
    sqrt(eta) also at the start: dt_A = 0.1 / 707.1 -> 2^-13, dt_B = 0.1 / 88.39 -> 2^-10."""
    pos, vel = [], []
    for cx, d in ((-5.0, 0.01), (5.0, 0.04)):
        w = math.sqrt(0.5 / d ** 3)
        pos += [[cx - d / 2, 0, 0], [cx + d / 2, 0, 0]]
        vel += [[0, -w * d / 2, 0], [0, w * d / 2, 0]]
    return np.full(4, 0.25), np.array(pos), np.array(vel)


def test_block_schedule_counts_two_binaries():
    """The scheduler takes exactly the particles that are due: over 2^-6 time units the
    tight binary makes 128 steps and the wide one 16, so there are 128 block steps and
    4 * (2 * 128 + 2 * 16) interactions after the initial 4 * 4."""
    m, pos, vel = _two_binaries()
    st = oracle.State(m, pos, vel)
    steps, inter = oracle.hermite_run(st, 2.0 ** -6, 0.0, eta=0.01, eta_s=0.1, dt_max=1.0 / 16)
    np.testing.assert_array_equal(st.dt, [2.0 ** -13] * 2 + [2.0 ** -10] * 2)
    assert steps == 128
    assert inter == 16 + 4 * (2 * 128 + 2 * 16)


# ---- the iterated corrector P(EC)^n -------------------------------------------

def _kepler_setup(nper):
    e, d = 0.5, 0.5
    a = d / (1 - e)
    m, pos, vel = _two_body(d, e_frac=e)
    return m, pos, vel, 2 * math.pi * a ** 1.5 / nper, a, e


def _kepler_error_corr(nper, n_corr):
    m, pos, vel, dt, a, e = _kepler_setup(nper)
    n = nper // 3
    st = oracle.State(m, pos, vel)
    steps, inter = oracle.hermite_run(st, math.inf, 0.0, dt_shared=dt, max_steps=n,
                                      n_corr=n_corr)
    assert inter == n_corr * n * 4 + 4      # every iteration is a full evaluation, plus init
    rel = st.pos[1] - st.pos[0]
    return np.abs(rel - _kepler_position(n * dt, a, e)).max()


def test_iterated_corrector_order_and_accuracy():
    """P(EC)^2 stays 4th order (error / 16 when dt halves) and is about twice as accurate
    as PEC on the e = 0.5 Kepler orbit; one iteration is PEC."""
    pec = _kepler_error_corr(768, 1)
    assert pec == _kepler_error(768)
    e1 = _kepler_error_corr(768, 2)
    e2 = _kepler_error_corr(1536, 2)
    assert 14.0 < e1 / e2 < 18.0
    assert e1 < 0.7 * pec


def _reversal_error(n_corr, nper=256, periods=3):
    """Integrate forward, reverse the velocities, integrate back: the distance to the start."""
    m, pos, vel, dt, _, _ = _kepler_setup(nper)
    n = nper * periods
    st = oracle.State(m, pos, vel)
    oracle.hermite_run(st, math.inf, 0.0, dt_shared=dt, max_steps=n, n_corr=n_corr)
    back = oracle.State(m, st.pos.copy(), -st.vel.copy())
    oracle.hermite_run(back, math.inf, 0.0, dt_shared=dt, max_steps=n, n_corr=n_corr)
    return np.abs(back.pos - pos).max()


def test_iterated_corrector_approaches_time_symmetry():
    """The iterations converge to the time-symmetric (implicit) Hermite scheme: every
    iteration shrinks the forward-backward return error by orders of magnitude."""
    r1, r2, r3 = (_reversal_error(k) for k in (1, 2, 3))
    assert r1 > 1e-5
    assert r2 < 1e-3 * r1
    assert r3 < 1e-2 * r2


def test_iterated_corrector_block_steps_energy():
    """Block steps with P(EC)^2 on a 256-particle Plummer sphere: synchronised at the end,
    and a smaller energy drift than PEC over the same 1/8 time unit."""
    p = ic.plummer(256, 5)
    eps2 = (1.0 / 64) ** 2
    e0 = _energy_of(p.m, p.pos, p.vel, eps2)
    drifts = []
    for nc in (1, 2):
        st = oracle.State(p.m, p.pos, p.vel)
        oracle.hermite_run(st, 0.125, eps2, eta=0.02, dt_max=1.0 / 16, n_corr=nc)
        np.testing.assert_array_equal(st.t, 0.125)
        drifts.append(abs(_energy_of(p.m, st.pos, st.vel, eps2) - e0) / abs(e0))
    assert drifts[1] < drifts[0]


def _energy_of(m, pos, vel, eps2):
    k, w = oracle.energy(m, pos, vel, eps2)
    return k + w
