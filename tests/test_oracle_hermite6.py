"""Pins of the oracle's 6th-order Hermite scheme (acc, jerk and snap per pair; the
two-point Hermite corrector of order 6; the generalised step criterion).

Facts used (none of them is the oracle's own formula typed again):
- jerk and snap are the first and second time derivatives of the acceleration along
  the motion: 5-point finite differences of the 4th-order force routine (a separate
  pair routine) along polynomial trajectories;
- Newton's third law for the snap (sum m_i snap_i = 0);
- uniform circular motion: snap = -omega^2 acc with the softened two-body omega;
- the predictor is exact for quintic trajectories; the corrector is exact for sextic
  ones and its velocity quadrature has the error constant h^7/140 on a = t^6;
- the block step of a circular orbit: Aarseth's criterion on (a, jerk, snap, crackle)
  with the closed-form derivatives of uniform circular motion, and with the crackle
  under a rounding floor;
- 6th-order convergence on the softened circular orbit and the Kepler ellipse
  (Kepler's equation), energy convergence;
- dyadic block times, resume = uninterrupted, forced-equal block steps = shared steps.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic


def _rel(got, ref):
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_force6_matches_the_4th_order_routine():
    p = ic.plummer(200, 61, masses="lognormal")
    rng = np.random.default_rng(61)
    aj = rng.normal(size=(200, 3))
    a, j, s, pot = oracle.force6(p.m, p.pos, p.vel, aj, 1e-4)
    a4, j4, pot4 = oracle.force(p.m, p.pos, p.vel, 1e-4)
    np.testing.assert_allclose(a, a4, rtol=1e-13, atol=1e-13 * np.abs(a4).max())
    np.testing.assert_allclose(j, j4, rtol=1e-13, atol=1e-13 * np.abs(j4).max())
    np.testing.assert_allclose(pot, pot4, rtol=1e-14)


def _trajectory(seed, n=7):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, 3))
    v = rng.normal(size=(n, 3))
    a = rng.normal(size=(n, 3))
    jk = rng.normal(size=(n, 3))
    m = rng.uniform(0.5, 1.5, size=n)
    return m, x, v, a, jk


def test_jerk_and_snap_are_time_derivatives_of_acc():
    """Each particle moves on x(t) = x + v t + a t^2/2 + j t^3/6; the acceleration of
    particle i from the others, acc_i(t), is differentiated numerically at t = 0
    (5-point stencils, error O(h^4)). Its first derivative is the jerk with the
    velocities v, its second the snap with the accelerations a."""
    m, x, v, a, jk = _trajectory(62)
    eps2 = 0.2 ** 2
    h = 2.5e-4

    def acc_at(t):
        pos = x + v * t + a * t * t / 2 + jk * t ** 3 / 6
        vel = v + a * t + jk * t * t / 2
        return oracle.force(m, pos, vel, eps2)[0]

    f = {k: acc_at(k * h) for k in (-2, -1, 0, 1, 2)}
    d1 = (f[-2] - 8 * f[-1] + 8 * f[1] - f[2]) / (12 * h)
    d2 = (-f[-2] + 16 * f[-1] - 30 * f[0] + 16 * f[1] - f[2]) / (12 * h * h)
    acc, jerk, snap, _ = oracle.force6(m, x, v, a, eps2)
    assert _rel(jerk, d1) < 1e-8
    assert _rel(snap, d2) < 1e-8
    # the snap really depends on the accelerations (it is not the a = 0 value)
    _, _, snap0, _ = oracle.force6(m, x, v, np.zeros_like(a), eps2)
    assert _rel(snap0, d2) > 1e-2


def test_snap_newton_third_law():
    p = ic.plummer(300, 63, masses="lognormal")
    aj = oracle.force(p.m, p.pos, p.vel, 1e-3)[0]
    _, _, snap, _ = oracle.force6(p.m, p.pos, p.vel, aj, 1e-3)
    tot = (p.m[:, None] * snap).sum(axis=0)
    scale = (p.m[:, None] * np.abs(snap)).sum()
    assert np.abs(tot).max() < 1e-13 * scale


def test_circular_orbit_snap_closed_form():
    """Uniform circular motion at angular rate omega: acc = -omega^2 x,
    jerk = -omega^2 v, snap = -omega^2 acc (softened two-body omega^2 = M / (d^2 +
    eps^2)^(3/2), equal masses 1/2 about the centre of mass)."""
    d, eps = 0.8, 0.25
    omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
    th = 0.7
    u = np.array([math.cos(th), math.sin(th), 0.0])
    w = np.array([-math.sin(th), math.cos(th), 0.0])
    pos = np.array([-d / 2 * u, d / 2 * u])
    vel = np.array([-d / 2 * omega * w, d / 2 * omega * w])
    m = np.array([0.5, 0.5])
    acc_true = -omega ** 2 * pos
    acc, jerk, snap, _ = oracle.force6(m, pos, vel, acc_true, eps * eps)
    np.testing.assert_allclose(acc, acc_true, atol=1e-15)
    np.testing.assert_allclose(jerk, -omega ** 2 * vel, atol=1e-15)
    np.testing.assert_allclose(snap, -omega ** 2 * acc_true, atol=1e-14)


def _poly(c):
    def deriv(t, d):
        out = 0.0
        for k in range(d, len(c)):
            out += c[k] * math.factorial(k) / math.factorial(k - d) * t ** (k - d)
        return out
    return deriv


def test_predictor6_exact_for_quintic():
    x = _poly([0.3, -1.1, 0.7, 2.0, -1.5, 0.9])
    t0, t1 = 0.25, 0.75
    ins = [np.full((1, 3), x(t0, d)) for d in range(6)]
    pp, vp, ap = oracle.predict6(t1, [t0], *ins)
    np.testing.assert_allclose(pp, x(t1, 0), rtol=1e-14)
    np.testing.assert_allclose(vp, x(t1, 1), rtol=1e-14)
    np.testing.assert_allclose(ap, x(t1, 2), rtol=1e-14)


def _correct_poly(c, dt):
    x = _poly(c)
    s0 = [np.full(3, x(0.0, d)) for d in range(5)]
    s1 = [np.full(3, x(dt, d)) for d in (2, 3, 4)]
    return x, oracle.correct6_one(dt, *s0, *s1)


def test_corrector6_exact_for_sextic():
    """x(t) of degree 6: a(t) is quartic, inside the quintic the corrector integrates
    exactly, so x1, v1 and the end-of-step 3rd-5th derivatives are exact."""
    dt = 0.125
    x, (x1, v1, a3, a4, a5) = _correct_poly([0.3, -1.1, 0.7, 2.0, -1.5, 0.9, 1.3], dt)
    np.testing.assert_allclose(x1, x(dt, 0), rtol=1e-14)
    np.testing.assert_allclose(v1, x(dt, 1), rtol=1e-14)
    np.testing.assert_allclose(a3, x(dt, 5), rtol=1e-10)
    np.testing.assert_allclose(a4, x(dt, 6), rtol=1e-10)
    np.testing.assert_allclose(a5, x(dt, 7), atol=1e-7)
    # degree 7 (quintic a): v1 and the interpolated derivatives are still exact
    x, (x1, v1, a3, a4, a5) = _correct_poly([0.3, -1.1, 0.7, 2.0, -1.5, 0.9, 1.3, -0.6], dt)
    np.testing.assert_allclose(v1, x(dt, 1), rtol=1e-14)
    np.testing.assert_allclose(a3, x(dt, 5), rtol=1e-9)
    np.testing.assert_allclose(a4, x(dt, 6), rtol=1e-9)
    np.testing.assert_allclose(a5, x(dt, 7), rtol=1e-9)


def test_corrector6_error_constant():
    """a(t) = t^6 (x = t^8 / 56): the velocity quadrature over [0, h] gives
    h^7 (1/2 - 6/10 + 30/120) = h^7 (1/7 + 1/140), i.e. an error of exactly h^7/140."""
    h = 0.5
    c = [0.0] * 8 + [1.0 / 56.0]
    x, (x1, v1, *_) = _correct_poly(c, h)
    assert v1[0] - x(h, 1) == pytest.approx(h ** 7 / 140.0, rel=1e-12)


def _two_body(d, e_frac=0.0, eps=0.0):
    if e_frac == 0.0:
        omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
        vrel = omega * d
    else:
        a = d / (1 - e_frac)
        vrel = math.sqrt((1 + e_frac) / (a * (1 - e_frac)))
    pos = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    vel = np.array([[0, -vrel / 2, 0], [0, vrel / 2, 0]])
    return np.array([0.5, 0.5]), pos, vel


def test_block6_circular_orbit_step_choice():
    """Uniform circular motion at rate omega has |jerk| = omega |a|, |snap| = omega^2 |a|,
    |crackle| = omega^3 |a|, so Aarseth's criterion on (a, jerk, snap, crackle) gives
    dt = sqrt(eta) / omega: with eta = 4e-4, d = 0.5, eps = 0.1 that is 0.00728, whose
    block step is 2^-8 (reached from the start-up step by doubling)."""
    d, eps = 0.5, 0.1
    m, pos, vel = _two_body(d, eps=eps)
    omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
    assert 2.0 ** -8 <= 0.02 / omega < 2.0 ** -7
    st = oracle.State6(m, pos, vel)
    oracle.hermite6_run(st, 1.0, eps * eps, eta=4e-4, eta_s=0.01, dt_max=1.0, max_steps=20000)
    np.testing.assert_array_equal(st.t, 1.0)
    np.testing.assert_array_equal(st.dt, 2.0 ** -8)
    # a rounding floor above the crackle (noise 1e-6: 30 noise |a| / T^3 >> omega^3 |a|)
    # leaves dt^2 = eta (|a||s| + |j|^2) / |s|^2 = 2 eta / omega^2: one level up
    assert 2.0 ** -7 <= math.sqrt(2 * 4e-4) / omega < 2.0 ** -6
    sf = oracle.State6(m, pos, vel)
    oracle.hermite6_run(sf, 1.0, eps * eps, eta=4e-4, eta_s=0.01, dt_max=1.0, max_steps=20000,
                        noise=1e-6)
    np.testing.assert_array_equal(sf.dt, 2.0 ** -7)
    # the start-up step eta_s |a| / |jerk| = 0.01 / omega lies one level lower
    assert 2.0 ** -9 <= 0.01 / omega < 2.0 ** -8
    st0 = oracle.State6(m, pos, vel)
    oracle.hermite6_run(st0, 0.0, eps * eps, eta=4e-4, eta_s=0.01, dt_max=1.0)
    np.testing.assert_array_equal(st0.dt, 2.0 ** -9)


def _run6_shared(m, pos, vel, eps2, dt, nsteps):
    st = oracle.State6(m, pos, vel)
    steps, _ = oracle.hermite6_run(st, math.inf, eps2, dt_shared=dt, max_steps=nsteps)
    assert steps == nsteps
    return st


def _circular_error6(nsteps):
    d, eps = 1.0, 0.3
    m, pos, vel = _two_body(d, eps=eps)
    omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
    st = _run6_shared(m, pos, vel, eps * eps, 2 * math.pi / omega / nsteps, nsteps)
    return np.abs(st.pos - pos).max()


def test_circular_orbit_sixth_order():
    e1, e2 = _circular_error6(32), _circular_error6(64)
    assert e2 < 1e-7
    assert 50.0 < e1 / e2 < 80.0   # 6th order: error / 64


def _kepler_position(t, a, e):
    mean = t / a ** 1.5
    ea = mean
    for _ in range(50):
        ea -= (ea - e * math.sin(ea) - mean) / (1 - e * math.cos(ea))
    return np.array([a * (math.cos(ea) - e), a * math.sqrt(1 - e * e) * math.sin(ea), 0.0])


def _kepler_error6(nsteps_per_period):
    e, d = 0.5, 0.5
    a = d / (1 - e)
    m, pos, vel = _two_body(d, e_frac=e)
    period = 2 * math.pi * a ** 1.5
    n = nsteps_per_period // 3
    dt = period / nsteps_per_period
    st = _run6_shared(m, pos, vel, 0.0, dt, n)
    return np.abs(st.pos[1] - st.pos[0] - _kepler_position(n * dt, a, e)).max()


def test_kepler_ellipse_sixth_order():
    e1, e2 = _kepler_error6(384), _kepler_error6(768)
    assert e2 < 2e-10
    assert 50.0 < e1 / e2 < 80.0


def test_energy_convergence_order6():
    """Energy error over a fixed interval falls by more than 2^6 per halving of dt."""
    p = ic.plummer(16, 25)
    eps2 = 0.05 ** 2

    def energy(st):
        k, w = oracle.energy(st.m, st.pos, st.vel, eps2)
        return k + w

    e0 = energy(oracle.State(p.m, p.pos, p.vel))
    errs = [abs(energy(_run6_shared(p.m, p.pos, p.vel, eps2, 0.5 / n, n)) - e0)
            for n in (64, 128)]
    assert errs[0] / errs[1] > 60.0


def test_block6_times_dyadic_and_resume():
    p = ic.plummer(96, 64)
    eps2 = 1e-3
    a = oracle.State6(p.m, p.pos, p.vel)
    steps, inter = oracle.hermite6_run(a, 0.125, eps2, eta=0.02, max_steps=20000)
    np.testing.assert_array_equal(a.t, 0.125)
    lg = np.log2(a.dt)
    np.testing.assert_array_equal(lg, np.round(lg))
    np.testing.assert_array_equal(np.fmod(a.t, a.dt), 0.0)
    assert len(np.unique(a.dt)) > 1 and steps > 4
    b = oracle.State6(p.m, p.pos, p.vel)
    oracle.hermite6_run(b, 1.0 / 16, eps2, eta=0.02, max_steps=20000)
    c = oracle.State6(b.m, b.pos, b.vel, acc=b.acc, jerk=b.jerk, snap=b.snap,
                      crackle=b.crackle, t=b.t, dt=b.dt)
    oracle.hermite6_run(c, 0.125, eps2, eta=0.02, max_steps=20000)
    np.testing.assert_array_equal(a.pos, c.pos)
    np.testing.assert_array_equal(a.vel, c.vel)


def test_block6_equal_steps_equal_shared_steps():
    p = ic.plummer(64, 24)
    dt = 1.0 / 256
    a = _run6_shared(p.m, p.pos, p.vel, 1e-3, dt, 16)
    b = oracle.State6(p.m, p.pos, p.vel)
    steps, _ = oracle.hermite6_run(b, 16 * dt, 1e-3, eta=0.02, dt_min=dt, dt_max=dt)
    assert steps == 16
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.vel, b.vel)


def test_plummer_block6_energy_beats_4th_order():
    """N = 256 Plummer to t = 1/4 with block steps: the 6th-order scheme at eta = 0.02
    spends fewer interactions than the 4th-order one at eta = 0.01 and conserves the
    energy better (1.2e-10 against 7.1e-10)."""
    p = ic.plummer(256, 7)
    eps2 = (1.0 / 64) ** 2

    def energy(st):
        k, w = oracle.energy(st.m, st.pos, st.vel, eps2)
        return k + w

    e0 = energy(oracle.State(p.m, p.pos, p.vel))
    s6 = oracle.State6(p.m, p.pos, p.vel)
    _, i6 = oracle.hermite6_run(s6, 0.25, eps2, eta=0.02, eta_s=0.01, max_steps=20000)
    np.testing.assert_array_equal(s6.t, 0.25)
    s4 = oracle.State(p.m, p.pos, p.vel)
    _, i4 = oracle.hermite_run(s4, 0.25, eps2, eta=0.01)
    d6 = abs(energy(s6) - e0) / abs(e0)
    d4 = abs(energy(s4) - e0) / abs(e0)
    assert i6 < i4
    assert d6 < 1e-9 and d6 < d4 / 3
