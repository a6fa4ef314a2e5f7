"""Pins of the oracle's force routine against facts fixed outside the oracle.

Each pin is chosen so that a plausible slip (a dropped term, a wrong sign,
a wrong power of the distance, a transposed operand, a missing factor 3 in
the jerk) fails at least one of them:
- hand-worked two-body values (tests/golden/two_body.json);
- exact symmetric configurations (cube vertices, equilateral triangle);
- Newton's third law: sum m a = sum m jerk = 0 for the full set;
- acc = -grad(pot) by central differences;
- jerk = d(acc)/dt along straight-line motion, by central differences;
- rigid rotation (jerk = omega x acc) and homologous expansion without
  softening (jerk = -2 H acc);
- the pairwise potential energy (a different summation of the same quantity);
- brute force in 50-digit arithmetic on tiny N.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_body.json")


def _eps2(case):
    return case.get("eps2", case["eps"] ** 2)


@pytest.mark.parametrize("ci", range(3))
def test_two_body_closed_forms(ci):
    case = json.load(open(GOLDEN))["cases"][ci]
    acc, jerk, pot = oracle.force(case["m"], case["pos"], case["vel"], _eps2(case))
    np.testing.assert_allclose(acc, case["acc"], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(jerk, case["jerk"], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(pot, case["pot"], rtol=1e-15)


def test_external_i_set_matches_member_case():
    """force_ext on a copy of particle 0 equals force on member 0 once the j-copy of 0 is
    dropped (Sect. III.A: the i-set may be disjoint from the j-set)."""
    case = json.load(open(GOLDEN))["cases"][0]
    m = np.array(case["m"])
    pos = np.array(case["pos"])
    vel = np.array(case["vel"])
    acc, jerk, pot = oracle.force_ext(m[1:], pos[1:], vel[1:], 0.0, pos[:1], vel[:1])
    np.testing.assert_allclose(acc[0], case["acc"][0], rtol=1e-15)
    np.testing.assert_allclose(jerk[0], case["jerk"][0], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(pot[0], case["pot"][0], rtol=1e-15)


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_cube_vertices(eps):
    """8 unit masses on the unit cube: by symmetry the force on the vertex at the origin
    is (c, c, c), with 3 edge, 3 face-diagonal and 1 body-diagonal neighbours."""
    pos = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    m = np.ones(8)
    vel = np.zeros((8, 3))
    e2 = eps * eps
    c = 1.0 / (1 + e2) ** 1.5 + 2.0 / (2 + e2) ** 1.5 + 1.0 / (3 + e2) ** 1.5
    p = -(3.0 / math.sqrt(1 + e2) + 3.0 / math.sqrt(2 + e2) + 1.0 / math.sqrt(3 + e2))
    acc, jerk, pot = oracle.force(m, pos, vel, e2)
    # vertex 0 at the origin pulls toward the centre (+,+,+)
    np.testing.assert_allclose(acc[0], [c, c, c], rtol=1e-15)
    # every vertex: magnitude equal, direction toward the centre
    toward = 0.5 - pos
    np.testing.assert_allclose(acc, 2 * c * toward, rtol=1e-14)
    np.testing.assert_allclose(pot, np.full(8, p), rtol=1e-15)
    np.testing.assert_array_equal(jerk, 0.0)


def test_equilateral_triangle():
    """Unit masses on a unit equilateral triangle: |acc| = 2 cos(30 deg) = sqrt(3),
    pointing at the centroid; pot = -2."""
    pos = np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]])
    acc, jerk, pot = oracle.force(np.ones(3), pos, np.zeros((3, 3)), 0.0)
    centroid = pos.mean(axis=0)
    for i in range(3):
        d = centroid - pos[i]
        np.testing.assert_allclose(acc[i], math.sqrt(3) * d / np.linalg.norm(d), rtol=1e-14,
                                   atol=1e-15)
    np.testing.assert_allclose(pot, -2.0, rtol=1e-15)


def _random_system(n, seed, spread=1.0):
    p = ic.plummer(n, seed, masses="lognormal")
    return p.m, p.pos * spread, p.vel


@pytest.mark.parametrize("eps2", [0.0, 1e-2])
def test_newton_third_law(eps2):
    m, pos, vel = _random_system(257, 11)
    acc, jerk, pot = oracle.force(m, pos, vel, eps2)
    scale_a = np.abs(m[:, None] * acc).sum()
    scale_j = np.abs(m[:, None] * jerk).sum()
    assert np.abs((m[:, None] * acc).sum(axis=0)).max() < 1e-14 * scale_a
    assert np.abs((m[:, None] * jerk).sum(axis=0)).max() < 1e-14 * scale_j


@pytest.mark.parametrize("eps2", [0.0, 1e-2])
def test_pot_matches_pairwise_energy(eps2):
    m, pos, vel = _random_system(200, 12)
    _, _, pot = oracle.force(m, pos, vel, eps2)
    _, w = oracle.energy(m, pos, vel, eps2)
    assert abs(0.5 * np.dot(m, pot) - w) < 1e-13 * abs(w)


@pytest.mark.parametrize("eps2", [0.0, 2e-2])
def test_acc_is_minus_grad_pot(eps2):
    """a_i = -d pot_i / d x_i, checked by central differences on particle i alone."""
    m, pos, vel = _random_system(24, 13)
    acc, _, _ = oracle.force(m, pos, vel, eps2)
    h = 1e-5
    for i in (0, 7, 23):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, c] += h
            pm[i, c] -= h
            fp = oracle.force(m, pp, vel, eps2, idx=[i])[2][0]
            fm = oracle.force(m, pm, vel, eps2, idx=[i])[2][0]
            grad = (fp - fm) / (2 * h)
            assert abs(-grad - acc[i, c]) < 1e-7 * (1 + abs(acc[i, c]))


@pytest.mark.parametrize("eps2", [0.0, 2e-2])
def test_jerk_is_time_derivative_of_acc(eps2):
    """jerk_i = d a_i / dt when every particle moves on a straight line x + v t."""
    m, pos, vel = _random_system(32, 14)
    _, jerk, _ = oracle.force(m, pos, vel, eps2)
    h = 1e-5
    ap = oracle.force(m, pos + h * vel, vel, eps2)[0]
    am = oracle.force(m, pos - h * vel, vel, eps2)[0]
    fd = (ap - am) / (2 * h)
    np.testing.assert_allclose(jerk, fd, rtol=1e-6, atol=1e-6 * np.abs(jerk).max())


def test_rigid_rotation_jerk():
    """Rigid rotation v = omega x x: the configuration turns without deforming, so every
    acceleration turns with it and jerk = omega x acc (any softening)."""
    m, pos, _ = _random_system(64, 15)
    omega = np.array([0.3, -0.7, 1.1])
    vel = np.cross(omega[None, :], pos) + np.array([0.2, 0.1, -0.4])
    for eps2 in (0.0, 1e-2):
        acc, jerk, _ = oracle.force(m, pos, vel, eps2)
        np.testing.assert_allclose(jerk, np.cross(omega[None, :], acc), rtol=1e-11,
                                   atol=1e-12 * np.abs(jerk).max())


def test_homologous_expansion_jerk():
    """v = H x without softening: every separation scales as (1 + H t), so |a| ~ 1/s^2 and
    jerk = -2 H acc exactly. (A missing or wrong factor 3 in the radial term breaks this.)"""
    m, pos, _ = _random_system(64, 16)
    hub = 0.37
    acc, jerk, _ = oracle.force(m, pos, hub * pos, 0.0)
    np.testing.assert_allclose(jerk, -2 * hub * acc, rtol=1e-12, atol=1e-13 * np.abs(acc).max())


def test_brute_force_50_digits():
    """Tiny N recomputed pair by pair in 50-digit arithmetic (mpmath)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    m, pos, vel = _random_system(7, 17)
    eps2 = 1e-3
    acc, jerk, pot = oracle.force(m, pos, vel, eps2, idx=[0, 3, 6, 3])
    for k, i in enumerate([0, 3, 6, 3]):
        a = [mp.mpf(0)] * 3
        jk = [mp.mpf(0)] * 3
        sa = [mp.mpf(0)] * 3   # sums of |term|: the scale a binary64 sum is accurate to
        sj = [mp.mpf(0)] * 3
        p = mp.mpf(0)
        for j in range(7):
            if j == i:
                continue
            r = [mp.mpf(pos[j, c]) - mp.mpf(pos[i, c]) for c in range(3)]
            v = [mp.mpf(vel[j, c]) - mp.mpf(vel[i, c]) for c in range(3)]
            s2 = sum(x * x for x in r) + mp.mpf(eps2)
            rv = sum(r[c] * v[c] for c in range(3))
            mj = mp.mpf(m[j])
            for c in range(3):
                ta = mj * r[c] / s2 ** mp.mpf(1.5)
                tj = mj * (v[c] / s2 ** mp.mpf(1.5) - 3 * rv * r[c] / s2 ** mp.mpf(2.5))
                a[c] += ta
                jk[c] += tj
                sa[c] += abs(ta)
                sj[c] += abs(mj * v[c] / s2 ** mp.mpf(1.5)) + abs(3 * mj * rv * r[c] / s2 ** mp.mpf(2.5))
            p -= mj / mp.sqrt(s2)
        for c in range(3):
            assert abs(acc[k, c] - float(a[c])) <= 1e-15 * float(sa[c])
            assert abs(jerk[k, c] - float(jk[c])) <= 1e-15 * float(sj[c])
        assert abs(pot[k] - float(p)) <= 1e-15 * abs(float(p))


def test_single_particle_and_empty():
    acc, jerk, pot = oracle.force([1.0], [[0.1, 0.2, 0.3]], [[0, 0, 0]], 0.0)
    np.testing.assert_array_equal(acc, 0.0)
    np.testing.assert_array_equal(jerk, 0.0)
    np.testing.assert_array_equal(pot, 0.0)
    acc, jerk, pot = oracle.force([1.0, 1.0], [[0, 0, 0], [1, 0, 0]], np.zeros((2, 3)), 0.0,
                                  idx=np.zeros(0, dtype=np.int32))
    assert acc.shape == (0, 3) and pot.shape == (0,)


def test_massless_particles_feel_but_do_not_pull():
    m, pos, vel = _random_system(16, 18)
    m0 = m.copy()
    m0[5] = 0.0
    acc0, jerk0, pot0 = oracle.force(m0, pos, vel, 1e-3)
    others = [i for i in range(16) if i != 5]
    acc1, jerk1, pot1 = oracle.force(m[others], pos[others], vel[others], 1e-3)
    np.testing.assert_allclose(acc0[others], acc1, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(pot0[others], pot1, rtol=1e-14)
    assert np.abs(acc0[5]).sum() > 0
