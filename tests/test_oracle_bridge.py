"""Pins of the oracle's bridge (Sect. V: a kick-drift-kick split of the Hamiltonian into
two systems and their interaction): the kick against a closed form, exact momentum
conservation, the decoupled limit, and 2nd-order convergence to a direct integration of
the combined system."""
import math

import numpy as np

import oracle


def _binary(cx, vy, d=0.02, m=0.25):
    """A circular binary of two masses m at separation d, centre (cx, 0, 0) moving with vy."""
    w = math.sqrt(2 * m / d ** 3)
    pos = np.array([[cx - d / 2, 0, 0], [cx + d / 2, 0, 0]])
    vel = np.array([[0, vy - w * d / 2, 0], [0, vy + w * d / 2, 0]])
    return np.array([m, m]), pos, vel


def _two_binaries(sep=1.0):
    """Two binaries of mass 0.5 each on a mutual circular orbit of separation sep."""
    v = 0.5 * math.sqrt(1.0 / sep)
    return _binary(-sep / 2, -v), _binary(sep / 2, v)


EPS2 = 1e-4 ** 2
SHARED = 1.0 / 8192


def test_kick_closed_form():
    """A particle at distance 2 from a unit point mass: dv = -dt M r / (r^2 + eps^2)^1.5,
    and its own acc/jerk re-evaluated (zero for a single particle)."""
    st = oracle.State([1e-3], [[2.0, 0, 0]], [[0, 0.1, 0]], acc=[[9, 9, 9]], jerk=[[9, 9, 9]])
    field = oracle.State([1.0], [[0, 0, 0]], [[0, 0, 0]])
    oracle.kick(st, field, 0.09, 0.0, 0.5)
    expect = -0.5 * 1.0 * 2.0 / (4.0 + 0.09) ** 1.5
    assert abs(st.vel[0, 0] - expect) < 1e-16
    assert st.vel[0, 1] == 0.1 and st.vel[0, 2] == 0.0
    assert not st.acc.any() and not st.jerk.any()


def _bridge(dt, t_end, sep=1.0):
    (ma, xa, va), (mb, xb, vb) = _two_binaries(sep)
    sa, sb = oracle.State(ma, xa, va), oracle.State(mb, xb, vb)
    oracle.bridge_run(sa, sb, EPS2, EPS2, dt, int(round(t_end / dt)), dt_shared=SHARED)
    return sa, sb


def _centres(m, pos):
    return (m[:, None] * pos).sum(0) / m.sum()


def test_bridge_second_order_against_direct_integration():
    t_end = 0.5
    (ma, xa, va), (mb, xb, vb) = _two_binaries()
    ref = oracle.State(np.concatenate([ma, mb]), np.concatenate([xa, xb]),
                       np.concatenate([va, vb]))
    oracle.hermite_run(ref, t_end, EPS2, dt_shared=SHARED)
    rca, rcb = _centres(ref.m[:2], ref.pos[:2]), _centres(ref.m[2:], ref.pos[2:])
    errs = []
    for dt in (1.0 / 8, 1.0 / 16, 1.0 / 32):
        sa, sb = _bridge(dt, t_end)
        errs.append(max(np.abs(_centres(sa.m, sa.pos) - rca).max(),
                        np.abs(_centres(sb.m, sb.pos) - rcb).max()))
    assert errs[-1] < 1e-4
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.0 < e1 / e2 < 5.5      # 2nd order: error / 4 when dt halves


def test_bridge_conserves_total_momentum():
    """The kicks are mutual (same softening both ways) and shared-step Hermite conserves
    each system's own momentum: the total momentum stays at its start value to rounding."""
    (ma, xa, va), (mb, xb, vb) = _two_binaries()
    p0 = (ma[:, None] * va).sum(0) + (mb[:, None] * vb).sum(0)
    sa, sb = _bridge(1.0 / 16, 0.25)
    p1 = (sa.m[:, None] * sa.vel).sum(0) + (sb.m[:, None] * sb.vel).sum(0)
    assert np.abs(p1 - p0).max() < 1e-15


def test_bridge_decoupled_limit():
    """Systems 1e6 apart: the kicks are ~1e-12 of the internal accelerations, so each
    system's centre of mass stays put and its internal motion is its own integration's
    (up to the Hermite restart after each kick, which re-evaluates acc and jerk at the
    corrected rather than the predicted state: a truncation-level difference)."""
    (ma, xa, va), (mb, xb, vb) = _binary(-5e5, 0.0), _binary(5e5, 0.0)
    sa, sb = oracle.State(ma, xa, va), oracle.State(mb, xb, vb)
    oracle.bridge_run(sa, sb, EPS2, EPS2, 1.0 / 16, 2, dt_shared=SHARED)
    for m, x, v, got in ((ma, xa, va, sa), (mb, xb, vb, sb)):
        alone = oracle.State(m, x, v)
        oracle.hermite_run(alone, 1.0 / 8, EPS2, dt_shared=SHARED)
        assert np.abs(_centres(got.m, got.pos) - _centres(m, x)).max() < 1e-9
        assert np.abs(got.pos - alone.pos).max() < 1e-7
