"""The 6th-order Hermite scheme on the GPU (nb_config.order = 6) against the oracle's
6th-order scheme: the pair force with snap at several tiles and a ragged tail (F32-DS,
F64), shared and block steps, energy, checkpoint / resume, and the argument checks."""
import math

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic
from tests.errstats import fmt, report

pytestmark = pytest.mark.gpu


def _rel_rms(got, ref):
    return np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())


# force gates (relative RMS over the i-set): acc, jerk, snap, pot
GATES = {"f32ds": (1e-6, 2e-6, 1e-6, 1e-6), "f64": (1e-12, 1e-11, 1e-10, 1e-12)}
# per-particle maximum of |d_i| / |ref_i|: acc, jerk, snap, pot (3-15x the largest value
# measured here on GB300: F32-DS 4.7e-7 / 1.9e-6 / 6.4e-6 / 2.0e-7, FP64 9.1e-15 / 2.1e-14
# / 7.3e-14 / 8.7e-16)
PP_GATES = {"f32ds": (1e-5, 1e-4, 1e-4, 2e-6), "f64": (1e-13, 3e-13, 1e-12, 1e-14)}


def _gate6(variant, got, ref, tag=None):
    """RMS and per-particle maximum gates of (acc, jerk, snap, pot) against the oracle."""
    names = ("acc", "jerk", "snap", "pot")
    rep = report({q: (g.T if g.ndim == 2 else g, r) for q, g, r in zip(names, got, ref)})
    print(variant, tag, fmt(rep))
    for q, g_rms, g_max in zip(names, GATES[variant], PP_GATES[variant]):
        assert rep[q][0] < g_rms, (variant, tag, q, rep[q])
        assert rep[q][1] < g_max, (variant, tag, q, rep[q])


def _predicted_oracle_state(s, t):
    """The oracle's prediction of the GPU system's state (and snap, crackle) to t."""
    g = s.state()
    snap, crk = s.snap()
    return oracle.predict6(t, g["t"], g["pos"].T, g["vel"].T, g["acc"].T, g["jerk"].T,
                           snap.T, crk.T), g["m"]


@pytest.mark.parametrize("variant", ["f32ds", "f64"])
def test_force_snap_matches_oracle(nb, variant):
    """N = 3000 (23 full j-tiles of 128 and a ragged one), lognormal masses: one block
    step taken so that accelerations, snap and crackle are non-trivial, then the
    predicted state at a later time; a ragged i-set with duplicates against the oracle."""
    n, eps = 3000, 0.01
    p = ic.plummer(n, 80, masses="lognormal")
    with nb.System(p.m, p.pos, p.vel, variant=variant, eps=eps, eta=0.02, order=6,
                   device=0) as s:
        s.step(1.0 / 64)
        t = 1.0 / 64 + 1.0 / 1024
        s.predict(t)
        rng = np.random.default_rng(81)
        idx = rng.integers(0, n, size=777).astype(np.int32)
        idx[:5] = idx[5]                              # duplicates
        acc, jerk, snap, pot = s.force_snap(idx)
        (pp, vp, ap), m = _predicted_oracle_state(s, t)
    ra, rj, rs, rp = oracle.force6(m, pp, vp, ap, eps * eps, idx)
    _gate6(variant, (acc, jerk, snap, pot), (ra, rj, rs, rp), "N=3000")


def test_force_snap_all_particles_small(nb):
    """Every particle of a small system (fewer than one tile, one i-block)."""
    p = ic.plummer(100, 82)
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=0.02, eta=0.02, eta_s=0.01, order=6,
                   device=0) as s:
        nb.nb_init(s.h)
        s.predict(0.0)
        acc, jerk, snap, pot = s.force_snap()
        g = s.state()
        snap0, crk0 = s.snap()
    ra, rj, rs, rp = oracle.force6(p.m, p.pos, p.vel, g["acc"].T, 0.02 ** 2)
    assert _rel_rms(acc.T, ra) < 1e-6 and _rel_rms(jerk.T, rj) < 1e-5
    assert _rel_rms(snap.T, rs) < 1e-4 and _rel_rms(pot, rp) < 1e-6
    # the handle's start-up (two passes) is the oracle's: acc, jerk, snap, zero crackle
    st = oracle.State6(p.m, p.pos, p.vel)
    oracle.hermite6_run(st, 0.0, 0.02 ** 2, eta=0.02, eta_s=0.01)
    assert _rel_rms(g["acc"].T, st.acc) < 1e-6 and _rel_rms(g["jerk"].T, st.jerk) < 1e-5
    assert _rel_rms(snap0.T, st.snap) < 1e-4
    assert not crk0.any()
    np.testing.assert_array_equal(g["dt"], st.dt)


@pytest.mark.parametrize("variant", ["f64", "f32ds"])
def test_shared_steps_vs_oracle(nb, variant):
    """N = 256, 32 shared steps of 1/256: the oracle's 6th-order state."""
    p = ic.plummer(256, 83)
    eps, dt = 1.0 / 64, 1.0 / 256
    st = oracle.State6(p.m, p.pos, p.vel)
    _, o_inter = oracle.hermite6_run(st, 32 * dt, eps * eps, dt_shared=dt)
    with nb.System(p.m, p.pos, p.vel, variant=variant, eps=eps, shared_dt=dt, order=6,
                   device=0) as s:
        stats = s.step(32 * dt)
        g = s.state()
        snap, crk = s.snap()
    assert stats["interactions"] == o_inter     # two start-up passes + 32 steps
    tol = (1e-11, 1e-10) if variant == "f64" else (1e-6, 1e-5)
    assert np.abs(g["pos"].T - st.pos).max() < tol[0]
    assert np.abs(g["vel"].T - st.vel).max() < tol[1]
    assert _rel_rms(snap.T, st.snap) < (1e-9 if variant == "f64" else 1e-4)
    assert _rel_rms(crk.T, st.crackle) < (1e-7 if variant == "f64" else 1e-2)


@pytest.mark.parametrize("variant", ["f64", "f32ds"])
def test_block_steps_vs_oracle(nb, variant):
    """Block steps (eta = 0.02) over 1/16 time unit: the oracle's schedule (FP64 pairs:
    the same block-step count) and state."""
    p = ic.plummer(512, 84)
    eps = 0.01
    st = oracle.State6(p.m, p.pos, p.vel)
    # the crackle's rounding floor of the double-single pairs (2^-23), none for FP64
    noise = 2.0 ** -23 if variant == "f32ds" else 0.0
    o_steps, o_inter = oracle.hermite6_run(st, 1.0 / 16, eps * eps, eta=0.02, eta_s=0.01,
                                           dt_max=1.0 / 16, noise=noise)
    with nb.System(p.m, p.pos, p.vel, variant=variant, eps=eps, eta=0.02, eta_s=0.01,
                   dt_max=1.0 / 16, order=6, device=0) as s:
        stats = s.step(1.0 / 16)
        g = s.state()
    np.testing.assert_array_equal(g["t"], 1.0 / 16)
    if variant == "f64":
        assert stats["block_steps"] == o_steps
        np.testing.assert_array_equal(g["dt"], st.dt)
        assert np.abs(g["pos"].T - st.pos).max() < 1e-10
    else:
        assert abs(stats["block_steps"] - o_steps) <= 0.02 * o_steps
        assert np.abs(g["pos"].T - st.pos).max() < 1e-5


def test_energy_drift_block_steps(nb):
    """N = 1024 Plummer, eps = 1/64, eta = 0.02, block steps to t = 1/4 in F32-DS."""
    p = ic.plummer(1024, 85)
    eps = 1.0 / 64
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, eta_s=0.01,
                   order=6, device=0) as s:
        k0, w0 = s.energy()
        s.step(0.25)
        k1, w1 = s.energy()
    assert abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0) < 1e-6


def test_close_encounter_steps_recover(nb):
    """N = 65536 Plummer with eps = 1e-3 (close encounters at r < eps) in F32-DS for 1/16
    time unit: no step is clamped at dt_min and the smallest step stays above 2^-20 (without
    the crackle's rounding floor a pair that had met closely kept a step of 2^-30)."""
    p = ic.plummer(65536, ic.MASTER_SEED, masses="equal")
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=1e-3, eta=0.02, eta_s=0.01,
                   order=6, device=0) as s:
        for k in range(1, 9):
            stats = s.step(k / 128)
            assert stats["dt_min_hits"] == 0, k
            assert s.state()["dt"].min() >= 2.0 ** -20, k


def test_checkpoint_resume_is_bitwise(nb):
    p = ic.plummer(700, 86)
    kw = dict(variant="f32ds", eps=0.01, eta=0.02, order=6, device=0)
    with nb.System(p.m, p.pos, p.vel, **kw) as a:
        a.step(1.0 / 8)
        ga = a.state()
    with nb.System(p.m, p.pos, p.vel, **kw) as b:
        b.step(1.0 / 16)
        gb = b.state()
        snap, crk = b.snap()
    with nb.System(p.m, p.pos, p.vel, **kw) as c:
        c.set_state(gb)
        with pytest.raises(nb.NBodyError) as e:
            c.step(1.0 / 8)
        assert e.value.status == nb.NB_ERR_STATE
        c.set_snap(snap, crk)
        c.step(1.0 / 8)
        gc = c.state()
    for k in ("pos", "vel", "acc", "jerk", "t", "dt"):
        np.testing.assert_array_equal(ga[k], gc[k])


def test_host_calls_equal_step(nb):
    """nb_predict + nb_force_snap + nb_correct on all particles at the shared step
    reproduce nb_step in shared-step mode bitwise."""
    p = ic.plummer(300, 87)
    kw = dict(variant="f32ds", eps=0.02, shared_dt=1.0 / 128, order=6, device=0)
    with nb.System(p.m, p.pos, p.vel, **kw) as a:
        a.step(2.0 / 128)
        ga = a.state()
    with nb.System(p.m, p.pos, p.vel, **kw) as b:
        nb.nb_init(b.h)
        for k in (1, 2):
            t = k / 128
            b.predict(t)
            b.force_snap()
            b.correct(None, t)
        gb = b.state()
    for k in ("pos", "vel", "acc", "jerk"):
        np.testing.assert_array_equal(ga[k], gb[k])


def test_order6_argument_checks(nb):
    p = ic.plummer(64, 88)
    with nb.System(p.m, p.pos, p.vel, eps=0.01, device=0) as s4:
        s4.predict(0.0)
        with pytest.raises(nb.NBodyError) as e:
            s4.force_snap()
        assert e.value.status == nb.NB_ERR_ARG
    for bad in (dict(order=5), dict(order=6, n_corr=2), dict(order=6, variant="f32")):
        with pytest.raises(nb.NBodyError) as e:
            nb.System(p.m, p.pos, p.vel, eps=0.01, device=0, **bad)
        assert e.value.status == nb.NB_ERR_ARG
    with nb.System(p.m, p.pos, p.vel, eps=0.01, order=6, eta=0.02, device=0) as s6:
        for bad in ([(1, 1, 4)], [(0, 3, 2)], [(0, 2, 0)]):   # kind 1, nwj 3, no splits
            with pytest.raises(nb.NBodyError) as e:
                nb.nb_set_plan_table(s6.h, bad)
            assert e.value.status == nb.NB_ERR_ARG
        s6.predict(0.0)
        with pytest.raises(nb.NBodyError) as e:
            s6.force_ext(p.pos[:4], p.vel[:4])
        assert e.value.status == nb.NB_ERR_ARG


def test_single_particle_and_circular_pair(nb):
    """Degenerate sizes: one particle moves on a straight line with dt = dt_max and zero
    derivatives; a softened circular pair in FP64 shared steps follows the oracle's
    6th-order orbit to rounding over one period."""
    m = np.array([1.0])
    pos = np.array([[0.1, -0.2, 0.3]])
    vel = np.array([[0.5, 0.25, -1.0]])
    with nb.System(m, pos, vel, variant="f32ds", eps=0.01, eta=0.02, order=6, device=0) as s:
        s.step(0.5)
        g = s.state()
        snap, crk = s.snap()
    np.testing.assert_allclose(g["pos"].T, pos + 0.5 * vel, rtol=0, atol=1e-15)
    assert g["dt"][0] == 1.0 / 16 and not g["acc"].any() and not snap.any() and not crk.any()
    d, eps = 1.0, 0.3
    omega = math.sqrt(1.0 / (d * d + eps * eps) ** 1.5)
    m2 = np.array([0.5, 0.5])
    p2 = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    v2 = np.array([[0, -omega * d / 2, 0], [0, omega * d / 2, 0]])
    dt = 2 * math.pi / omega / 64
    st = oracle.State6(m2, p2, v2)
    oracle.hermite6_run(st, math.inf, eps * eps, dt_shared=dt, max_steps=64)
    with nb.System(m2, p2, v2, variant="f64", eps=eps, shared_dt=dt, order=6, device=0) as s:
        stats = s.step(64.5 * dt)         # 64 steps: the 65th would end past 64.5 dt
        g = s.state()
    assert stats["block_steps"] == 64
    assert np.abs(g["pos"].T - st.pos).max() < 1e-13
    assert np.abs(g["pos"].T - p2).max() < 1e-6   # back where it started after one period


def test_full_size_h6block65536_sampled(nb):
    """The bench's 6th-order configuration at full size (N = 65536, eps = 1e-3, eta =
    0.02): after 1/64 time unit the snap force on a seeded 512-particle sample of the
    predicted state (positions, velocities, accelerations) against the oracle."""
    p = ic.plummer(65536, ic.MASTER_SEED, masses="equal")
    eps = 1e-3
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, eta_s=0.01, order=6,
                   device=0) as s:
        s.step(1.0 / 64)
        t = 1.0 / 64 + 1.0 / 4096
        s.predict(t)
        rng = np.random.default_rng(65537)
        sample = np.sort(rng.choice(65536, size=512, replace=False)).astype(np.int32)
        acc, jerk, snap, pot = s.force_snap(sample)
        (pp, vp, ap), m = _predicted_oracle_state(s, t)
    ra, rj, rs, rp = oracle.force6(m, pp, vp, ap, eps * eps, sample)
    _gate6("f32ds", (acc, jerk, snap, pot), (ra, rj, rs, rp), "N=65536 sample of 512")


def test_fused6_steps_force_vs_oracle(nb):
    """Single block steps with due sets of at most NB_FUSED6_MAX_NA particles, each taken
    by the order-6 fused kernel (N = 3000: 24 j-tiles' worth of chunks, groups of four
    slots with idle ones): the due particles' new acc, jerk and snap are the kernel's force
    on the j-set predicted to t_next, against the oracle (on the oracle's order-6
    prediction of the state before the step) and against the planned tile kernel
    (nb_predict + nb_force_snap on the same state: the same pair terms, summed in another
    order)."""
    n, eps = 3000, 0.01
    p = ic.plummer(n, 89)
    sizes = []
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, eta_s=0.01, order=6,
                   device=0) as s:
        s.step(1.0 / 256)
        for _ in range(300):
            if len(sizes) >= 6 and max(sizes) > 4:
                break
            g0 = s.state()
            snap0, crk0 = s.snap()
            t_next = float((g0["t"] + g0["dt"]).min())
            due = np.nonzero(g0["t"] + g0["dt"] == t_next)[0].astype(np.int32)
            small = len(due) <= nb.NB_FUSED6_MAX_NA
            if small:
                s.predict(t_next)
                h_acc, h_jerk, h_snap, _ = s.force_snap(due)
            st = s.step(t_next)
            assert st["block_steps"] == 1 and st["fused_steps"] == (1 if small else 0), st
            if not small:
                continue
            g1 = s.state()
            snap1, _ = s.snap()
            pp, vp, ap = oracle.predict6(t_next, g0["t"], g0["pos"].T, g0["vel"].T, g0["acc"].T,
                                         g0["jerk"].T, snap0.T, crk0.T)
            ra, rj, rs, _ = oracle.force6(g0["m"], pp, vp, ap, eps * eps, due)
            got = {"acc": g1["acc"][:, due].T, "jerk": g1["jerk"][:, due].T,
                   "snap": snap1[:, due].T}
            rep = report({"acc": (got["acc"], ra), "jerk": (got["jerk"], rj),
                          "snap": (got["snap"], rs)})
            rep_h = report({"acc": (got["acc"], h_acc.T), "jerk": (got["jerk"], h_jerk.T),
                            "snap": (got["snap"], h_snap.T)})
            print(len(due), "oracle:", fmt(rep), "| tile kernel:", fmt(rep_h))
            # per-particle gates: with a handful of due particles the RMS over the set is
            # one particle's error
            for q, g_max in zip(("acc", "jerk", "snap"), PP_GATES["f32ds"]):
                assert rep[q][1] < g_max, (len(due), q, rep[q])
                assert rep_h[q][1] < g_max, (len(due), q, rep_h[q])
            np.testing.assert_array_equal(g1["t"][due], t_next)
            sizes.append(len(due))
    print("due-set sizes", sizes)
    assert len(sizes) >= 6 and max(sizes) > 4               # more than one group of slots


def test_fused6_matches_separate_launches(nb):
    """1/16 time unit of order-6 block steps, with and without the fused kernel (N = 5000):
    the same schedule (block steps, final steps), states equal to the double-single force
    error, and the hand-over to the planned kernels for due sets above NB_FUSED6_MAX_NA
    (the oracle takes 147 of its 214 steps here with at most 64 due)."""
    p = ic.plummer(5000, 90)
    kw = dict(variant="f32ds", eps=1e-2, eta=0.02, eta_s=0.01, dt_max=1.0 / 16, order=6,
              device=0)
    with nb.System(p.m, p.pos, p.vel, **kw) as a:
        sa = a.step(1.0 / 16)
        ga = a.state()
        sna, cra = a.snap()
    with nb.System(p.m, p.pos, p.vel, flags=nb.NB_FLAG_NO_FUSED, **kw) as b:
        sb = b.step(1.0 / 16)
        gb = b.state()
        snb, crb = b.snap()
    print(sa["block_steps"], sa["fused_steps"], sb["block_steps"])
    assert sb["fused_steps"] == 0
    assert 0.5 * sa["block_steps"] < sa["fused_steps"] < sa["block_steps"]
    assert abs(sa["block_steps"] - sb["block_steps"]) <= 0.01 * sb["block_steps"]
    assert sa["interactions"] == pytest.approx(sb["interactions"], rel=0.02)
    np.testing.assert_array_equal(ga["t"], gb["t"])
    assert (ga["dt"] == gb["dt"]).mean() > 0.99
    scale = np.abs(gb["pos"]).max()
    assert np.abs(ga["pos"] - gb["pos"]).max() < 1e-6 * scale
    assert _rel_rms(sna, snb) < 1e-3


@pytest.mark.parametrize("n", [3000, 20000])
def test_autotuned_plans_force_snap_vs_oracle(nb, n):
    """nb_autotune on an order-6 handle: every bucket gets a tile-kernel entry (1, 2, 4 or 8
    warp rows), and the snap force with the tuned plans on i-sets of other sizes than the
    tuned 2^b (so with scaled split counts) still meets the force gates against the
    oracle."""
    p = ic.plummer(n, 91, masses="lognormal")
    eps = 0.01
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, order=6,
                   device=0) as s:
        s.step(1.0 / 128)
        table = nb.nb_autotune(s.h, 2)
        nb_max = int(np.ceil(np.log2(n)))
        for b in range(nb_max + 1):
            assert table[b][0] == 0 and table[b][1] in (1, 2, 4, 8) and table[b][2] >= 1, (b, table[b])
        assert all(t[0] == -1 for t in table[nb_max + 1:])
        t = 1.0 / 128 + 1.0 / 2048
        s.predict(t)
        rng = np.random.default_rng(92)
        for n_i in (45, 700, n - 7):
            plan = nb.nb_plan_for(s.h, n_i)
            assert plan[0] == 0 and plan[1] in (1, 2, 4, 8)
            idx = np.sort(rng.choice(n, size=n_i, replace=False)).astype(np.int32)
            acc, jerk, snap, pot = s.force_snap(idx)
            (pp, vp, ap), m = _predicted_oracle_state(s, t)
            ra, rj, rs, rp = oracle.force6(m, pp, vp, ap, eps * eps, idx)
            _gate6("f32ds", (acc, jerk, snap, pot), (ra, rj, rs, rp), "tuned N=%d n_i=%d" % (n, n_i))
