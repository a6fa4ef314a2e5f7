"""Parity of the CUDA block-step Hermite path (K1-K5 through nb_step) with the
FP64 CPU oracle, plus the invariants that hold at any size.

Trajectories of N-body systems diverge exponentially (paper Sect. VI), so
long-horizon comparisons use energy and invariants; short horizons compare
states directly.
"""
import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu


def _energy_oracle(m, pos, vel, eps2):
    k, w = oracle.energy(m, pos, vel, eps2)
    return k + w


def test_small_case_shared_steps_fp64(nb):
    """N = 1024 Plummer, eps = 1/64, shared dt = 1/256, FP64 pairs, one time unit:
    energy drift <= 1e-6; state close to the oracle's; per-step force parity 1e-12."""
    p = ic.plummer(1024)
    eps = 1.0 / 64
    eps2 = eps * eps
    st = oracle.State(p.m, p.pos, p.vel)
    e0 = _energy_oracle(p.m, p.pos, p.vel, eps2)
    oracle.hermite_run(st, 0.25, eps2, dt_shared=1.0 / 256)
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=eps, shared_dt=1.0 / 256, device=0) as s:
        k0, w0 = s.energy()
        assert abs((k0 + w0) - e0) < 1e-13
        stats = s.step(0.25)
        assert stats["block_steps"] == 64
        g = s.state()
        # state after a quarter time unit agrees with the oracle's run
        assert np.abs(g["pos"].T - st.pos).max() < 1e-9
        # per-evaluation parity on the GPU's own state
        s.predict(0.25)
        acc, jerk, pot = s.force()
        ra, rj, rp = oracle.force(p.m, g["pos"].T, g["vel"].T, eps2)
        assert np.sqrt(((acc.T - ra) ** 2).sum() / (ra ** 2).sum()) < 1e-12
        assert np.sqrt(((jerk.T - rj) ** 2).sum() / (rj ** 2).sum()) < 1e-12
        s.step(1.0)
        k1, w1 = s.energy()
    assert abs((k1 + w1 - e0) / e0) < 1e-6


@pytest.mark.parametrize("variant", ["f64", "f32ds"])
def test_block_steps_short_horizon(nb, variant):
    """Block steps (eta = 0.02, dt_max = 1/16) over 1/16 time unit: same schedule as the
    oracle (block-step count and interactions within a few percent), positions close."""
    p = ic.plummer(512, 31)
    eps = 0.01
    st = oracle.State(p.m, p.pos, p.vel)
    o_steps, o_inter = oracle.hermite_run(st, 1.0 / 16, eps * eps, eta=0.02, dt_max=1.0 / 16)
    with nb.System(p.m, p.pos, p.vel, variant=variant, eps=eps, eta=0.02, dt_max=1.0 / 16,
                   device=0) as s:
        stats = s.step(1.0 / 16)
        g = s.state()
    np.testing.assert_array_equal(g["t"], 1.0 / 16)
    if variant == "f64":
        assert stats["block_steps"] == o_steps
        assert abs(stats["interactions"] - o_inter) <= 0.02 * o_inter
        assert np.abs(g["pos"].T - st.pos).max() < 1e-8
        assert (g["dt"] == st.dt).mean() > 0.99
    else:
        assert abs(stats["block_steps"] - o_steps) <= 0.05 * o_steps
        assert np.abs(g["pos"].T - st.pos).max() < 1e-5


def test_block_invariants_and_energy(nb):
    p = ic.plummer(5000, 32)  # three scheduler tiles of 2048
    eps = 1e-3
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.01, dt_max=1.0 / 16,
                   device=0) as s:
        k0, w0 = s.energy()
        stats = s.step(0.125)
        g = s.state()
        k1, w1 = s.energy()
    np.testing.assert_array_equal(g["t"], 0.125)
    lg = np.log2(g["dt"])
    np.testing.assert_array_equal(lg, np.round(lg))
    np.testing.assert_array_equal(np.fmod(g["t"], g["dt"]), 0.0)
    assert stats["block_steps"] >= 8 and sum(stats["active_hist"]) == stats["block_steps"]
    assert abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0) < 1e-5


def test_schedule_counts_two_binaries(nb):
    """Exact scheduler counts: tight binary 128 steps, wide binary 16 over 2^-6."""
    pos, vel = [], []
    import math
    for cx, d in ((-5.0, 0.01), (5.0, 0.04)):
        w = math.sqrt(0.5 / d ** 3)
        pos += [[cx - d / 2, 0, 0], [cx + d / 2, 0, 0]]
        vel += [[0, -w * d / 2, 0], [0, w * d / 2, 0]]
    with nb.System(np.full(4, 0.25), np.array(pos), np.array(vel), variant="f64", eps=0.0,
                   eta=0.01, eta_s=0.1, dt_max=1.0 / 16, device=0) as s:
        stats = s.step(2.0 ** -6)
        g = s.state()
    np.testing.assert_array_equal(g["dt"], [2.0 ** -13] * 2 + [2.0 ** -10] * 2)
    assert stats["block_steps"] == 128
    assert stats["interactions"] == 16 + 4 * (2 * 128 + 2 * 16)


def test_checkpoint_resume_bitwise(nb):
    p = ic.plummer(800, 33)
    kw = dict(variant="f32ds", eps=0.01, eta=0.02, device=0)
    with nb.System(p.m, p.pos, p.vel, **kw) as a:
        a.step(1.0 / 16)
        ck = a.state()
        a.step(1.0 / 8)
        full = a.state()
    with nb.System(ck["m"], ck["pos"].T, ck["vel"].T, **kw) as b:
        b.set_state(ck)
        b.step(1.0 / 8)
        res = b.state()
    for k in ("pos", "vel", "acc", "jerk", "dt"):
        np.testing.assert_array_equal(res[k], full[k])


def test_equal_block_steps_equal_shared_steps(nb):
    p = ic.plummer(300, 34)
    dt = 1.0 / 256
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=0.01, shared_dt=dt, device=0) as a:
        a.step(16 * dt)
        sa = a.state()
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=0.01, dt_min=dt, dt_max=dt,
                   device=0) as b:
        b.step(16 * dt)
        sb = b.state()
    np.testing.assert_array_equal(sa["pos"], sb["pos"])
    np.testing.assert_array_equal(sa["vel"], sb["vel"])


def test_manual_calls_equal_one_block_step(nb):
    """nb_predict + nb_force(due set) + nb_correct reproduce the first block step of nb_step:
    the due set the scheduler compacts (over several tiles) is the one t_i + dt_i == t_next
    defines."""
    p = ic.plummer(5000, 35)
    kw = dict(variant="f64", eps=0.01, eta=0.02, device=0)
    with nb.System(p.m, p.pos, p.vel, **kw) as a:
        nb.nb_init(a.h)
        s0 = a.state()
        t_next = float((s0["t"] + s0["dt"]).min())
        due = np.nonzero(s0["t"] + s0["dt"] == t_next)[0].astype(np.int32)
        a.predict(t_next)
        a.force(due)
        a.correct(due, t_next)
        ma = a.state()
    with nb.System(p.m, p.pos, p.vel, **kw) as b:
        nb.nb_init(b.h)
        stats = b.step(t_next)
        mb = b.state()
    assert stats["block_steps"] == 1
    for k in ("pos", "vel", "acc", "jerk", "t", "dt"):
        np.testing.assert_array_equal(ma[k], mb[k])


def test_block_steps_multi_tile_vs_oracle(nb):
    """N = 6000 (three scheduler tiles), FP64 pairs, 1/64 time unit: the same block-step
    schedule as the oracle and states that agree to 1e-9."""
    p = ic.plummer(6000, 36)
    eps = 0.01
    st = oracle.State(p.m, p.pos, p.vel)
    o_steps, o_inter = oracle.hermite_run(st, 1.0 / 64, eps * eps, eta=0.02, dt_max=1.0 / 16)
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=eps, eta=0.02, dt_max=1.0 / 16,
                   device=0) as s:
        stats = s.step(1.0 / 64)
        g = s.state()
    assert stats["block_steps"] == o_steps
    assert abs(stats["interactions"] - o_inter) <= 1e-3 * o_inter
    np.testing.assert_array_equal(g["t"], st.t)
    assert (g["dt"] == st.dt).mean() > 0.999
    assert np.abs(g["pos"].T - st.pos).max() < 1e-9


def test_set_state_rejects_broken_block_invariant(nb):
    p = ic.plummer(100, 37)
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=0.01, device=0) as s:
        s.step(1.0 / 32)
        ck = s.state()
        bad = dict(ck)
        bad["t"] = ck["t"].copy()
        bad["dt"] = ck["dt"].copy()
        bad["dt"][3] = 1.0 / 16
        bad["t"][3] = 1.0 / 32 + 1.0 / 64   # not a multiple of its step
        with pytest.raises(nb.NBodyError) as e:
            s.set_state(bad)
        assert e.value.status == nb.NB_ERR_ARG
        s.set_state(ck)                     # the genuine checkpoint is accepted
        s.step(1.0 / 16)


def test_double_single_against_fp64_pairs_block_steps(nb):
    """The config-2 cross-check at N = 16384 (the oracle cannot run it in seconds): the
    F32-DS path (fused small steps, planned large ones) against the FP64-pair path over
    1/16 time unit of block steps: the same schedule to a few steps, states and energy
    agreeing to the double-single level."""
    p = ic.plummer(16384, 90)
    kw = dict(eps=1e-3, eta=0.01, dt_max=1.0 / 16, device=0)
    runs = {}
    for variant in ("f32ds", "f64"):
        with nb.System(p.m, p.pos, p.vel, variant=variant, **kw) as s:
            st = s.step(1.0 / 16)
            k, w = s.energy()
            runs[variant] = (st, s.state(), k + w)
    (sd, gd, ed), (s64, g64, e64) = runs["f32ds"], runs["f64"]
    assert sd["fused_steps"] > 0
    assert abs(sd["block_steps"] - s64["block_steps"]) <= 0.02 * s64["block_steps"]
    np.testing.assert_array_equal(gd["t"], g64["t"])
    assert np.abs(gd["pos"] - g64["pos"]).max() < 1e-5
    assert abs(ed - e64) < 1e-6 * abs(e64)


def test_full_size_block65536_sampled(nb):
    """The bench's block-step configuration at full size (Plummer N = 65536, eps = 1e-3,
    eta = 0.01, autotuned plans, fused small steps): after 1/16 time unit (one dt_max, all
    particles synchronised) the planned force on a seeded 512-particle sample of the
    predicted state against the oracle, the fused kernel having taken steps, and the
    energy."""
    p = ic.plummer(65536, ic.MASTER_SEED, masses="equal")
    eps = 1e-3
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.01, device=0) as s:
        nb.nb_autotune(s.h, 1)
        k0, w0 = s.energy()
        stats = s.step(1.0 / 16)
        assert stats["fused_steps"] > 0 and stats["block_steps"] > stats["fused_steps"] > 0
        k1, w1 = s.energy()
        g = s.state()
        t = 1.0 / 16 + 1.0 / 4096
        s.predict(t)
        rng = np.random.default_rng(65536)
        sample = np.sort(rng.choice(65536, size=512, replace=False)).astype(np.int32)
        acc, jerk, pot = s.force(sample)
    pp, vp = oracle.predict(t, g["t"], g["pos"].T, g["vel"].T, g["acc"].T, g["jerk"].T)
    ra, rj, rp = oracle.force(g["m"], pp, vp, eps * eps, idx=sample)
    rel = lambda x, y: np.sqrt(((x - y) ** 2).sum() / (y ** 2).sum())
    assert rel(acc.T, ra) < 1e-6 and rel(jerk.T, rj) < 1e-5 and rel(pot, rp) < 1e-6
    assert abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0) < 1e-6


@pytest.mark.slow
def test_full_size_block65536_first_64_block_steps_vs_oracle(nb):
    """Config 2 at full size: the bench's system (Plummer N = 65536, eps = 1e-3, eta = 0.01,
    dt_max = 1/16, F32-DS with autotuned plans and the fused small-step kernel) from t = 0
    through the block time the oracle reaches after its initial evaluation and first 64
    block steps (the run the bench's CPU baseline times). The GPU takes the same number of
    block steps (within 2), gives at least 99% of the particles the same time and step,
    and the particles at the same time agree in position to 1e-5 (the force's FP32 rounding
    grows through the corrector) and in velocity to 1e-4."""
    import math
    p = ic.plummer(65536, ic.MASTER_SEED)
    eps = 1e-3
    st = oracle.State(p.m, p.pos, p.vel)
    o_steps, o_inter = oracle.hermite_run(st, math.inf, eps * eps, eta=0.01, dt_max=1.0 / 16,
                                          max_steps=64)
    assert o_steps == 64
    t64 = float(st.t.max())
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.01, dt_max=1.0 / 16,
                   device=0) as s:
        nb.nb_autotune(s.h, 3)
        stats = s.step(t64)
        g = s.state()
    print("block steps GPU %d oracle %d; interactions GPU %.4g oracle %.4g"
          % (stats["block_steps"], o_steps, stats["interactions"], o_inter))
    assert abs(stats["block_steps"] - o_steps) <= 2
    assert stats["interactions"] == pytest.approx(o_inter, rel=0.02)
    same = (g["t"] == st.t) & (g["dt"] == st.dt)
    assert same.mean() > 0.99, same.mean()
    dx = np.linalg.norm(g["pos"].T[same] - st.pos[same], axis=1).max()
    dv = np.linalg.norm(g["vel"].T[same] - st.vel[same], axis=1).max()
    print("same time and step: %d of %d; max |dx| %.2e, max |dv| %.2e"
          % (same.sum(), same.size, dx, dv))
    assert dx < 1e-5 and dv < 1e-4
