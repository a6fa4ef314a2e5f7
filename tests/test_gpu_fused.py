"""Fused persistent block steps (the cooperative kernel nb_step uses for small due sets):
its force against the FP64 oracle on the predicted state, its schedule and states against
the separate-launch path (NB_FLAG_NO_FUSED), and the hand-over to the planned kernels for
large due sets."""
import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic
from tests.errstats import fmt, report

pytestmark = pytest.mark.gpu


def _rel_rms(got, ref):
    return np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())


@pytest.mark.parametrize("n", [700, 3000, 20000])
def test_fused_first_step_force_vs_oracle(nb, n):
    """One block step from the initial state: the due particles' new acc and jerk are the
    fused kernel's force on the j-set predicted to t_next (the predictor is a cubic in
    FP64, recomputed here); the due set spans many CTAs' particle ranges at N = 20000."""
    p = ic.plummer(n, 60 + n)
    eps = 0.25 / np.cbrt(n)
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, device=0) as s:
        nb.nb_init(s.h)
        s0 = s.state()
        t_next = float((s0["t"] + s0["dt"]).min())
        due = np.nonzero(s0["t"] + s0["dt"] == t_next)[0].astype(np.int32)
        assert 1 <= len(due) <= nb.NB_FUSED_DEFAULT_NA
        st = s.step(t_next)
        s1 = s.state()
    assert st["block_steps"] == 1 and st["fused_steps"] == 1 and st["fused_launches"] >= 1
    d = t_next - s0["t"]
    x, v, a, j = s0["pos"], s0["vel"], s0["acc"], s0["jerk"]
    xp = x + d * (v + d * (a / 2 + d * j / 6))
    vp = v + d * (a + d * j / 2)
    ra, rj, _ = oracle.force(p.m, xp.T, vp.T, eps * eps, idx=due)
    assert _rel_rms(s1["acc"][:, due].T, ra) < 1e-6
    assert _rel_rms(s1["jerk"][:, due].T, rj) < 1e-5
    np.testing.assert_array_equal(s1["t"][due], t_next)


def test_fused_matches_separate_launches(nb):
    """1/16 time unit of block steps, with and without the fused kernel: the same schedule
    (block steps, final steps), states equal to the double-single force error, and the
    hand-over to the planned kernels (steps with more than NB_FUSED_DEFAULT_NA due) used."""
    p = ic.plummer(5000, 61)
    kw = dict(variant="f32ds", eps=1e-2, eta=0.02, dt_max=1.0 / 16, device=0)
    with nb.System(p.m, p.pos, p.vel, **kw) as a:
        sa = a.step(1.0 / 16)
        ga = a.state()
    with nb.System(p.m, p.pos, p.vel, flags=nb.NB_FLAG_NO_FUSED, **kw) as b:
        sb = b.step(1.0 / 16)
        gb = b.state()
    assert sb["fused_steps"] == 0
    assert sa["fused_steps"] > 0.8 * sa["block_steps"]
    assert sa["fused_steps"] < sa["block_steps"]          # some steps went to the planned path
    assert abs(sa["block_steps"] - sb["block_steps"]) <= 0.01 * sb["block_steps"]
    assert sa["interactions"] == pytest.approx(sb["interactions"], rel=0.02)
    np.testing.assert_array_equal(ga["t"], gb["t"])
    assert (ga["dt"] == gb["dt"]).mean() > 0.99
    scale = np.abs(gb["pos"]).max()
    assert np.abs(ga["pos"] - gb["pos"]).max() < 1e-6 * scale


def test_fused_block_steps_vs_oracle(nb):
    """The block-step run of the short-horizon oracle test through the fused path."""
    p = ic.plummer(512, 31)
    eps = 0.01
    st = oracle.State(p.m, p.pos, p.vel)
    o_steps, _ = oracle.hermite_run(st, 1.0 / 16, eps * eps, eta=0.02, dt_max=1.0 / 16)
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, dt_max=1.0 / 16,
                   device=0) as s:
        stats = s.step(1.0 / 16)
        g = s.state()
    assert stats["fused_steps"] == stats["block_steps"]      # N < NB_FUSED_DEFAULT_NA
    assert abs(stats["block_steps"] - o_steps) <= 0.05 * o_steps
    np.testing.assert_array_equal(g["t"], 1.0 / 16)
    assert np.abs(g["pos"].T - st.pos).max() < 1e-5


def test_fused_f32_variant_and_energy(nb):
    p = ic.plummer(2000, 62)
    with nb.System(p.m, p.pos, p.vel, variant="f32", eps=0.02, eta=0.01, device=0) as s:
        k0, w0 = s.energy()
        st = s.step(0.25)
        k1, w1 = s.energy()
    assert st["fused_steps"] > 0
    assert abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0) < 1e-4


def test_fused_single_steps_both_paths_vs_oracle_and_planned(nb):
    """Single block steps taken by the fused kernel at N = 8000, through both of its force
    paths: group items (at most 16 due) and tile items (17 to NB_FUSED_DEFAULT_NA due: 32
    due slots per item against j-chunks staged in shared memory, then one warp per due
    particle reducing and correcting). The due particles' new acc and jerk against the
    oracle on the cubic prediction of the state before the step, and against the planned
    kernels (nb_predict + nb_force on the same state: the same pair terms summed in
    another order)."""
    n, eps = 8000, 0.01
    p = ic.plummer(n, 63)
    sizes = []
    with nb.System(p.m, p.pos, p.vel, variant="f32ds", eps=eps, eta=0.02, device=0) as s:
        s.step(1.0 / 256)
        for _ in range(400):
            if sum(k > 16 for k in sizes) >= 3 and sum(k <= 16 for k in sizes) >= 3:
                break
            g0 = s.state()
            t_next = float((g0["t"] + g0["dt"]).min())
            due = np.nonzero(g0["t"] + g0["dt"] == t_next)[0].astype(np.int32)
            fused = len(due) <= nb.NB_FUSED_DEFAULT_NA
            if fused:
                s.predict(t_next)
                h_acc, h_jerk, _ = s.force(due)
            st = s.step(t_next)
            assert st["block_steps"] == 1 and st["fused_steps"] == (1 if fused else 0), st
            if not fused:
                continue
            g1 = s.state()
            d = t_next - g0["t"]
            x, v, a, j = g0["pos"], g0["vel"], g0["acc"], g0["jerk"]
            xp = x + d * (v + d * (a / 2 + d * j / 6))
            vp = v + d * (a + d * j / 2)
            ra, rj, _ = oracle.force(g0["m"], xp.T, vp.T, eps * eps, idx=due)
            got_a, got_j = g1["acc"][:, due].T, g1["jerk"][:, due].T
            rep = report({"acc": (got_a, ra), "jerk": (got_j, rj)})
            rep_h = report({"acc": (got_a, h_acc.T), "jerk": (got_j, h_jerk.T)})
            print(len(due), "oracle:", fmt(rep), "| planned:", fmt(rep_h))
            # per-particle gates of the force tests (F32-DS: acc 1e-5, jerk 1e-4); the
            # RMS gates where the set is large enough for the RMS to mean one
            for q, g_max, g_rms in (("acc", 1e-5, 1e-6), ("jerk", 1e-4, 2e-6)):
                assert rep[q][1] < g_max and rep_h[q][1] < g_max, (len(due), q, rep[q], rep_h[q])
                if len(due) >= 32:
                    assert rep[q][0] < g_rms, (len(due), q, rep[q])
            np.testing.assert_array_equal(g1["t"][due], t_next)
            sizes.append(len(due))
    print("due-set sizes", sizes)
    assert sum(k > 16 for k in sizes) >= 3 and sum(k <= 16 for k in sizes) >= 3, sizes
