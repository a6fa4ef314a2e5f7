"""Batched systems (nb_batch_*): many independent Plummer clusters of uneven N advanced
with shared-step Hermite in one graph-replayed step, against the FP64 oracle run cluster
by cluster, and each cluster alone against the same cluster in the mix."""
import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu


def _clusters(n, lo, hi, seed):
    sizes = ic.cluster_sizes(n, lo, hi, seed)
    systems = [ic.plummer(int(k), int(ic.key(seed, 8, c))) for c, k in enumerate(sizes)]
    return systems, ic.cluster_eps(sizes)


def test_batch_matches_oracle_per_cluster(nb):
    systems, eps = _clusters(24, 16, 600, 41)
    dt, nsteps = 1.0 / 512, 8
    with nb.Batch(systems, eps, dt, variant="f32ds", device=0) as b:
        st = b.step(nsteps)
        pos, vel, t = b.get()
        k, w = b.energy()
    assert t == nsteps * dt
    assert st["block_steps"] == nsteps
    # the first call also evaluates the initial acc/jerk
    assert st["interactions"] == (nsteps + 1) * sum(len(p.m) ** 2 for p in systems)
    for s, p in enumerate(systems):
        o = oracle.State(p.m, p.pos, p.vel)
        oracle.hermite_run(o, np.inf, eps[s] ** 2, dt_shared=dt, max_steps=nsteps)
        got = b.system(s, pos).T
        scale = np.abs(p.pos).max()
        assert np.abs(got - o.pos).max() < 1e-7 * scale, s
        ko, wo = oracle.energy(p.m, o.pos, o.vel, eps[s] ** 2)
        assert abs(k[s] - ko) < 1e-7 * abs(ko)   # velocities carry the DS force error
        assert abs(w[s] - wo) < 1e-6 * abs(wo)


def test_cluster_alone_equals_cluster_in_the_mix(nb):
    systems, eps = _clusters(10, 16, 900, 42)
    dt = 1.0 / 512
    with nb.Batch(systems, eps, dt, variant="f32ds", device=0) as b:
        b.step(5)
        mix, _, _ = b.get()
    for s in (0, 3, 9):
        with nb.Batch([systems[s]], eps[s:s + 1], dt, variant="f32ds", device=0) as a:
            a.step(5)
            alone, _, _ = a.get()
        np.testing.assert_array_equal(alone, b.system(s, mix))


def test_batch_energy_conservation_and_autotune(nb):
    systems, eps = _clusters(64, 16, 1000, 43)
    with nb.Batch(systems, eps, 1.0 / 512, variant="f32ds", device=0) as b:
        assert b.autotune() in (64, 128, 256)
        k0, w0 = b.energy()
        b.step(64)
        k1, w1 = b.energy()
    e0, e1 = k0 + w0, k1 + w1
    assert np.median(np.abs((e1 - e0) / e0)) < 1e-5


def test_batch_errors(nb):
    cfg = nb.nb_config_default(variant="f64", device=0)
    with pytest.raises(nb.NBodyError) as e:
        nb.nb_batch_create(cfg, [10, 20], [0.1, 0.1], 1.0 / 512)
    assert e.value.status == nb.NB_ERR_ARG
    cfg = nb.nb_config_default(variant="f32ds", device=0)
    with pytest.raises(nb.NBodyError) as e:
        nb.nb_batch_create(cfg, [10, 0], [0.1, 0.1], 1.0 / 512)
    assert e.value.status == nb.NB_ERR_ARG
    with pytest.raises(nb.NBodyError) as e:
        nb.nb_batch_create(cfg, [10], [0.1], 0.0)
    assert e.value.status == nb.NB_ERR_ARG


@pytest.mark.slow
def test_full_size_batch4096_sampled_clusters(nb):
    """Config 4 at its own size: the 4096 clusters of the bench (N log-uniform in
    [16, 4096], seeded as the bench seeds them, about 3e6 particles), CTA size chosen by
    the autotuner, four graph-replayed shared steps of dt = 1/512. Ten clusters across the
    size range, the largest and the smallest among them, against the oracle run cluster by
    cluster: positions and velocities per particle, and the energy."""
    systems = ic.cluster_batch(4096, 16, 4096)
    sizes = np.array([len(p.m) for p in systems])
    eps = ic.cluster_eps(sizes)
    dt, nsteps = 1.0 / 512, 4
    with nb.Batch(systems, eps, dt, variant="f32ds", device=0) as b:
        assert b.autotune() in (64, 128, 256)
        st = b.step(nsteps)
        pos, vel, t = b.get()
        k, w = b.energy()
    assert t == nsteps * dt and st["block_steps"] == nsteps
    order = np.argsort(sizes, kind="stable")
    picks = sorted(set(order[np.linspace(0, len(order) - 1, 9).round().astype(int)].tolist())
                   | {int(order[-2])})
    assert sizes[picks].max() == sizes.max() and sizes[picks].min() == sizes.min()
    for s in picks:
        p = systems[s]
        o = oracle.State(p.m, p.pos, p.vel)
        oracle.hermite_run(o, np.inf, eps[s] ** 2, dt_shared=dt, max_steps=nsteps)
        gp, gv = b.system(s, pos).T, b.system(s, vel).T
        scale = np.abs(p.pos).max()
        dpos = np.linalg.norm(gp - o.pos, axis=1).max() / scale
        dvel = np.linalg.norm(gv - o.vel, axis=1).max() / np.abs(p.vel).max()
        print("cluster %d N=%d: max |dx|/scale %.2e, max |dv|/scale %.2e" % (s, sizes[s], dpos, dvel))
        assert dpos < 1e-7 and dvel < 1e-6, (s, sizes[s], dpos, dvel)
        ko, wo = oracle.energy(p.m, o.pos, o.vel, eps[s] ** 2)
        assert abs(k[s] - ko) < 1e-6 * abs(ko) and abs(w[s] - wo) < 1e-6 * abs(wo), s
