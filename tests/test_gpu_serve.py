"""The serving loop (nb_server_* / nb_submit / nb_poll): force and integration requests on
subsystems of uneven N, batched into one force launch per tick. Each request against the
FP64 oracle, each request alone against the same request in a mix, and the admission,
cancellation and error paths."""
import time

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu


def _rel_rms(got, ref):
    return np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())


def _req(n, seed):
    p = ic.plummer(n, seed)
    return p.m, p.pos.T.copy(), p.vel.T.copy()


SIZES = (1, 2, 3, 17, 255, 256, 257, 1000, 4100)


def test_force_requests_match_oracle(nb):
    with nb.Server(variant=nb.NB_F32DS, device=0) as srv:
        reqs = {n: _req(n, 100 + n) for n in SIZES}
        tickets = {n: srv.force(*reqs[n], eps=0.25 / np.cbrt(n)) for n in SIZES}
        for n in SIZES:
            r = srv.wait(tickets[n])
            assert r["status"] == nb.NB_STATUS_DONE and r["error"] == nb.NB_OK
            m, pos, vel = reqs[n]
            eps = 0.25 / np.cbrt(n)
            ra, rj, rp = oracle.force(m, pos.T, vel.T, eps * eps)
            assert r["interactions"] == n * n
            assert r["t_submit"] <= r["t_start"] <= r["t_done"]
            if n == 1:  # no pairs: exact zeros
                assert not r["acc"].any() and not r["jerk"].any() and not r["pot"].any()
                continue
            assert _rel_rms(r["acc"].T, ra) < 1e-6, n
            assert _rel_rms(r["jerk"].T, rj) < 1e-6, n
            assert _rel_rms(r["pot"], rp) < 1e-6, n
        st = srv.stats()
    assert st["submitted"] == st["completed"] == len(SIZES)
    assert st["failed"] == st["cancelled"] == 0
    assert st["interactions"] == sum(n * n for n in SIZES)


def test_request_alone_equals_request_in_the_mix(nb):
    reqs = [_req(n, 200 + n) for n in (5, 300, 1500, 64, 2049)]
    evo = _req(200, 299)
    kw = dict(variant=nb.NB_F32DS, eta=0.02, dt_max=1.0 / 16, device=0)
    alone = []
    with nb.Server(**kw) as srv:
        for m, pos, vel in reqs:
            alone.append(srv.wait(srv.force(m, pos, vel, eps=0.01)))
        ev_alone = srv.wait(srv.evolve(*evo, eps=0.01, t_span=1.0 / 16))
    with nb.Server(**kw) as srv:
        # the integration shares every tick with the force requests and a second one
        te = srv.evolve(*evo, eps=0.01, t_span=1.0 / 16)
        t2 = srv.evolve(*_req(700, 298), eps=0.02, t_span=1.0 / 8)
        tf = [srv.force(m, pos, vel, eps=0.01) for m, pos, vel in reqs]
        mix = [srv.wait(t) for t in tf]
        ev_mix = srv.wait(te)
        assert srv.wait(t2)["status"] == nb.NB_STATUS_DONE
    for a, b in zip(alone, mix):
        for k in ("acc", "jerk", "pot"):
            np.testing.assert_array_equal(a[k], b[k])
    for k in ("pos", "vel"):
        np.testing.assert_array_equal(ev_alone[k], ev_mix[k])
    assert ev_alone["block_steps"] == ev_mix["block_steps"]
    assert ev_alone["interactions"] == ev_mix["interactions"]


def test_evolve_request_matches_oracle_and_engine(nb):
    """A block-step integration as a request: the oracle's schedule and state, and the
    engine's (nb_step) block-step count."""
    n, eps, span = 512, 0.01, 1.0 / 16
    m, pos, vel = _req(n, 31)
    with nb.Server(variant=nb.NB_F32DS, eta=0.02, dt_max=1.0 / 16, device=0) as srv:
        r = srv.wait(srv.evolve(m, pos, vel, eps=eps, t_span=span))
    assert r["status"] == nb.NB_STATUS_DONE
    st = oracle.State(m, pos.T, vel.T)
    o_steps, o_inter = oracle.hermite_run(st, span, eps * eps, eta=0.02, dt_max=1.0 / 16)
    assert abs(r["block_steps"] - o_steps) <= 0.05 * o_steps
    assert np.abs(r["pos"].T - st.pos).max() < 1e-5
    assert np.abs(r["vel"].T - st.vel).max() < 1e-4
    with nb.System(m, pos.T, vel.T, variant="f32ds", eps=eps, eta=0.02, dt_max=1.0 / 16,
                   device=0) as s:
        stats = s.step(span)
    assert abs(r["block_steps"] - stats["block_steps"]) <= 0.02 * stats["block_steps"]


def test_energy_of_evolve_requests(nb):
    kw = dict(variant=nb.NB_F32DS, eta=0.01, dt_max=1.0 / 16, device=0)
    sizes = (64, 256, 1024)
    with nb.Server(**kw) as srv:
        reqs = [_req(n, 400 + n) for n in sizes]
        tk = [srv.evolve(*q, eps=0.25 / np.cbrt(n), t_span=0.25) for q, n in zip(reqs, sizes)]
        res = [srv.wait(t, timeout_s=120) for t in tk]
    for (m, pos, vel), n, r in zip(reqs, sizes, res):
        eps2 = (0.25 / np.cbrt(n)) ** 2
        k0, w0 = oracle.energy(m, pos.T, vel.T, eps2)
        k1, w1 = oracle.energy(m, r["pos"].T, r["vel"].T, eps2)
        assert abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0) < 1e-5, n


def test_admission_budget_busy_and_cancel(nb):
    m, pos, vel = _req(256, 500)
    with nb.Server(variant=nb.NB_F32DS, max_inflight=1, max_queue=1, device=0) as srv:
        # a long integration holds the one in-flight slot
        long_t = srv.evolve(m, pos, vel, eps=1e-3, t_span=64.0)
        t_end = time.time() + 60
        while srv.poll(long_t)["block_steps"] < 10 and time.time() < t_end:
            time.sleep(0.01)
        st = srv.poll(long_t)
        assert st["status"] == nb.NB_STATUS_RUNNING and st["block_steps"] >= 10
        queued = srv.force(m, pos, vel, eps=0.01)
        with pytest.raises(nb.NBodyError) as e:
            srv.force(m, pos, vel, eps=0.01)
        assert e.value.status == nb.NB_ERR_BUSY
        # cancel the queued one, then the running one
        srv.cancel(queued)
        assert srv.poll(queued)["status"] == nb.NB_STATUS_CANCELLED
        srv.cancel(long_t)
        r = srv.wait(long_t, timeout_s=60)
        assert r["status"] == nb.NB_STATUS_CANCELLED
        assert r["block_steps"] >= 10
        with pytest.raises(nb.NBodyError) as e:
            srv.cancel(long_t)
        assert e.value.status == nb.NB_ERR_NOTFOUND  # released by wait
        # the slot is free again
        r = srv.wait(srv.force(m, pos, vel, eps=0.01))
        assert r["status"] == nb.NB_STATUS_DONE
        st = srv.stats()
    assert st["cancelled"] == 2 and st["completed"] == 1


def test_request_errors(nb):
    m, pos, vel = _req(100, 501)
    with nb.Server(variant=nb.NB_F32DS, budget_bytes=1 << 20, device=0) as srv:
        big = _req(20000, 502)
        with pytest.raises(nb.NBodyError) as e:
            srv.force(*big, eps=0.01)
        assert e.value.status == nb.NB_ERR_BUDGET
        bad = pos.copy()
        bad[1, 7] = np.nan
        with pytest.raises(nb.NBodyError) as e:
            srv.force(m, bad, vel, eps=0.01)
        assert e.value.status == nb.NB_ERR_NONFINITE
        with pytest.raises(nb.NBodyError) as e:
            srv.force(m, pos, vel, eps=-1.0)
        assert e.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NBodyError) as e:
            srv.evolve(m, pos, vel, eps=0.01, t_span=0.1)  # not a multiple of dt_max
        assert e.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NBodyError) as e:
            nb.nb_submit(srv.s, 7, m, pos, vel, 0.01)
        assert e.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NBodyError) as e:
            srv.poll(12345)
        assert e.value.status == nb.NB_ERR_NOTFOUND
        # a small request still runs within the budget
        r = srv.wait(srv.force(m, pos, vel, eps=0.01))
        assert r["status"] == nb.NB_STATUS_DONE
    with pytest.raises(nb.NBodyError) as e:
        nb.nb_server_create(variant=nb.NB_F64, device=0)
    assert e.value.status == nb.NB_ERR_ARG


def test_many_small_requests_share_ticks(nb):
    """Requests of a Poisson-like stream of uneven sizes: all complete, and there are
    fewer force launches than requests (they were batched)."""
    sizes = ic.cluster_sizes(200, 16, 2000, 77)
    reqs = [_req(int(n), 600 + i) for i, n in enumerate(sizes)]
    with nb.Server(variant=nb.NB_F32DS, device=0) as srv:
        tk = [srv.force(*q, eps=0.25 / np.cbrt(n)) for q, n in zip(reqs, sizes)]
        res = [srv.wait(t) for t in tk]
        st = srv.stats()
    assert all(r["status"] == nb.NB_STATUS_DONE for r in res)
    assert st["force_launches"] < len(sizes)
    i = int(np.argmax(sizes))
    m, pos, vel = reqs[i]
    eps = 0.25 / np.cbrt(sizes[i])
    ra, _, _ = oracle.force(m, pos.T, vel.T, eps * eps)
    assert _rel_rms(res[i]["acc"].T, ra) < 1e-6


def test_sixty_four_stream_requests_alone_equal_mix(nb):
    """64 requests drawn from the serving stream (galaxy subsystems with a central point
    mass, N log-uniform in [2^8, 2^12], half force, half 1/16 time unit of block steps):
    every result of the concurrent run is bitwise the result of the request served alone."""
    reqs = ic.request_stream(64, 1e6, n_lo=2 ** 8, n_hi=2 ** 12, t_span=1.0 / 16)
    parts = [ic.request_particles(r) for r in reqs]
    kw = dict(variant=nb.NB_F32DS, eta=0.02, dt_max=1.0 / 16, device=0)

    def submit(srv, r, p):
        eps = 0.25 / np.cbrt(r.n)
        if r.kind == "force":
            return srv.force(p.m, p.pos.T, p.vel.T, eps)
        return srv.evolve(p.m, p.pos.T, p.vel.T, eps, r.t_span)

    with nb.Server(**kw) as srv:
        mix = [srv.wait(t, timeout_s=300) for t in [submit(srv, r, p) for r, p in zip(reqs, parts)]]
    with nb.Server(**kw) as srv:
        alone = [srv.wait(submit(srv, r, p), timeout_s=300) for r, p in zip(reqs, parts)]
    for r, a, b in zip(reqs, alone, mix):
        assert a["status"] == b["status"] == nb.NB_STATUS_DONE
        keys = ("acc", "jerk", "pot") if r.kind == "force" else ("pos", "vel")
        for k in keys:
            np.testing.assert_array_equal(a[k], b[k])
        assert a["interactions"] == b["interactions"]
