"""bench.py's multi-GPU mode runs independent replicas: a barrier and a max over ranks of
the timed seconds, units summed. The host logic runs here as two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    d = bench.Dist(world, "gloo")
    d.barrier()
    pairs = d.gather_pairs(100.0 * (rank + 1), 1.0 + 0.5 * rank)
    d.barrier()
    d.close()
    q.put((rank, pairs, bench.aggregate(pairs)))


def test_replicas_sum_units_and_take_slowest_rank():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, pairs, (units, secs) in out:
        assert pairs == [(100.0, 1.0), (200.0, 1.5)]
        assert units == 300.0 and secs == 1.5


def test_aggregate_single():
    assert bench.aggregate([(5.0, 2.0)]) == (5.0, 2.0)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
