"""bench.py's multi-process path (replicas, one rank per GPU) on CPU with
the gloo backend: every rank's counters reach rank 0, the whole-job value is
all node-updates over the slowest rank's time, and the reference arm runs
on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = {"node_updates": 1000 * (rank + 1), "ms": 10.0 * (rank + 1),
             "e2e_nu": 500 * (rank + 1), "e2e_ms": 20.0 + rank}
    bench._barrier(world, None)
    agg = bench._gather(world, local, None)
    q.put((rank, bench.aggregate(agg), len(agg)))
    dist.destroy_process_group()


def test_replicas_aggregate_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (value, ms, e2e), n in res:
        assert n == world
        assert ms == 20.0
        assert value == pytest.approx(3000 / 0.020)
        assert e2e == pytest.approx(1500 / 0.021)


def test_reference_arm_only_on_rank0(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "reference_arm", lambda *a: called.append(a) or 0)
    assert bench.main() == 0
    assert not called
