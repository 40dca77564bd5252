"""The N > 1 path of bench.py (independent replicas, barrier, slowest-rank
time, whole-job MLUPS) with world_size 2 on the gloo backend, CPU only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist(backend="gloo")
    d.barrier()
    # each replica reports its own time; the slowest counts
    t = d.max(1.0 + rank)
    out[rank] = bench.weak_scaling_value(1000, 10, d.world, t)
    d.close()


def test_two_rank_replicas_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # 2 replicas x 1000 nodes x 10 steps over the slowest rank's 2 s
    assert out[0] == out[1] == pytest.approx(2 * 1000 * 10 / 2.0 / 1e6)


def test_single_rank_value():
    import bench
    assert bench.weak_scaling_value(512 ** 3, 50, 1, 1.0) == pytest.approx(512 ** 3 * 50 / 1e6)
