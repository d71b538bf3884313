"""The benchmark's multi-rank bookkeeping on CPU: world_size 2 over gloo.  Every rank must
end with the maximum of the ranks' times, and the reported rate counts all ranks' units
over that time (replicas: weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [10.0 + rank, 4.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, world, "cpu")
    rate = bench.whole_job_rate(1000, world, got[1])
    q.put((rank, got, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
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
    for rank, got, rate in res:
        assert got == [11.0, 8.0]
        assert rate == pytest.approx(2 * 1000 / 0.008)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 1.5], 1, "cpu") == [3.0, 1.5]
    assert bench.whole_job_rate(500, 1, 2.0) == pytest.approx(250000.0)
