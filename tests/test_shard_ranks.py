"""Replication and sharding across ranks (section 5.4) on CPU: world_size 2 over gloo.

Each rank holds half the database (sharding) or answers half the queries (replication);
the local search is the oracle's exact search on the rank's part (global ids), and the
join of the gathered shard lists keeps the k best by (value, id).  Both must equal the
unsplit exact search, ids included (ties resolved by the lower id on duplicated rows)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1702_08734_gb300 import datagen
from paper_1702_08734_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _data():
    xb = datagen.gaussian_matrix(31, 3000, 16)
    xb[2500:2600] = xb[10:110]  # duplicates in the other half: ties across shards
    xq = datagen.gaussian_matrix(32, 57, 16)
    xq[:5] = xb[10:15]
    return xq, xb


def _cpu_merge(Dp, Ip, k, largest):
    """k best of the stacked lists by (value, id); padding entries (id -1) last."""
    S, nq, kin = Dp.shape
    D = Dp.permute(1, 0, 2).reshape(nq, S * kin).numpy()
    I = Ip.permute(1, 0, 2).reshape(nq, S * kin).numpy()
    outD, outI = np.empty((nq, k), D.dtype), np.empty((nq, k), I.dtype)
    for q in range(nq):
        key = -D[q] if largest else D[q]
        o = np.lexsort((I[q], np.where(I[q] < 0, np.inf, key)))[:k]
        outD[q], outI[q] = D[q][o], I[q][o]
    return torch.from_numpy(outD), torch.from_numpy(outI)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    xq, xb = _data()
    k = 12
    r0, r1 = shard.part_range(xb.shape[0], rank, world)

    def local(xqs, kk):
        D, I = oracle.knn(xqs.numpy(), xb[r0:r1], kk)
        return torch.from_numpy(D), torch.from_numpy(I + r0)

    Ds, Is = shard.sharded_search(local, torch.from_numpy(xq), k, merge=_cpu_merge)

    def full(xqs, kk):
        D, I = oracle.knn(xqs.numpy(), xb, kk)
        return torch.from_numpy(D), torch.from_numpy(I)

    Dr, Ir = shard.replicated_search(full, torch.from_numpy(xq), k)
    q.put((rank, Ds.numpy(), Is.numpy(), Dr.numpy(), Ir.numpy()))
    dist.destroy_process_group()


def test_sharded_and_replicated_equal_unsplit_gloo():
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    qq = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, qq)) for r in range(world)]
    for p in procs:
        p.start()
    res = [qq.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    xq, xb = _data()
    Do, Io = oracle.knn(xq, xb, 12)
    for rank, Ds, Is, Dr, Ir in res:
        np.testing.assert_array_equal(Is, Io)
        np.testing.assert_array_equal(Ds, Do)
        np.testing.assert_array_equal(Ir, Io)
        np.testing.assert_array_equal(Dr, Do)


@pytest.mark.parametrize("n,world", [(10, 3), (7, 7), (5, 8), (1000, 4)])
def test_part_ranges_cover_once(n, world):
    seen = np.zeros(n, int)
    sizes = []
    for r in range(world):
        r0, r1 = shard.part_range(n, r, world)
        seen[r0:r1] += 1
        sizes.append(r1 - r0)
    assert np.all(seen == 1) and max(sizes) - min(sizes) <= 1


def test_single_process_forms_are_the_local_search():
    xq, xb = _data()

    def local(x, k):
        import oracle
        D, I = oracle.knn(x.numpy(), xb, k)
        return torch.from_numpy(D), torch.from_numpy(I)

    D1, I1 = shard.replicated_search(local, torch.from_numpy(xq), 5)
    D2, I2 = shard.sharded_search(local, torch.from_numpy(xq), 5, merge=_cpu_merge)
    assert torch.equal(I1, I2) and torch.equal(D1, D2)
