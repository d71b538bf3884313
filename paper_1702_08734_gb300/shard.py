"""Multi-GPU forms of the search (section 5.4), one process per GPU.

* Replication: the queries are split over the ranks, each rank searches its part against
  its full copy of the index, and the results are concatenated in query order.
* Sharding: the database is split over the ranks (each rank indexes its part with global
  ids); every rank searches all queries on its shard, the per-shard top-k lists (nq x k
  values and ids) are gathered, and one more k-selection by (value, id) keeps the k best -
  the same join the paper applies to shard results.

The exchange is ``torch.distributed.all_gather`` over the process group (NCCL between
GPUs; gloo on CPU in the tests).  The join runs in the library (``merge_topk``) unless the
caller passes another function of the same contract.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def part_range(n: int, rank: int, world: int):
    """Contiguous rows [r0, r1) of rank `rank` when n rows are split over `world` ranks
    (the first n % world ranks take one more)."""
    base, extra = divmod(int(n), int(world))
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def _group_world(group):
    return dist.get_world_size(group) if dist.is_initialized() else 1


def gather_rows(t: torch.Tensor, counts, group=None) -> torch.Tensor:
    """Concatenation over the ranks of each rank's rows of t (rank r holds counts[r] rows)."""
    world = _group_world(group)
    if world == 1:
        return t
    m = max(counts)
    pad = torch.zeros((m,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


def replicated_search(search, xq: torch.Tensor, k: int, group=None):
    """Replication: rank r answers queries part_range(nq, r, world) with
    search(xq_part, k) -> (D [n][k], I [n][k]); returns all queries' (D, I) on every rank."""
    world = _group_world(group)
    rank = dist.get_rank(group) if world > 1 else 0
    nq = xq.shape[0]
    r0, r1 = part_range(nq, rank, world)
    D, I = search(xq[r0:r1].contiguous(), k)
    counts = [part_range(nq, r, world)[1] - part_range(nq, r, world)[0] for r in range(world)]
    return gather_rows(D, counts, group), gather_rows(I, counts, group)


def sharded_search(search, xq: torch.Tensor, k: int, group=None, largest: bool = False,
                   merge=None):
    """Sharding: search(xq, k) -> (D [nq][k], I [nq][k] global ids, padding (+-inf, -1)) on
    this rank's shard; the partial lists of all ranks are gathered and joined into the k
    best per query by (value, id).  merge(Dp [S][nq][k], Ip, k, largest) -> (D, I); default
    the library's merge_topk."""
    D, I = search(xq, k)
    world = _group_world(group)
    if world > 1:
        Dp = [torch.empty_like(D) for _ in range(world)]
        Ip = [torch.empty_like(I) for _ in range(world)]
        dist.all_gather(Dp, D.contiguous(), group=group)
        dist.all_gather(Ip, I.contiguous(), group=group)
        Dp, Ip = torch.stack(Dp), torch.stack(Ip)
    else:
        Dp, Ip = D[None], I[None]
    if merge is None:
        from . import merge_topk
        return merge_topk(Dp.contiguous(), Ip.contiguous(), k, largest=largest)
    return merge(Dp, Ip, k, largest)
