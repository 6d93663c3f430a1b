"""Replica coordination for runs on several GPUs of one node.

The sort has no exchange step: a workload (one table, a batch of lists, a
request stream) is either replicated per GPU or split into independent units
(lists, requests) routed to ranks on the host.  Nothing here moves sorted
data between GPUs; the only collectives are the barrier and the reductions of
the timing, over whatever process group the caller initialised (NCCL on GPUs,
gloo on CPU).
"""
from __future__ import annotations

import heapq


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over all ranks (x itself when no process group is up)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    """The sum of x over all ranks (x itself when no process group is up)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def throughput(words_all_ranks: float, slowest_ms: float) -> float:
    """Whole-job Mwords/s: every rank's words over the slowest rank's time."""
    return words_all_ranks / (slowest_ms * 1e-3) / 1e6


def route(sizes, world: int) -> list[list[int]]:
    """Assigns independent units (list or request sizes) to world ranks:
    largest first, each to the least loaded rank (ties to the lowest rank), so
    no rank carries more than the mean load plus one unit.  Deterministic;
    returns the unit indices of every rank in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(u) for u in out]


def shard_lists(sizes, world: int, rank: int):
    """The lists rank `rank` of `world` sorts (route's share, ascending list
    ids) and, for the concatenated arrays of all lists, the first word of
    each: returns (ids, starts) with starts[i] the offset of list i."""
    import numpy as np
    sizes = np.asarray(sizes, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]) if sizes.size else np.zeros(0, np.int64)
    return np.asarray(route(sizes, world)[rank], dtype=np.int64), starts


def gather_shard(rec, ln, sizes, ids, starts):
    """This rank's lists, back to back: (rec, len, sizes) of lists `ids`."""
    import numpy as np
    W = rec.shape[1]
    if len(ids) == 0:
        return np.zeros((0, W), rec.dtype), np.zeros(0, ln.dtype), np.zeros(0, np.int64)
    parts = [(int(starts[i]), int(sizes[i])) for i in ids]
    r = np.concatenate([rec[a:a + m] for a, m in parts])
    l = np.concatenate([ln[a:a + m] for a, m in parts])
    return r, l, np.asarray([m for _, m in parts], dtype=np.int64)


def sort_shard(rec, ln, sizes, world: int, rank: int, W: int, max_list_words: int,
               alg="merge", tune=None):
    """Sorts rank `rank`'s share of independent lists (given for the whole
    batch, concatenated) in one batched call on this rank's GPU; returns
    (ids, BatchSorter, descriptors) so that list ids[k] is result k."""
    import torch
    from . import batch
    ids, starts = shard_lists(sizes, world, rank)
    r, l, sz = gather_shard(rec, ln, sizes, ids, starts)
    desc = batch.record_lists(sz)
    b = batch.BatchSorter(max(int(l.size), 1), max(len(sz), 1), W)
    if len(sz):
        b.set_lists(desc)
        b.run(torch.from_numpy(r).cuda(), torch.from_numpy(l).cuda(), text=False,
              max_list_words=max_list_words, alg=alg, tune=tune)
    return ids, b, desc
