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
