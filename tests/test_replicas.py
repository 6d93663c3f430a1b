"""Replica coordination on CPU: two gloo ranks agree on the slowest time and
the whole-job throughput; routing covers every unit exactly once and keeps
the ranks balanced."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_1411_5283_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        my_ms = [3.5, 7.25][rank]
        my_words = [1000, 1000][rank]
        slowest = replicas.max_over_ranks(my_ms)
        words = replicas.sum_over_ranks(my_words)
        units = replicas.route([5, 1, 9, 3, 3, 8, 2], world)[rank]
        q.put((rank, slowest, words, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_and_total():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [7.25, 7.25]
    assert [r[2] for r in res] == [2000.0, 2000.0]
    assert replicas.throughput(2000, 7.25) == pytest.approx(2000 / 7.25e-3 / 1e6)
    # the two ranks' units partition the seven units
    units = sorted(res[0][3] + res[1][3])
    assert units == list(range(7))


def test_single_process_is_identity():
    assert replicas.max_over_ranks(4.0) == 4.0
    assert replicas.sum_over_ranks(4.0) == 4.0


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_route_covers_and_balances(world):
    rng = np.random.default_rng(world)
    sizes = np.exp(rng.uniform(np.log(64), np.log(65_537), size=500)).astype(np.int64)
    parts = replicas.route(sizes, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(sizes.size))
    loads = [int(sizes[p].sum()) for p in parts]
    assert max(loads) <= sizes.sum() / world + sizes.max()
    assert parts == replicas.route(sizes, world)  # deterministic


def test_route_rejects_empty_world():
    with pytest.raises(ValueError):
        replicas.route([1, 2], 0)


def _shard_main(rank, world, port, q):
    """A rank takes its share of a batch of independent lists (the batched
    workload's generator), builds its concatenated arrays and descriptors,
    and reports what it would sort; rank 0 collects every rank's share."""
    import torch.distributed as dist
    from paper_1411_5283_gb300 import batch, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rec, ln, sizes = synth.batch_lists(48, V=50_000, width=16, lo=64, hi=4096, seed0=500)
        ids, starts = replicas.shard_lists(sizes, world, rank)
        r, l, sz = replicas.gather_shard(rec, ln, sizes, ids, starts)
        desc = batch.record_lists(sz)
        # every list of the share is the input's list, at its descriptor's offset
        ok = all(np.array_equal(r[int(desc["word_off"][k]):int(desc["word_off"][k]) + int(sz[k])],
                                rec[int(starts[i]):int(starts[i]) + int(sizes[i])])
                 for k, i in enumerate(ids))
        shares = [None] * world
        dist.all_gather_object(shares, (rank, ids.tolist(), int(l.size), ok))
        if rank == 0:
            q.put((shares, sizes.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_a_list_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    shares, sizes = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids = sorted(i for _, share, _, _ in shares for i in share)
    assert ids == list(range(len(sizes)))                     # every list exactly once
    assert all(ok for *_, ok in shares)                       # shares hold the right words
    words = [w for _, _, w, _ in shares]
    assert sum(words) == sum(sizes)
    assert max(words) <= sum(sizes) / 2 + max(sizes)          # balanced within one list
