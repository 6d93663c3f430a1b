"""GPU parity of the batched call (bsort_sort_many): every list against the
oracle alone, bit for bit, in record and text mode, for every algorithm; the
same list gives the same bytes alone and inside a mix; per-list errors stay
with their list; a CUDA-graph replay gives the same result as a direct call.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda, table, to_dev
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import batch
    bs._lib.load()
    return torch, bs, batch, orc


def concat(lists, W):
    rec = np.concatenate([r for r, _ in lists]) if lists else np.zeros((0, W), np.uint8)
    ln = np.concatenate([l for _, l in lists]) if lists else np.zeros(0, np.uint8)
    return np.ascontiguousarray(rec), np.ascontiguousarray(ln)


def check_list(bsorter, desc, i, rec, ln, orc):
    st, out_rec, perm, off = bsorter.result(i, desc)
    expect = orc.stable_sort(orc.Words(rec, ln)) if ln.size > 3000 else \
        orc.bubble_sort(orc.Words(rec, ln))
    assert st == 0, f"list {i}: status {st}"
    assert np.array_equal(off, expect.off), f"list {i}: offsets"
    assert np.array_equal(perm, expect.out_perm), f"list {i}: permutation"
    assert np.array_equal(out_rec, expect.out_rec), f"list {i}: records"


@pytest.mark.parametrize("alg", ["merge", "odd_even", "auto"])
def test_record_lists_match_oracle(env, alg):
    torch, bs, batch, orc = env
    W = 16
    sizes = [0, 1, 2, 63, 64, 1000, 4096, 4097, 9000, 30_000, 5]
    lists = [synth.list_words(100 + i, m, 50_000, W) for i, m in enumerate(sizes)]
    rec, ln = concat(lists, W)
    desc = batch.record_lists(sizes)
    b = batch.BatchSorter(ln.size, len(sizes), W)
    b.set_lists(desc)
    b.run(to_dev(rec, torch), to_dev(ln, torch), text=False, max_list_words=max(sizes), alg=alg)
    torch.cuda.synchronize()
    for i, (r, l) in enumerate(lists):
        check_list(b, desc, i, r, l, orc)


def test_text_lists_match_oracle(env):
    torch, bs, batch, orc = env
    W = 16
    texts = [synth.prose(7 + i, m, 4500) for i, m in enumerate([1, 50, 3000, 20_000, 700])]
    texts.insert(2, b"")
    texts.append(b"12 !? ,,")
    tbytes = b"".join(texts)
    maxw = [len(t) // 2 + 1 for t in texts]
    desc = batch.text_lists([len(t) for t in texts], maxw)
    b = batch.BatchSorter(int(sum(maxw)), len(texts), W)
    b.set_lists(desc)
    b.run(to_dev(np.frombuffer(tbytes, np.uint8), torch), None, text=True,
          max_list_words=max(maxw), alg="merge")
    torch.cuda.synchronize()
    for i, t in enumerate(texts):
        st, w, expect = orc.sort_text(t, W, "stable")
        assert st == 0
        st2, out_rec, perm, off = b.result(i, desc)
        assert st2 == 0
        assert np.array_equal(off, expect.off)
        assert np.array_equal(perm, expect.out_perm)
        assert np.array_equal(out_rec, expect.out_rec)


def test_alone_equals_in_mix(env):
    torch, bs, batch, orc = env
    W = 16
    sizes = [5000, 70, 12_000, 300]
    lists = [synth.list_words(500 + i, m, 50_000, W) for i, m in enumerate(sizes)]
    rec, ln = concat(lists, W)
    desc = batch.record_lists(sizes)
    mix = batch.BatchSorter(ln.size, len(sizes), W)
    mix.set_lists(desc)
    mix.run(to_dev(rec, torch), to_dev(ln, torch), text=False, max_list_words=max(sizes))
    torch.cuda.synchronize()
    for i, (r, l) in enumerate(lists):
        alone = batch.BatchSorter(l.size, 1, W)
        d1 = batch.record_lists([l.size])
        alone.set_lists(d1)
        alone.run(to_dev(r, torch), to_dev(l, torch), text=False, max_list_words=l.size)
        torch.cuda.synchronize()
        a = alone.result(0, d1)
        m = mix.result(i, desc)
        assert a[0] == m[0] == 0
        for x, y in zip(a[1:], m[1:]):
            assert np.array_equal(x, y)


def test_per_list_errors(env):
    torch, bs, batch, orc = env
    W = 8
    good = table(1, 500, W)
    bad_long = table(2, 300, W)
    bad_long[1][7] = W + 1          # a length above W
    bad_zero = table(3, 200, W)
    bad_zero[1][0] = 0              # a zero length
    lists = [good, bad_long, bad_zero, table(4, 100, W)]
    rec, ln = concat(lists, W)
    sizes = [l.size for _, l in lists]
    desc = batch.record_lists(sizes)
    desc["n_words"][3] = 101        # more words than the list's capacity
    b = batch.BatchSorter(ln.size + 64, len(lists), W)
    b.set_lists(desc)
    b.run(to_dev(rec, torch), to_dev(ln, torch), text=False, max_list_words=1000)
    torch.cuda.synchronize()
    st = b.status[:4].cpu().numpy().tolist()
    assert st == [0, 2, 1, 3]
    check_list(b, desc, 0, *good, orc)


def test_graph_replay_equals_direct(env):
    torch, bs, batch, orc = env
    W = 16
    rec, ln, sizes = synth.batch_lists(64, V=50_000, width=W, seed0=0)
    desc = batch.record_lists(sizes)
    b = batch.BatchSorter(ln.size, len(sizes), W)
    b.set_lists(desc)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    b.run(d_rec, d_len, text=False, max_list_words=65_536)
    torch.cuda.synchronize()
    direct = (b.out_rec.clone(), b.out_perm.clone(), b.out_off.clone())
    b.out_rec.zero_()
    b.out_perm.zero_()
    b.capture(d_rec, d_len, text=False, max_list_words=65_536)
    b.out_rec.zero_()
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(direct[0], b.out_rec) and torch.equal(direct[1], b.out_perm)
    assert torch.equal(direct[2], b.out_off)
    assert int(b.status[:len(sizes)].abs().sum()) == 0
    # spot-check a few lists against the oracle
    starts = np.concatenate([[0], np.cumsum(sizes)])
    for i in (0, 17, 63):
        r, l = rec[starts[i]:starts[i + 1]], ln[starts[i]:starts[i + 1]]
        check_list(b, desc, i, r, l, orc)


@pytest.mark.parametrize("cross", [1, 128, 2048])
def test_crossover_keeps_every_list(env, cross):
    """(list, length) buckets of at most cross words take the odd-even tile,
    larger ones bitonic tiles and merges; every list stays the oracle's."""
    torch, bs, batch, orc = env
    W = 16
    sizes = [70, 900, 2100, 30_000, 5]
    lists = [synth.list_words(800 + i, m, 50_000, W) for i, m in enumerate(sizes)]
    rec, ln = concat(lists, W)
    desc = batch.record_lists(sizes)
    b = batch.BatchSorter(ln.size, len(sizes), W)
    b.set_lists(desc)
    b.run(to_dev(rec, torch), to_dev(ln, torch), text=False, max_list_words=max(sizes),
          alg="merge", tune=dict(tile=2048, oddeven_cross=cross))
    torch.cuda.synchronize()
    for i, (r, l) in enumerate(lists):
        check_list(b, desc, i, r, l, orc)


def test_sharded_batch_every_list_matches_oracle(env):
    """The batch split over two ranks by the host router (each share sorted by
    its own batched call, here one after the other on this GPU): every list of
    every share is the oracle's answer for that list."""
    torch, bs, batch, orc = env
    from paper_1411_5283_gb300 import replicas
    W = 16
    rec, ln, sizes = synth.batch_lists(96, V=50_000, width=W, seed0=900)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    seen = []
    for rank in range(2):
        ids, b, desc = replicas.sort_shard(rec, ln, sizes, 2, rank, W, max_list_words=65_536)
        torch.cuda.synchronize()
        for k, i in enumerate(ids):
            a, z = int(starts[i]), int(starts[i + 1])
            check_list(b, desc, k, rec[a:z], ln[a:z], orc)
        seen += list(ids)
    assert sorted(seen) == list(range(len(sizes)))
