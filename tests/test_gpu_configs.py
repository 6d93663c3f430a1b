"""GPU parity at the workloads the benchmarks quote, element by element
against the oracle (records, permutation and bucket offsets, bit for bit).

* the 32,768-word text of seed 0 (vocabulary 4,500) under ODD_EVEN, against
  the paper's bubble sort per length;
* the 240,000-word text of seed 1 (vocabulary 12,000) under ODD_EVEN and
  MERGE, against the bubble sort per length;
* the benchmark's table itself: 16,777,216 pre-tokenised 32-byte records of
  seed 2, under AUTO (the benchmarked call) and MERGE, against the oracle's
  stable-sort formulation, and in the one-call packed form against the
  oracle's packing; its first 65,536 words sorted alone against the bubble
  sort;
* the 4,096-list batch (seeds 0..4,095, sizes log-uniform in 64..65,536),
  every list against the oracle;
* served requests up to 1,048,576 words, pre-tokenised and raw text, every
  response against the oracle.

Every expected value comes from the oracle (``oracle/``) on the same seeded
inputs; nothing is derived from the CUDA path.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import assert_same_answer, need_cuda, to_dev
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    return torch, bs, orc


def sort_text_on_gpu(env, text: bytes, W: int, alg: str):
    torch, bs, _ = env
    s = bs.Sorter(len(text) // 2 + 1, W)
    out_rec, out_perm, off, n_dev, *_ = s.sort_text(to_dev(np.frombuffer(text, np.uint8), torch),
                                                   alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    return out_rec, out_perm, off, int(n_dev.item())


@pytest.fixture(scope="module")
def text0(env):
    _, _, orc = env
    text = synth.prose(0, 32_768, 4_500)
    st, w, expect = orc.sort_text(text, 16, "bubble")
    assert st == 0 and w.n == 32_768
    return text, expect


@pytest.fixture(scope="module")
def text1(env):
    _, _, orc = env
    text = synth.prose(1, 240_000, 12_000)
    st, w, expect = orc.sort_text(text, 16, "bubble")
    assert st == 0 and w.n == 240_000
    return text, expect


def test_small_text_odd_even_matches_bubble_sort(env, text0):
    text, expect = text0
    out_rec, out_perm, off, n = sort_text_on_gpu(env, text, 16, "odd_even")
    assert n == 32_768
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("alg", ["odd_even", "merge"])
def test_medium_text_matches_bubble_sort(env, text1, alg):
    text, expect = text1
    out_rec, out_perm, off, n = sort_text_on_gpu(env, text, 16, alg)
    assert n == 240_000
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.fixture(scope="module")
def large(env):
    _, _, orc = env
    rec, ln = synth.large_records(2, 16_777_216, 32)
    expect = orc.stable_sort(orc.Words(rec, ln))
    assert expect.status == 0
    return rec, ln, expect


@pytest.mark.parametrize("alg", ["auto", "merge"])
def test_benchmark_table_matches_oracle(env, large, alg):
    torch, bs, _ = env
    rec, ln, expect = large
    n = ln.size
    s = bs.Sorter(n, 32)
    out_rec, out_perm, off = s.sort_records(to_dev(rec, torch), to_dev(ln, torch), n, alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_benchmark_table_packed_matches_oracle(env, large):
    """The benchmark's table through the one-call packed form (§3.1): bytes,
    offsets, permutation and bucket offsets against the oracle's packing of
    the oracle's answer."""
    torch, bs, orc = env
    rec, ln, expect = large
    n = ln.size
    want_bytes, want_off = orc.pack_words(expect.out_rec, ln[expect.out_perm])
    s = bs.Sorter(n, 32)
    b, offsets, perm, off = s.sort_records_packed(to_dev(rec, torch), to_dev(ln, torch), n,
                                                  alg="auto")
    torch.cuda.synchronize()
    assert s.status() == 0
    assert np.array_equal(offsets.cpu().numpy().view(np.uint32), want_off)
    assert np.array_equal(b[:int(want_off[-1])].cpu().numpy(), want_bytes)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), expect.out_perm)
    assert np.array_equal(off.cpu().numpy().view(np.uint32), expect.off)


def test_benchmark_table_prefix_matches_bubble_sort(env, large):
    """The first 65,536 words of the table: the paper's bubble sort per length
    on the CPU, the benchmarked call on the GPU; and the oracle's two
    formulations agree on it."""
    torch, bs, orc = env
    rec, ln = large[0][:65_536].copy(), large[1][:65_536].copy()
    bubble = orc.bubble_sort(orc.Words(rec, ln))
    stable = orc.stable_sort(orc.Words(rec, ln))
    assert np.array_equal(bubble.out_perm, stable.out_perm)
    s = bs.Sorter(rec.shape[0], 32)
    out_rec, out_perm, off = s.sort_records(to_dev(rec, torch), to_dev(ln, torch), ln.size,
                                            alg="auto")
    torch.cuda.synchronize()
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, bubble, ln.size)


def test_full_batch_every_list_matches_oracle(env):
    torch, bs, orc = env
    from paper_1411_5283_gb300 import autotune, batch
    W = 16
    rec, ln, sizes = synth.batch_lists(4096, V=50_000, width=W, seed0=0)
    assert sizes.max() <= 65_536 and sizes.min() >= 64
    desc = batch.record_lists(sizes)
    b = batch.BatchSorter(int(ln.size), len(sizes), W)
    b.set_lists(desc)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    # the benchmark's configuration: tuned knobs, one graph replay
    tune = autotune.tune_batch(b, d_rec, d_len, text=False, max_list_words=65_536,
                               total_words=int(ln.size), alg="merge", max_candidates=4)
    b.capture(d_rec, d_len, text=False, max_list_words=65_536, alg="merge", tune=tune)
    b.out_rec.zero_()
    b.out_perm.zero_()
    b.replay()
    torch.cuda.synchronize()
    status = b.status[:len(sizes)].cpu().numpy()
    assert not status.any()
    all_rec = b.out_rec[:ln.size].cpu().numpy()
    all_perm = b.out_perm[:ln.size].cpu().numpy().view(np.uint32)
    all_off = b.out_off[:len(sizes)].cpu().numpy().view(np.uint32)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    for i in range(len(sizes)):
        a, z = int(starts[i]), int(starts[i + 1])
        expect = orc.stable_sort(orc.Words(rec[a:z], ln[a:z]))
        assert np.array_equal(all_off[i], expect.off), f"list {i}: offsets"
        assert np.array_equal(all_perm[a:z], expect.out_perm), f"list {i}: permutation"
        assert np.array_equal(all_rec[a:z], expect.out_rec), f"list {i}: records"


def test_served_responses_up_to_a_million_words(env):
    """Requests from the served workload's size law up to its upper end
    (1,048,576 words), raw text among them, checked response by response."""
    torch, bs, orc = env
    from paper_1411_5283_gb300 import serve
    W = 16
    sizes = [1_048_576, 1024, 310_000, 52_000, 700_000, 4_000, 131_072]
    text_at = {1, 4}
    reqs, expects = [], []
    for i, m in enumerate(sizes):
        if i in text_at:
            text = synth.prose(20_000 + i, m, 12_000)
            st, _, res = orc.sort_text(text, W, "stable")
            reqs.append(serve.Request(i, arrival=0.001 * i, text=text, max_words=m))
        else:
            rec, ln = synth.list_words(20_000 + i, m, 50_000, W)
            res = orc.stable_sort(orc.Words(rec, ln))
            st = res.status
            reqs.append(serve.Request(i, arrival=0.001 * i, rec=rec, ln=ln))
        assert st == 0
        expects.append(res)
    srv = serve.Server(W, 1 << 30, max_list_words=1 << 20, max_batch_lists=64)
    stats = srv.run_trace(reqs, release=False)
    assert stats["completed"] == len(sizes) and stats["rejected"] == 0
    for r, res in zip(reqs, expects):
        st, out_rec, perm, off = srv.result(r)
        assert st == 0
        assert np.array_equal(off, res.off), f"request {r.rid}: offsets"
        assert np.array_equal(perm, res.out_perm), f"request {r.rid}: permutation"
        assert np.array_equal(out_rec, res.out_rec), f"request {r.rid}: records"
