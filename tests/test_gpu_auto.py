"""GPU parity of the sample-sort strategy (alg="auto", n >= 65,536 words).

Expected answers come from the oracle only (stable-sort formulation, itself
pinned against the bubble sort).  Cases cover many buckets, one bucket, one
repeated word, the text path with the word count on the device, and an input
built so that the stratified sample misrepresents the data, which forces the
exact retry pass and the global-memory sort of an oversized segment.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import assert_same_answer, need_cuda, table, to_dev
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
MIXED = bytes(range(ord("A"), ord("Z") + 1)) + bytes(range(ord("a"), ord("z") + 1))


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    return torch, bs, orc


def run(env, rec, ln, alg="auto"):
    torch, bs, _ = env
    n, W = ln.size, rec.shape[1]
    s = bs.Sorter(n, W)
    out = s.sort_records(to_dev(rec, torch), to_dev(ln, torch), n, alg=alg)
    torch.cuda.synchronize()
    return s, out


@pytest.mark.parametrize("n,W", [(70_000, 16), (1_000_000, 32), (300_000, 8), (200_003, 24)])
def test_auto_large_tables(env, n, W):
    torch, bs, orc = env
    rec, ln = synth.large_records(5 + n % 7, n, W) if W in (16, 32) else table(n, n, W)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_auto_one_repeated_word(env):
    torch, bs, orc = env
    n, W = 300_000, 16
    rec = np.zeros((n, W), np.uint8)
    rec[:, :4] = np.frombuffer(b"same", np.uint8)
    ln = np.full(n, 4, np.uint8)
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert np.array_equal(out_perm.cpu().numpy().view(np.uint32), np.arange(n, dtype=np.uint32))
    assert np.array_equal(out_rec.cpu().numpy(), rec)


def test_auto_one_bucket_few_keys(env):
    torch, bs, orc = env
    n, W = 400_000, 8
    rec, ln = table(9, n, W, b"ab", 7, 7)  # 128 distinct words, one bucket
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_auto_text_path(env):
    torch, bs, orc = env
    text = synth.prose(1, 240_000, 12_000)
    st, w, expect = orc.sort_text(text, 16, "stable")
    assert st == 0
    s = bs.Sorter(250_000, 16)
    out_rec, out_perm, off, n_dev, *_ = s.sort_text(to_dev(np.frombuffer(text, np.uint8), torch),
                                                   alg="auto")
    torch.cuda.synchronize()
    assert s.status() == 0
    n = int(n_dev.item())
    assert n == w.n
    assert_same_answer(out_rec, out_perm, off, expect, n)


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_auto_unrepresentative_sample_takes_exact_retry(env):
    """Words at the sampled positions are spread out; every other word is one
    key, so nearly all words land in one segment: the optimistic regions
    overflow, the exact retry runs, and that segment exceeds shared memory."""
    torch, bs, orc = env
    n, W = 120_000, 8
    rng = np.random.default_rng(3)
    rec = np.zeros((n, W), np.uint8)
    rec[:, :5] = np.frombuffer(b"aaaaa", np.uint8)
    ln = np.full(n, 5, np.uint8)
    for s in range((n + 31) // 32):
        i = s * 32 + (_mix64((s + 0x9E3779B97F4A7C15) & M64) & 31)
        if i < n:
            rec[i, :5] = rng.integers(ord("b"), ord("z") + 1, size=5, dtype=np.uint8)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_auto_frequent_words_split_their_buckets(env):
    """Three frequent four-letter words (70% of the words, two of them one
    letter apart) among random ones: the segments at the edges of their runs
    hold a few hundred to a few thousand copies in one bucket of the first
    counting pass, which the block splits again on lower bits, down to the
    index bits that tell copies apart."""
    torch, bs, orc = env
    n, W = 400_000, 8
    rng = np.random.default_rng(17)
    rec = np.zeros((n, W), np.uint8)
    rec[:, :4] = rng.integers(ord("a"), ord("z") + 1, size=(n, 4), dtype=np.uint8)
    pick = rng.random(n)
    for word, lo, hi in ((b"abca", 0.0, 0.40), (b"abcb", 0.40, 0.60), (b"abda", 0.60, 0.70)):
        rec[(pick >= lo) & (pick < hi), :4] = np.frombuffer(word, np.uint8)
    ln = np.full(n, 4, np.uint8)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("L,alphabet", [(8, bytes(range(1, 256))), (12, b"abcdefghijklmnopqrstuvwxyz")])
def test_auto_frequent_words_split_two_part_items(env, L, alphabet):
    """As above with codes too wide for one machine word next to the index:
    eight bytes of any value (one key word) and twelve lower-case letters (two
    key words) make (code, index) items, whose overfull buckets split on the
    code bits first and on the index bits once the code is shared."""
    torch, bs, orc = env
    n, W = 400_000, 16
    rng = np.random.default_rng(19 + L)
    a = np.frombuffer(alphabet, np.uint8)
    rec = np.zeros((n, W), np.uint8)
    rec[:, :L] = a[rng.integers(0, a.size, size=(n, L))]
    pick = rng.random(n)
    base = a[rng.integers(0, a.size, size=L)]
    for k, (lo, hi) in enumerate(((0.0, 0.35), (0.35, 0.55), (0.55, 0.62))):
        w = base.copy()
        w[-1] = a[(k * 7) % a.size]
        rec[(pick >= lo) & (pick < hi), :L] = w
    ln = np.full(n, L, np.uint8)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("L,alphabet", [(4, b"abcdefghijklmnopqrstuvwxyz"), (8, MIXED)])
def test_auto_frequent_word_missed_by_sample_overfills_a_bucket(env, L, alphabet):
    """4,000 copies of one word, all at positions the stratified sample skips,
    among random words: the segment that receives them stays resident but one
    bucket of the first counting pass holds more items than the split copy
    area, so the segment takes the radix passes (one-word items for four
    lower-case letters, two-part items for eight mixed-case ones)."""
    torch, bs, orc = env
    n, W = 120_000, 8
    rng = np.random.default_rng(5)
    rec = np.zeros((n, W), np.uint8)
    a = np.frombuffer(alphabet, np.uint8)
    rec[:, :L] = a[rng.integers(0, a.size, size=(n, L))]
    sampled = np.zeros(n, bool)
    for s in range((n + 31) // 32):
        i = s * 32 + (_mix64((s + 0x9E3779B97F4A7C15) & M64) & 31)
        if i < n:
            sampled[i] = True
    free = np.flatnonzero(~sampled)
    rec[rng.choice(free, 4000, replace=False), :L] = ord("m")
    ln = np.full(n, L, np.uint8)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("alphabet", [bytes(range(256)), b"q", b"pq", MIXED])
def test_auto_byte_ranges(env, alphabet):
    """Segment byte codes follow from the splitters and the range of all bytes
    inside words: every byte value (fields of 8 bits, codes too wide for one
    machine word), a single letter (every field empty), two letters, and
    mixed-case letters (6-bit fields: two-part items from seven letters on)."""
    torch, bs, orc = env
    n, W = 200_000, 16
    rec, ln = table(23, n, W, alphabet)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, (out_rec, out_perm, off) = run(env, rec, ln)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_auto_equals_merge_and_odd_even(env):
    torch, bs, orc = env
    rec, ln = synth.large_records(11, 150_000, 32)
    outs = []
    for alg in ("auto", "merge", "odd_even"):
        s, (out_rec, out_perm, off) = run(env, rec, ln, alg)
        outs.append((out_rec.cpu().numpy(), out_perm.cpu().numpy(), off.cpu().numpy()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
