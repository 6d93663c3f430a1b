"""GPU parity: every step of the CUDA path against the CPU oracle, bit for bit.

Inputs are seeded synthetic tables / texts (paper_1411_5283_gb300.synth or
small random tables); expected values come from the oracle only.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import assert_same_answer, need_cuda, table, to_dev, u32
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu

ALGS = ["odd_even", "merge", "auto"]


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    return torch, bs, orc


def run_records(env, rec, ln, alg, tune=None, W=None):
    torch, bs, _ = env
    W = rec.shape[1] if W is None else W
    n = ln.size
    s = bs.Sorter(max(n, 1), W)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    out_rec, out_perm, off = s.sort_records(d_rec, d_len, n, alg=alg, tune=tune)
    torch.cuda.synchronize()
    return s, out_rec, out_perm, off


# ---------------------------------------------------------------------------
# Phase 1: tokeniser
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed,n_words", [(0, 32768), (3, 1000), (4, 1)])
def test_tokenize_prose(env, seed, n_words):
    torch, bs, orc = env
    text = synth.prose(seed, n_words, 4500)
    st, w, nw = orc.tokenize(text, 16)
    assert st == 0
    s = bs.Sorter(n_words + 16, 16)
    d_text = to_dev(np.frombuffer(text, np.uint8), torch)
    rec, ln, so, n_dev = s.tokenize(d_text)
    torch.cuda.synchronize()
    assert s.status() == 0
    n = int(n_dev.item())
    assert n == nw == n_words
    assert np.array_equal(rec[:n].cpu().numpy(), w.rec)
    assert np.array_equal(ln[:n].cpu().numpy(), w.len)
    assert np.array_equal(u32(so[:n]), w.src_off)


@pytest.mark.parametrize("seed", range(4))
def test_tokenize_random_bytes(env, seed):
    torch, bs, orc = env
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300_000))
    t = rng.integers(0, 256, size=n, dtype=np.uint8)
    t[rng.random(n) < 0.7] = ord("q")  # long letter runs across block boundaries
    t[rng.random(n) < 0.05] = ord(" ")
    text = bytes(t)
    W = 32
    st, w, nw = orc.tokenize(text, 255)
    too_long = bool((w.len > W).any())
    s = bs.Sorter(nw + 16, W)
    rec, ln, so, n_dev = s.tokenize(to_dev(t, torch))
    torch.cuda.synchronize()
    assert int(n_dev.item()) == nw
    assert s.status() == (2 if too_long else 0)
    ok = w.len <= W
    assert np.array_equal(ln[:nw].cpu().numpy()[ok], w.len[ok])
    assert np.array_equal(u32(so[:nw]), w.src_off)
    assert np.array_equal(rec[:nw].cpu().numpy()[ok], w.rec[ok][:, :W])


def test_tokenize_capacity(env):
    torch, bs, orc = env
    text = b"a b c d e f"
    s = bs.Sorter(16, 8)
    _, _, _, n_dev = s.tokenize(to_dev(np.frombuffer(text, np.uint8), torch), max_words=4)
    torch.cuda.synchronize()
    assert int(n_dev.item()) == 4
    assert s.status() == 3


# ---------------------------------------------------------------------------
# Phase 2: buckets, stable order and big-endian keys
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,W", [(5000, 16), (70_000, 32), (1, 8), (33, 24)])
def test_bucket_by_length(env, n, W):
    torch, bs, orc = env
    rec, ln = table(11 + n, n, W)
    st, off, ids = orc.split_by_length(ln, W)
    s = bs.Sorter(n, W)
    s.bucket_by_length(to_dev(rec, torch), to_dev(ln, torch), n)
    keys, idx = s.export_buckets(n)
    torch.cuda.synchronize()
    assert np.array_equal(u32(s.off), off)
    assert np.array_equal(u32(idx), ids)
    # keys: big-endian packing of each word's bytes, zero past the word
    k = keys.cpu().numpy().view(np.uint64)
    src = rec[ids].reshape(n, W // 8, 8)
    be = np.zeros((n, W // 8), dtype=np.uint64)
    for b in range(8):
        be |= src[:, :, b].astype(np.uint64) << np.uint64(56 - 8 * b)
    assert np.array_equal(k.T, be)


# ---------------------------------------------------------------------------
# Phases 2-3 + concatenation: whole answers
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("n,W,alpha,max_len", [
    (0, 16, b"ab", None), (1, 16, b"ab", None), (7, 8, b"ab", 3), (1000, 16, b"ab", 4),
    (4099, 32, b"abcdefghijklmnopqrstuvwxyz", None), (20_000, 8, b"xyz", 5),
    (12_345, 24, b"aAbB", None), (9000, 16, b"a", 2)])
def test_sort_records_small(env, alg, n, W, alpha, max_len):
    torch, bs, orc = env
    rec, ln = table(n * 7 + W, n, W, alpha, max_len)
    expect = orc.bubble_sort(orc.Words(rec, ln)) if n <= 4100 else orc.stable_sort(orc.Words(rec, ln))
    s, out_rec, out_perm, off = run_records(env, rec, ln, alg)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("alg", ALGS)
def test_sort_high_bytes(env, alg):
    """Pre-tokenised records may hold any byte: order is unsigned."""
    torch, bs, orc = env
    rng = np.random.default_rng(5)
    n, W = 6000, 16
    ln = rng.integers(1, W + 1, size=n).astype(np.uint8)
    rec = rng.integers(1, 256, size=(n, W)).astype(np.uint8)
    rec[rng.random((n, W)) < 0.5] = 0xFF
    rec[np.arange(W)[None, :] >= ln[:, None]] = 0
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, out_rec, out_perm, off = run_records(env, rec, ln, alg)
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("alg", ["merge", "auto"])
@pytest.mark.parametrize("stray", [None, b"@", b"[", b"`", b"{"])
@pytest.mark.parametrize("lens", [(7, 8), (13, 16)])
def test_letter_coded_tiles(env, alg, stray, lens):
    """Tiles of 7- or 8-byte one-key words sort on 6-bit letter codes when
    every word of the tile is letters only, else on the raw keys; bytes just
    outside the letter ranges put some tiles on the raw path.  Two-key words of
    13 to 16 bytes with the same strays check the (keys, index) network."""
    torch, bs, orc = env
    n, W = 60_000, 16
    rec, ln = table(91 + lens[0], n, W, b"aAzZmMbY", lens[1], lens[0])
    if stray is not None:
        rng = np.random.default_rng(92)
        rows = rng.choice(n, size=12, replace=False)
        rec[rows, rng.integers(0, lens[0], size=12)] = stray[0]
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, out_rec, out_perm, off = run_records(env, rec, ln, alg)
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("alg", ALGS)
def test_single_big_bucket_forces_merges(env, alg):
    torch, bs, orc = env
    n, W = 150_000, 16
    rec, ln = table(77, n, W, b"abcd", 6, 6)  # one bucket, many duplicates
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, out_rec, out_perm, off = run_records(env, rec, ln, alg)
    assert_same_answer(out_rec, out_perm, off, expect, n)


@pytest.mark.parametrize("alg", ALGS)
def test_reverse_and_identical(env, alg):
    torch, bs, orc = env
    words = [bytes([97 + (k // 676) % 26, 97 + (k // 26) % 26, 97 + k % 26]) for k in range(9000)]
    words = words[::-1] + [b"zzz"] * 3000
    W = 8
    rec = np.zeros((len(words), W), np.uint8)
    for i, w in enumerate(words):
        rec[i, :3] = np.frombuffer(w, np.uint8)
    ln = np.full(len(words), 3, np.uint8)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, out_rec, out_perm, off = run_records(env, rec, ln, alg)
    assert_same_answer(out_rec, out_perm, off, expect, len(words))


@pytest.mark.parametrize("tune", [dict(tile=256, merge_fanin=256), dict(tile=4096),
                                  dict(oddeven_max=64), dict(oddeven_max=2048),
                                  dict(threads_per_bucket=512, tile=1024, merge_fanin=1024)])
def test_tuning_does_not_change_answer(env, tune):
    torch, bs, orc = env
    rec, ln = table(3, 30_000, 16, b"abcdefg", 7)
    expect = orc.stable_sort(orc.Words(rec, ln))
    for alg in ("odd_even", "merge"):
        s, out_rec, out_perm, off = run_records(env, rec, ln, alg, tune=tune)
        assert_same_answer(out_rec, out_perm, off, expect, ln.size)


def test_phase_by_phase_equals_one_call(env):
    torch, bs, orc = env
    rec, ln = table(8, 40_000, 16)
    n = ln.size
    expect = orc.stable_sort(orc.Words(rec, ln))
    s = bs.Sorter(n, 16)
    s.bucket_by_length(to_dev(rec, torch), to_dev(ln, torch), n)
    s.sort_buckets(n, alg="merge")
    out_rec, out_perm, off = s.gather(n)
    torch.cuda.synchronize()
    assert_same_answer(out_rec, out_perm, off, expect, n)


# ---------------------------------------------------------------------------
# Raw text end to end (configuration-0 shape) and errors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alg", ALGS)
def test_sort_text_prose(env, alg):
    torch, bs, orc = env
    text = synth.prose(0, 32768, 4500)
    st, w, expect = orc.sort_text(text, 16, "bubble")
    assert st == 0
    s = bs.Sorter(40_000, 16)
    out_rec, out_perm, off, n_dev, *_ = s.sort_text(to_dev(np.frombuffer(text, np.uint8), torch),
                                                   alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    n = int(n_dev.item())
    assert n == w.n
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_errors_reported(env):
    torch, bs, orc = env
    rec, ln = table(1, 100, 8)
    ln[5] = 9
    s, *_ = run_records(env, rec, ln, "merge")
    assert s.status() == 2
    ln[5] = 0
    s, *_ = run_records(env, rec, ln, "merge")
    assert s.status() == 1
    s = bs.Sorter(8, 8)
    with pytest.raises(bs.BsortError):
        s.sort_records(to_dev(rec, torch), to_dev(ln, torch), 100)  # workspace too small
    text = b"ok " + b"x" * 40
    s = bs.Sorter(16, 32)
    s.sort_text(to_dev(np.frombuffer(text, np.uint8), torch))
    assert s.status() == 2


@pytest.mark.parametrize("cross", [1, 2, 64, 700, 2048])
def test_odd_even_merge_crossover_keeps_the_answer(env, cross):
    """Buckets from a handful of words (lengths near 32) to tens of thousands
    (length 3): with the crossover at cross, buckets of at most cross words
    are sorted whole by odd-even transposition, the rest by bitonic tiles and
    merges; the answer is the oracle's for every crossover."""
    torch, bs, orc = env
    rec, ln = synth.large_records(13, 60_000, 32)
    counts = np.bincount(ln, minlength=33)[1:]
    assert counts.min() <= 64 and counts.max() > 2048  # buckets on both sides
    expect = orc.stable_sort(orc.Words(rec, ln))
    s, out_rec, out_perm, off = run_records(env, rec, ln, "merge",
                                            tune=dict(tile=2048, oddeven_cross=cross))
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, ln.size)
