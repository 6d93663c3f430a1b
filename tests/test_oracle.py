"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of the oracle's own code: hand-worked examples
(tests/golden), a regular-expression tokeniser, Python's sort, brute-force
enumeration, closed forms of bubble sort (§2, §3.2: n(n-1)/2 exchanges for a
reversed list; exchanges = inversions) and output invariants.
"""
from __future__ import annotations

import itertools
import re

import numpy as np
import pytest

from conftest import load_golden, sort_key_order
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def words_table(words: list[bytes], W: int):
    rec = np.zeros((len(words), W), dtype=np.uint8)
    ln = np.zeros(len(words), dtype=np.uint8)
    for i, w in enumerate(words):
        rec[i, :len(w)] = np.frombuffer(w, np.uint8)
        ln[i] = len(w)
    return rec, ln


def inversions(seq) -> int:
    """Counts pairs i < j with seq[i] > seq[j] by merge sort (independent of bubble sort)."""
    def rec(a):
        if len(a) <= 1:
            return a, 0
        m = len(a) // 2
        l, x = rec(a[:m])
        r, y = rec(a[m:])
        out, inv, i, j = [], x + y, 0, 0
        while i < len(l) and j < len(r):
            if r[j] < l[i]:
                out.append(r[j]); j += 1; inv += len(l) - i
            else:
                out.append(l[i]); i += 1
        out += l[i:] + r[j:]
        return out, inv
    return rec(list(seq))[1]


def check_invariants(rec, ln, res, W):
    n = ln.size
    perm = res.out_perm.astype(np.int64)
    # perm is a bijection on 0..n-1
    assert sorted(perm.tolist()) == list(range(n))
    # out_rec[r] == rec[perm[r]] (records are zero padded)
    assert np.array_equal(res.out_rec, rec[perm])
    # (length, bytes, index) strictly increasing
    keys = [(int(ln[p]), bytes(rec[p, :ln[p]]), int(p)) for p in perm]
    assert all(keys[i] < keys[i + 1] for i in range(n - 1))
    # off[] = prefix sums of the length histogram
    hist = np.bincount(ln, minlength=W + 1)[:W + 1]
    expect = np.concatenate([[0], np.cumsum(hist)]).astype(np.uint32)
    assert np.array_equal(res.off, expect)
    # padding bytes after each word are zero
    for r in range(n):
        assert not res.out_rec[r, ln[perm[r]]:].any()


# --------------------------------------------------------------------------
# Hand-worked examples
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
@pytest.mark.parametrize("method", ["bubble", "stable"])
def test_golden(orc, case, method):
    st, w, res = orc.sort_text(case["text"], case["W"], method)
    assert st == case["status"]
    if st != 0:
        return
    got = [bytes(res.out_rec[r, :w.len[res.out_perm[r]]]) for r in range(w.n)]
    assert got == case["words"]
    assert res.out_perm.tolist() == case["perm"]
    W = case["W"]
    counts = {L: int(res.off[L + 1] - res.off[L]) for L in range(1, W + 1)
              if res.off[L + 1] > res.off[L]}
    assert counts == case["counts"]
    if "swaps" in case and method == "bubble":
        assert {L: int(res.swaps[L]) for L in range(1, W + 1) if res.swaps[L]} == case["swaps"]
    if "packed" in case:
        b, offsets = orc.pack_words(res.out_rec, w.len[res.out_perm])
        assert bytes(b) == case["packed"]
        assert offsets.tolist() == case["offsets"]


# --------------------------------------------------------------------------
# Phase 1: tokeniser against a regular expression over all 256 byte values
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_tokenize_matches_regex(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 4000))
    # mix uniform bytes with letter runs so words of all lengths appear
    t = rng.integers(0, 256, size=n, dtype=np.uint8)
    runs = rng.random(n) < 0.6
    t[runs] = rng.choice(np.frombuffer(b"abcXYZazAZ", np.uint8), size=int(runs.sum()))
    text = bytes(t)
    W = 255
    st, w, nw = orc.tokenize(text, W)
    found = [(m.start(), m.group()) for m in re.finditer(rb"[A-Za-z]+", text)]
    assert st == 0 and nw == len(found)
    for i, (s, word) in enumerate(found):
        assert w.src_off[i] == s
        assert w.len[i] == len(word)
        assert bytes(w.rec[i, :len(word)]) == word
        assert not w.rec[i, len(word):].any()


def test_tokenize_letter_boundaries(orc):
    # every byte value on its own between spaces: exactly the 52 ASCII letters are words
    text = b" ".join(bytes([b]) for b in range(256))
    st, w, nw = orc.tokenize(text, 8)
    assert st == 0
    got = sorted(bytes(w.rec[i, :1]) for i in range(nw))
    assert got == sorted(bytes([b]) for b in range(256) if chr(b).isascii() and chr(b).isalpha())


def test_tokenize_errors(orc):
    assert orc.tokenize(b"a" * 9, 8)[0] == orc.E_WORD_TOO_LONG
    assert orc.tokenize(b"a" * 8, 8)[0] == orc.OK
    st, _, nw = orc.tokenize(b"a b c d", 8, max_words=3)
    assert st == orc.E_CAPACITY and nw == 4
    # both errors: the smaller code is reported
    assert orc.tokenize(b"a b c " + b"x" * 20, 8, max_words=2)[0] == orc.E_WORD_TOO_LONG


# --------------------------------------------------------------------------
# Phases 2-3: against Python's sort, invariants and brute force
# --------------------------------------------------------------------------

def random_table(seed, n, W, alphabet=None, high_bytes=False):
    rng = np.random.default_rng(seed)
    ln = rng.integers(1, W + 1, size=n).astype(np.uint8)
    if alphabet is None:
        lo, hi = (1, 256) if high_bytes else (97, 123)
        rec = rng.integers(lo, hi, size=(n, W)).astype(np.uint8)
    else:
        a = np.frombuffer(alphabet, np.uint8)
        rec = a[rng.integers(0, a.size, size=(n, W))]
    rec[np.arange(W)[None, :] >= ln[:, None]] = 0
    return rec, ln


@pytest.mark.parametrize("seed,n,W,alpha,high", [
    (0, 300, 8, b"ab", False), (1, 500, 16, b"abc", False), (2, 400, 32, None, False),
    (3, 600, 8, None, True), (4, 1, 8, None, False), (5, 0, 8, None, False),
    (6, 700, 24, b"aA", False)])
def test_sort_matches_python_sort(orc, seed, n, W, alpha, high):
    rec, ln = random_table(seed, n, W, alpha, high)
    w = orc.Words(rec, ln)
    expect = sort_key_order(rec, ln)
    b = orc.bubble_sort(w)
    s = orc.stable_sort(w)
    assert b.status == 0 and s.status == 0
    assert b.out_perm.tolist() == expect
    assert s.out_perm.tolist() == expect
    assert np.array_equal(b.out_rec, s.out_rec) and np.array_equal(b.off, s.off)
    check_invariants(rec, ln, b, W)
    # bubble sort makes exactly one exchange per inversion in each length group
    for L in range(1, W + 1):
        ids = np.flatnonzero(ln == L)
        assert int(b.swaps[L]) == inversions([bytes(rec[i, :L]) for i in ids])


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 9))
    W = 8
    rec, ln = random_table(1000 + seed, n, 3, b"abc")
    rec8 = np.zeros((n, W), np.uint8)
    rec8[:, :3] = rec
    keys = [(int(ln[i]), bytes(rec8[i, :ln[i]]), i) for i in range(n)]
    ordered = [p for p in itertools.permutations(range(n))
               if all(keys[p[k]] <= keys[p[k + 1]] for k in range(n - 1))]
    assert len(ordered) == 1
    res = orc.bubble_sort(orc.Words(rec8, ln))
    assert res.out_perm.tolist() == list(ordered[0])


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_reverse_sorted_swaps(orc):
    m = 200
    words = [bytes([97 + (k // 26) % 26, 97 + k % 26, 97]) for k in range(m)][::-1]
    rec, ln = words_table(words, 8)
    res = orc.bubble_sort(orc.Words(rec, ln))
    assert res.out_perm.tolist() == list(range(m))[::-1]
    assert int(res.swaps[3]) == m * (m - 1) // 2


def test_identical_and_sorted_are_identity(orc):
    rec, ln = words_table([b"same"] * 50, 8)
    res = orc.bubble_sort(orc.Words(rec, ln))
    assert res.out_perm.tolist() == list(range(50)) and int(res.swaps.sum()) == 0
    words = sorted({bytes(r[:l]) for r, l in zip(*random_table(7, 300, 8))},
                   key=lambda x: (len(x), x))
    rec, ln = words_table(words, 8)
    res = orc.bubble_sort(orc.Words(rec, ln))
    assert res.out_perm.tolist() == list(range(len(words))) and int(res.swaps.sum()) == 0


def test_length_errors(orc):
    rec, ln = words_table([b"ab", b"c"], 8)
    ln2 = ln.copy(); ln2[1] = 0
    assert orc.bubble_sort(orc.Words(rec, ln2)).status == orc.E_INVALID
    ln3 = ln.copy(); ln3[0] = 9
    assert orc.stable_sort(orc.Words(rec, ln3)).status == orc.E_WORD_TOO_LONG


def test_split_by_length(orc):
    rec, ln = random_table(11, 500, 16)
    st, off, ids = orc.split_by_length(ln, 16)
    assert st == 0
    expect = sorted(range(500), key=lambda i: (int(ln[i]), i))
    assert ids.tolist() == expect
    assert off[0] == 0 and off[17] == 500


# --------------------------------------------------------------------------
# The synthetic workloads: oracle answer is consistent on a sample
# --------------------------------------------------------------------------

def test_prose_sample_bubble_equals_stable(orc):
    text = synth.prose(0, 4096, 4500)
    st, w, nw = orc.tokenize(text, 16)
    assert st == 0 and nw == 4096
    b = orc.bubble_sort(w)
    s = orc.stable_sort(w)
    assert np.array_equal(b.out_perm, s.out_perm)
    check_invariants(w.rec, w.len, b, 16)


# --------------------------------------------------------------------------
# The whole file sorted without length sub-arrays (Table 2, second row)
# --------------------------------------------------------------------------

def whole_order(rec, ln):
    """Input indices in (byte string, index) order: Python's own sort."""
    return sorted(range(ln.size), key=lambda i: (bytes(rec[i, :ln[i]]), i))


def test_whole_hand_worked(orc):
    # "b", "ab", "a", "ab": a proper prefix first, equal words in input order;
    # bubble sort exchanges once per inversion: (b,ab) (b,a) (b,ab) (ab,a)
    rec, ln = words_table([b"b", b"ab", b"a", b"ab"], 8)
    b = orc.bubble_sort_whole(orc.Words(rec, ln))
    assert b.status == 0
    assert b.out_perm.tolist() == [2, 1, 3, 0]
    assert b.swaps == 4
    assert [bytes(r).rstrip(b"\0") for r in b.out_rec] == [b"a", b"ab", b"ab", b"b"]


@pytest.mark.parametrize("seed,n,W,alpha,high", [
    (10, 300, 8, b"ab", False), (11, 500, 16, b"abc", False), (12, 400, 32, None, False),
    (13, 600, 8, None, True), (14, 1, 8, None, False), (15, 0, 8, None, False),
    (16, 700, 24, b"aA", False)])
def test_whole_matches_python_sort(orc, seed, n, W, alpha, high):
    rec, ln = random_table(seed, n, W, alpha, high)
    w = orc.Words(rec, ln)
    expect = whole_order(rec, ln)
    b = orc.bubble_sort_whole(w)
    s = orc.stable_sort_whole(w)
    assert b.status == 0 and s.status == 0
    assert b.out_perm.tolist() == expect and s.out_perm.tolist() == expect
    assert np.array_equal(b.out_rec, s.out_rec)
    for r, i in enumerate(expect):
        assert np.array_equal(b.out_rec[r], rec[i])
    # one exchange per inversion of the byte strings (independent merge count)
    assert b.swaps == inversions([bytes(rec[i, :ln[i]]) for i in range(n)])


@pytest.mark.parametrize("seed", range(8))
def test_whole_brute_force_tiny(orc, seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 8))
    rec, ln = random_table(2000 + seed, n, 3, b"ab")
    keys = [(bytes(rec[i, :ln[i]]), i) for i in range(n)]
    ordered = [p for p in itertools.permutations(range(n))
               if all(keys[p[k]] <= keys[p[k + 1]] for k in range(n - 1))]
    assert len(ordered) == 1
    assert orc.bubble_sort_whole(orc.Words(rec, ln)).out_perm.tolist() == list(ordered[0])


def test_whole_reverse_sorted_swaps_and_differs_from_bucketed(orc):
    # distinct words in descending byte order: m(m-1)/2 exchanges (§3.2 worst case)
    m = 120
    words = sorted({bytes([97 + (k * 7) % 26] * (1 + k % 5)) + bytes([97 + k % 26]) for k in range(400)},
                   reverse=True)[:m]
    rec, ln = words_table(words, 8)
    b = orc.bubble_sort_whole(orc.Words(rec, ln))
    assert b.swaps == m * (m - 1) // 2
    assert b.out_perm.tolist() == list(range(m))[::-1]
    # the length-bucketed answer puts shorter words first instead
    assert orc.stable_sort(orc.Words(rec, ln)).out_perm.tolist() != b.out_perm.tolist()


def test_whole_length_errors(orc):
    rec = np.zeros((2, 8), np.uint8)
    assert orc.bubble_sort_whole(orc.Words(rec, np.array([0, 1], np.uint8))).status == 1
    assert orc.stable_sort_whole(orc.Words(rec, np.array([1, 9], np.uint8))).status == 2


# --------------------------------------------------------------------------
# Packed output ("vectors of string", §3.1)
# --------------------------------------------------------------------------

def test_pack_words_round_trip(orc):
    rec, ln = random_table(21, 500, 16, b"abcXYZ")
    res = orc.stable_sort(orc.Words(rec, ln))
    out_len = ln[res.out_perm]
    buf, offs = orc.pack_words(res.out_rec, out_len)
    assert offs[0] == 0 and int(offs[-1]) == int(ln.sum()) == buf.size
    assert np.all(np.diff(offs.astype(np.int64)) == out_len)
    # unpacking and padding gives the records back
    for r in range(ln.size):
        word = bytes(buf[offs[r]:offs[r + 1]])
        assert word == bytes(rec[res.out_perm[r], :ln[res.out_perm[r]]])
        assert word + b"\0" * (16 - len(word)) == bytes(res.out_rec[r])


def test_pack_words_hand_worked(orc):
    rec, ln = words_table([b"bb", b"a", b"ab"], 8)
    res = orc.stable_sort(orc.Words(rec, ln))  # length first: a, ab, bb
    buf, offs = orc.pack_words(res.out_rec, ln[res.out_perm])
    assert bytes(buf) == b"aabbb" and offs.tolist() == [0, 1, 3, 5]
