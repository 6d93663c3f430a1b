"""GPU parity of the unbucketed variant (the paper's Table 2, second row: the
whole file sorted alphabetically without length sub-arrays) against the
oracle's whole-file bubble sort and its stable-sort formulation, bit for bit.

Words compare as unsigned byte strings, a proper prefix first; records may
hold zero bytes inside a word, so "a" and "a\\0" share a padded record and
only their lengths tell them apart.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda, table, to_dev, u32
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    return torch, bs, orc


def run_whole(env, rec, ln, alg):
    torch, bs, _ = env
    n, W = ln.size, rec.shape[1]
    s = bs.Sorter(max(n, 1), W)
    out_rec, out_perm = s.sort_records_whole(to_dev(rec, torch), to_dev(ln, torch), n, alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    return out_rec.cpu().numpy(), u32(out_perm)


def check(env, rec, ln, alg, bubble=False):
    _, _, orc = env
    w = orc.Words(rec, ln)
    expect = orc.bubble_sort_whole(w) if bubble else orc.stable_sort_whole(w)
    assert expect.status == 0
    got_rec, got_perm = run_whole(env, rec, ln, alg)
    if not np.array_equal(got_perm, expect.out_perm):
        bad = np.flatnonzero(got_perm != expect.out_perm)
        raise AssertionError(f"perm differs at {bad.size} ranks, first {bad[:8]}")
    assert np.array_equal(got_rec, expect.out_rec)


def test_prefixes_and_zero_bytes(env):
    W = 8
    words = [b"ab", b"a", b"a\0", b"a\0\0b", b"b", b"a", b"\0", b"\0\0", b"ab\0", b"a\0"]
    rec = np.zeros((len(words), W), np.uint8)
    ln = np.array([len(x) for x in words], np.uint8)
    for i, x in enumerate(words):
        rec[i, :len(x)] = np.frombuffer(x, np.uint8)
    for alg in ("odd_even", "merge", "auto"):
        check(env, rec, ln, alg, bubble=True)


@pytest.mark.parametrize("alg", ["odd_even", "merge", "auto"])
@pytest.mark.parametrize("W,n", [(8, 0), (8, 1), (16, 3000), (24, 2500), (32, 5001)])
def test_small_tables_match_bubble_sort(env, alg, W, n):
    rec, ln = table(60 + W + n, n, W)
    check(env, rec, ln, alg, bubble=True)


@pytest.mark.parametrize("alg", ["merge", "auto"])
@pytest.mark.parametrize("W,n,alphabet", [(16, 70_000, b"abcdefghijklmnopqrstuvwxyz"),
                                          (32, 150_000, b"abc"),
                                          (8, 90_000, bytes(range(256))),
                                          (24, 66_000, b"ab\0")])
def test_tables_match_oracle(env, alg, W, n, alphabet):
    rec, ln = table(7 * W + n, n, W, alphabet)
    check(env, rec, ln, alg)


def test_large_table_matches_oracle(env):
    rec, ln = synth.large_records(9, 1_000_000, 32)
    check(env, rec, ln, "auto")


def test_text_matches_oracle(env):
    torch, bs, orc = env
    text = synth.prose(1, 240_000, 12_000)
    st, w, _ = orc.tokenize(text, 16)
    assert st == 0
    expect = orc.stable_sort_whole(w)
    s = bs.Sorter(len(text) // 2 + 1, 16)
    for alg in ("odd_even", "merge", "auto"):
        out_rec, out_perm, n_dev, *_ = s.sort_text_whole(
            to_dev(np.frombuffer(text, np.uint8), torch), alg=alg)
        torch.cuda.synchronize()
        assert s.status() == 0
        n = int(n_dev.item())
        assert n == w.n
        assert np.array_equal(u32(out_perm[:n]), expect.out_perm)
        assert np.array_equal(out_rec[:n].cpu().numpy(), expect.out_rec)


@pytest.mark.parametrize("W", [8, 24])
def test_permutation_output_off_16_byte_boundary(env, W):
    """The merge levels stage permutation ranges from the 16-byte boundary at
    or below their first entry, so a permutation array that starts 4 bytes
    past a boundary (only 4-byte alignment is required of it) still gives the
    oracle's answer; W = 8 and 24 put odd records off 16-byte boundaries."""
    torch, bs, orc = env
    n = 40_000
    rec, ln = table(300 + W, n, W, b"abcdefgh")
    w = orc.Words(rec, ln)
    expect = orc.stable_sort_whole(w)
    s = bs.Sorter(n, W)
    perm_buf = torch.empty(n + 4, dtype=torch.int32, device="cuda")
    out_perm = perm_buf[1:n + 1]
    bs._lib.bsort_sort_records_whole(to_dev(rec, torch), to_dev(ln, torch), n, W, "auto", None, s.out_rec,
                                     out_perm, s.ws, s.ws_bytes)
    torch.cuda.synchronize()
    assert s.status() == 0
    assert np.array_equal(u32(out_perm), expect.out_perm)
    assert np.array_equal(s.out_rec[:n].cpu().numpy(), expect.out_rec)
