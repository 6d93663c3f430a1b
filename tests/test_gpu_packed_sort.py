"""GPU parity of the one-call packed answer (bsort_sort_records_packed,
bsort_sort_text_packed): the sort's last kernel (the AUTO segment sort, or the
gather of the MERGE and ODD_EVEN paths) writes the "vectors of string" form of
§3.1 directly.  Expected bytes and offsets are the oracle's packing of the
oracle's answer; the permutation and bucket offsets are the oracle's too."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda, table, to_dev, u32
from paper_1411_5283_gb300 import synth
from test_gpu_auto import M64, _mix64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    return torch, bs, orc


def check_packed(env, rec, ln, alg, cap=None):
    torch, bs, orc = env
    n, W = ln.size, rec.shape[1]
    expect = orc.stable_sort(orc.Words(rec, ln))
    want_bytes, want_off = orc.pack_words(expect.out_rec, ln[expect.out_perm])
    s = bs.Sorter(max(n, 1), W)
    out_bytes = torch.zeros(max(n * W, 16), dtype=torch.uint8, device="cuda")
    if cap is not None:
        out_bytes = out_bytes[:cap]
    b, offsets, perm, off = s.sort_records_packed(to_dev(rec, torch), to_dev(ln, torch), n,
                                                  alg=alg, out_bytes=out_bytes)
    torch.cuda.synchronize()
    return s, b, offsets, perm, off, expect, want_bytes, want_off


@pytest.mark.parametrize("W,n,alg", [
    (8, 0, "merge"), (8, 1, "odd_even"), (16, 10_000, "merge"), (24, 4097, "odd_even"),
    (32, 5000, "auto"),            # below the sample sort's minimum: the merge path's gather
    (16, 200_000, "auto"), (24, 200_003, "auto"), (8, 300_000, "auto"),
    (32, 1_000_000, "auto"), (32, 150_000, "merge")])
def test_records_packed_matches_oracle(env, W, n, alg):
    torch, bs, orc = env
    rec, ln = synth.large_records(7 + n % 5, n, W) if W in (16, 32) and n >= 100_000 \
        else table(60 + W + n, n, W)
    s, b, offsets, perm, off, expect, want_bytes, want_off = check_packed(env, rec, ln, alg)
    assert s.status() == 0
    assert np.array_equal(u32(offsets), want_off)
    total = int(want_off[-1])
    assert np.array_equal(b[:total].cpu().numpy(), want_bytes)
    assert np.array_equal(u32(perm), expect.out_perm)
    assert np.array_equal(u32(off), expect.off)


def test_records_packed_through_the_exact_retry(env):
    """The sampled positions misrepresent the words, so one segment exceeds
    shared memory after the exact retry and takes the chunked sort."""
    torch, bs, orc = env
    n, W = 120_000, 8
    rng = np.random.default_rng(3)
    rec = np.zeros((n, W), np.uint8)
    rec[:, :5] = np.frombuffer(b"aaaaa", np.uint8)
    ln = np.full(n, 5, np.uint8)
    for g in range((n + 31) // 32):
        i = g * 32 + (_mix64((g + 0x9E3779B97F4A7C15) & M64) & 31)
        if i < n:
            rec[i, :5] = rng.integers(ord("b"), ord("z") + 1, size=5, dtype=np.uint8)
    s, b, offsets, perm, off, expect, want_bytes, want_off = check_packed(env, rec, ln, "auto")
    assert s.status() == 0
    assert np.array_equal(u32(offsets), want_off)
    assert np.array_equal(b[:int(want_off[-1])].cpu().numpy(), want_bytes)
    assert np.array_equal(u32(perm), expect.out_perm)


@pytest.mark.parametrize("alg", ["auto", "merge"])
def test_records_packed_equals_sort_then_pack(env, alg):
    torch, bs, orc = env
    n, W = 250_000, 16
    rec, ln = synth.large_records(11, n, W)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    s = bs.Sorter(n, W)
    _, perm_a, _ = s.sort_records(d_rec, d_len, n, alg=alg)
    perm_a = perm_a.clone()
    b_a, off_a = s.pack(n, bucketed=True)
    b_a, off_a = b_a.clone(), off_a.clone()
    b_b, off_b, perm_b, _ = s.sort_records_packed(d_rec, d_len, n, alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    total = int(u32(off_a)[n])
    assert torch.equal(off_a, off_b) and torch.equal(perm_a, perm_b)
    assert torch.equal(b_a[:total], b_b[:total])


@pytest.mark.parametrize("alg", ["auto", "merge", "odd_even"])
def test_text_packed_uses_the_device_word_count(env, alg):
    torch, bs, orc = env
    text = synth.prose(1, 200_000, 30_000)
    st, w, expect = orc.sort_text(text, 16, "stable")
    want_bytes, want_off = orc.pack_words(expect.out_rec, w.len[expect.out_perm])
    cap_words = len(text) // 2 + 1
    s = bs.Sorter(cap_words, 16)
    b, offsets, perm, off, nw = s.sort_text_packed(to_dev(np.frombuffer(text, np.uint8), torch),
                                                   alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    n = w.n
    assert int(nw.item()) == n
    assert np.array_equal(u32(offsets[:n + 1]), want_off)
    assert np.array_equal(b[:int(want_off[-1])].cpu().numpy(), want_bytes)
    assert np.array_equal(u32(perm[:n]), expect.out_perm)
    assert np.array_equal(u32(off), expect.off)


@pytest.mark.parametrize("alg", ["auto", "merge"])
def test_records_packed_rejects_a_small_buffer(env, alg):
    torch, bs, orc = env
    W, n = 16, 100_000
    rec, ln = table(5, n, W)
    total = int(ln.astype(np.int64).sum())
    s, b, offsets, perm, off, expect, _, want_off = check_packed(env, rec, ln, alg, cap=total - 1)
    assert s.status() == bs._lib.E_CAPACITY
    assert int(u32(offsets)[n]) == 0
    assert np.array_equal(u32(offsets)[:n], want_off[:n])  # the offsets are still written
    assert not b.cpu().numpy().any()  # no byte written
    assert np.array_equal(u32(perm), expect.out_perm)


def test_records_packed_size_limits(env):
    """n W must stay below 2^32 and n at most 2^28: refused before any work."""
    torch, bs, orc = env
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    ws_bytes = bs.bsort_workspace_size(16, 8)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    for n, W in [((1 << 28), 16), ((1 << 28) + 1, 8)]:
        with pytest.raises(bs.BsortError) as e:
            bs.bsort_sort_records_packed(d, d, n, W, "auto", None, d, 64, d, d, d, ws, ws_bytes)
        assert e.value.status == bs._lib.E_CAPACITY


@pytest.mark.parametrize("alg", ["auto", "merge", "odd_even"])
def test_text_packed_hand_worked_examples(env, alg):
    """The hand-worked examples whose packed form is written out in
    tests/golden (§3.1), through the one-call packed text path."""
    torch, bs, orc = env
    from conftest import load_golden
    cases = [c for c in load_golden() if "packed" in c]
    assert cases
    for case in cases:
        text = case["text"]
        s = bs.Sorter(len(text) // 2 + 1, case["W"])
        b, offsets, perm, off, nw = s.sort_text_packed(
            to_dev(np.frombuffer(text, np.uint8), torch), alg=alg)
        torch.cuda.synchronize()
        assert s.status() == 0
        n = int(nw.item())
        assert n == len(case["perm"])
        assert u32(offsets[:n + 1]).tolist() == case["offsets"], case["name"]
        assert bytes(b[:case["offsets"][-1]].cpu().numpy()) == case["packed"], case["name"]
        assert u32(perm[:n]).tolist() == case["perm"], case["name"]
