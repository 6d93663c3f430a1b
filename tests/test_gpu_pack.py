"""GPU parity of the packed "vectors of string" output (the paper's §3.1
alternative to the fixed-width char array): the sorted words back to back
without padding plus offsets[n + 1], against the oracle's packing of the
oracle's answer, bit for bit, for the bucketed and the unbucketed order."""
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


def packed_on_gpu(env, s, n, bucketed, d_perm=None, d_len=None, cap=None):
    torch, bs, _ = env
    out_bytes = torch.zeros(max(n * s.W if cap is None else cap, 16), dtype=torch.uint8,
                            device="cuda")
    if cap is not None:
        out_bytes = out_bytes[:cap] if cap else out_bytes[:0]
    b, offsets = s.pack(n, bucketed=bucketed, perm=d_perm, ln=d_len, out_bytes=out_bytes)
    torch.cuda.synchronize()
    return b, offsets


@pytest.mark.parametrize("W,n,alg", [(8, 0, "merge"), (8, 1, "odd_even"), (16, 10_000, "merge"),
                                     (24, 4097, "odd_even"), (32, 300_000, "auto")])
def test_bucketed_pack_matches_oracle(env, W, n, alg):
    torch, bs, orc = env
    rec, ln = table(80 + W + n, n, W) if n < 100_000 else synth.large_records(3, n, W)
    expect = orc.stable_sort(orc.Words(rec, ln))
    want_bytes, want_off = orc.pack_words(expect.out_rec, ln[expect.out_perm])
    s = bs.Sorter(max(n, 1), W)
    s.sort_records(to_dev(rec, torch), to_dev(ln, torch), n, alg=alg)
    b, offsets = packed_on_gpu(env, s, n, True)
    assert s.status() == 0
    assert np.array_equal(u32(offsets), want_off)
    total = int(want_off[-1])
    assert np.array_equal(b[:total].cpu().numpy(), want_bytes)


@pytest.mark.parametrize("W,n,alg", [(16, 5000, "merge"), (32, 120_000, "auto"),
                                     (8, 3000, "odd_even")])
def test_unbucketed_pack_matches_oracle(env, W, n, alg):
    torch, bs, orc = env
    rec, ln = table(90 + W + n, n, W, b"ab\0cd")
    expect = orc.stable_sort_whole(orc.Words(rec, ln))
    want_bytes, want_off = orc.pack_words(expect.out_rec, ln[expect.out_perm])
    s = bs.Sorter(n, W)
    d_len = to_dev(ln, torch)
    _, out_perm = s.sort_records_whole(to_dev(rec, torch), d_len, n, alg=alg)
    b, offsets = packed_on_gpu(env, s, n, False, d_perm=out_perm, d_len=d_len)
    assert s.status() == 0
    assert np.array_equal(u32(offsets), want_off)
    assert np.array_equal(b[:int(want_off[-1])].cpu().numpy(), want_bytes)


def test_text_pack_uses_the_device_word_count(env):
    torch, bs, orc = env
    text = synth.prose(0, 32_768, 4_500)
    st, w, expect = orc.sort_text(text, 16, "stable")
    want_bytes, want_off = orc.pack_words(expect.out_rec, w.len[expect.out_perm])
    cap_words = len(text) // 2 + 1
    s = bs.Sorter(cap_words, 16)
    s.sort_text(to_dev(np.frombuffer(text, np.uint8), torch), alg="merge")
    # n = the capacity; the offsets' word count off[W+1] bounds it on the device
    b, offsets = packed_on_gpu(env, s, cap_words, True)
    assert s.status() == 0
    n = w.n
    assert np.array_equal(u32(offsets[:n + 1]), want_off)
    assert np.array_equal(b[:int(want_off[-1])].cpu().numpy(), want_bytes)


def test_pack_rejects_a_small_buffer(env):
    torch, bs, orc = env
    W, n = 16, 3000
    rec, ln = table(5, n, W)
    s = bs.Sorter(n, W)
    s.sort_records(to_dev(rec, torch), to_dev(ln, torch), n, alg="merge")
    total = int(ln.astype(np.int64).sum())
    b, offsets = packed_on_gpu(env, s, n, True, cap=total - 1)
    assert s.status() == bs._lib.E_CAPACITY
    assert int(u32(offsets)[n]) == 0
    assert not b.cpu().numpy().any()  # no byte written
