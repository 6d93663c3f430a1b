"""bsort_sort_records_noalloc: the workspace-free entry point for callers that
may not allocate device memory (their memory belongs to a host framework's
pool, or cudaMalloc's possible device synchronisation is not acceptable).

It must give exactly the oracle's answer and the answer of
bsort_sort_records, call after call, even though every call reuses the same
static scratch array: a device error of one call (a word longer than W) is
reported in that call's status word and does not leak into the next call,
and an empty input is answered with empty buckets.  Collected last on purpose
(file name) so that a failure here never hides another test.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda, table, to_dev

pytestmark = pytest.mark.gpu

MAX_WORDS = 32768


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    return torch, bs, orc


def reference_answer(bs, torch, rec, ln, W, alg):
    s = bs.Sorter(ln.size, W)
    out_rec, out_perm, off = s.sort_records(to_dev(rec, torch), to_dev(ln, torch), ln.size,
                                            alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    return out_rec.cpu().numpy(), out_perm.cpu().numpy(), off.cpu().numpy()


def noalloc_call(bs, torch, rec, ln, W, alg):
    n = ln.size
    out_rec = torch.empty((max(n, 1), W), dtype=torch.uint8, device="cuda")
    out_perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.full((W + 2,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    bs._lib.bsort_sort_records_noalloc(to_dev(rec, torch) if n else None,
                                       to_dev(ln, torch) if n else None, n, W, alg, None,
                                       out_rec if n else None, out_perm if n else None, off,
                                       status)
    torch.cuda.synchronize()
    return (int(status.item()), out_rec[:n].cpu().numpy(), out_perm[:n].cpu().numpy(),
            off.cpu().numpy())


@pytest.mark.parametrize("W,alg", [(16, "merge"), (32, "auto"), (8, "odd_even")])
def test_noalloc_matches_oracle_and_workspace_path_twice(env, W, alg):
    torch, bs, orc = env
    # two different inputs, one call each, back to back on the same scratch
    cases = [table(100 + W, MAX_WORDS, W), table(200 + W, 5000, W, b"abc", 5)]
    for rec, ln in cases:
        expect = orc.stable_sort(orc.Words(rec, ln))
        want = reference_answer(bs, torch, rec, ln, W, alg)
        st, *got = noalloc_call(bs, torch, rec, ln, W, alg)
        assert st == 0
        assert np.array_equal(got[0], expect.out_rec)
        assert np.array_equal(got[1].view(np.uint32), expect.out_perm)
        assert np.array_equal(got[2].view(np.uint32), expect.off)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)


def test_noalloc_error_then_clean_call_then_empty(env):
    torch, bs, orc = env
    W = 16
    rec, ln = table(31, 4000, W)
    bad = ln.copy()
    bad[123] = W + 1  # one length above W
    st, *_ = noalloc_call(bs, torch, rec, bad, W, "merge")
    assert st == bs._lib.E_WORD_TOO_LONG
    # the next call on the same scratch starts from a clean status
    st, out_rec, out_perm, off = noalloc_call(bs, torch, rec, ln, W, "merge")
    assert st == 0
    expect = orc.bubble_sort(orc.Words(rec, ln))
    assert np.array_equal(out_rec, expect.out_rec)
    assert np.array_equal(out_perm.view(np.uint32), expect.out_perm)
    assert np.array_equal(off.view(np.uint32), expect.off)
    # no words: OK, every offset zero
    st, out_rec, out_perm, off = noalloc_call(bs, torch, rec[:0], ln[:0], W, "merge")
    assert st == 0 and out_perm.size == 0
    assert not off.any()


def test_noalloc_rejects_too_many_words(env):
    torch, bs, orc = env
    n = MAX_WORDS + 1
    rec, ln = table(7, n, 16)
    out_rec = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
    out_perm = torch.empty(n, dtype=torch.int32, device="cuda")
    off = torch.empty(18, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BsortError) as e:
        bs._lib.bsort_sort_records_noalloc(to_dev(rec, torch), to_dev(ln, torch), n, 16, "merge",
                                           None, out_rec, out_perm, off)
    assert e.value.status == bs._lib.E_CAPACITY
