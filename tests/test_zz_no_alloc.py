"""bsort_sort_records_noalloc: the workspace-free entry point for callers that
may not allocate device memory (their memory belongs to a host framework's
pool, or cudaMalloc's possible device synchronisation is not acceptable).

It must give exactly the answer of bsort_sort_records, call after call, even
though every call reuses the same static scratch array.  Collected last on
purpose (file name) so that a failure here never hides another test.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda, table, to_dev

pytestmark = pytest.mark.gpu

MAX_WORDS = 32768


def reference_answer(bs, torch, rec, ln, W, alg):
    s = bs.Sorter(ln.size, W)
    out_rec, out_perm, off = s.sort_records(to_dev(rec, torch), to_dev(ln, torch), ln.size,
                                            alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    return out_rec.cpu().numpy(), out_perm.cpu().numpy(), off.cpu().numpy()


def noalloc_answer(bs, torch, rec, ln, W, alg):
    n = ln.size
    out_rec = torch.empty((max(n, 1), W), dtype=torch.uint8, device="cuda")
    out_perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.empty(W + 2, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    bs._lib.bsort_sort_records_noalloc(to_dev(rec, torch), to_dev(ln, torch), n, W, alg, None,
                                       out_rec, out_perm, off, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return out_rec[:n].cpu().numpy(), out_perm[:n].cpu().numpy(), off.cpu().numpy()


@pytest.mark.parametrize("W,alg", [(16, "merge"), (32, "auto"), (8, "odd_even")])
def test_noalloc_matches_workspace_path_twice(W, alg):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    # two different inputs, one call each, back to back on the same scratch
    cases = [table(100 + W, MAX_WORDS, W), table(200 + W, 5000, W, b"abc", 5)]
    for rec, ln in cases:
        want = reference_answer(bs, torch, rec, ln, W, alg)
        got = noalloc_answer(bs, torch, rec, ln, W, alg)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)


def test_noalloc_rejects_too_many_words():
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    bs._lib.load()
    n = MAX_WORDS + 1
    rec, ln = table(7, n, 16)
    out_rec = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
    out_perm = torch.empty(n, dtype=torch.int32, device="cuda")
    off = torch.empty(18, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BsortError) as e:
        bs._lib.bsort_sort_records_noalloc(to_dev(rec, torch), to_dev(ln, torch), n, 16, "merge",
                                           None, out_rec, out_perm, off)
    assert e.value.status == bs._lib.E_CAPACITY
