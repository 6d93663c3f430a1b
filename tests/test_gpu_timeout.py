"""The timeout path of the kernels' bounded waits, made to run out on
purpose without faulting anything.

Every kernel that stages data with the bulk-copy engine waits for the copy
on an mbarrier for a bounded number of polls.  With the bound set to zero
polls, each first wait gives up at once: the kernel records BSORT_E_TIMEOUT,
lets its copy land (that drain keeps the default bound) and returns.  The
call must then report BSORT_E_TIMEOUT, the context must stay usable, and the
next call with the default bound must give the oracle's answer again.
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
    yield torch, bs, orc
    bs._lib.bsort_set_wait_limit(bs._lib.WAIT_DEFAULT)


# odd-even and bitonic tiles (tile sort kernel), and the segment sort of the
# sample-sort path (n >= 65,536)
@pytest.mark.parametrize("alg,n", [("odd_even", 20_000), ("merge", 20_000), ("auto", 100_000)])
def test_wait_runs_out_then_next_call_is_exact(env, alg, n):
    torch, bs, orc = env
    rec, ln = synth.large_records(41, n, 16)
    expect = orc.stable_sort(orc.Words(rec, ln))
    s = bs.Sorter(n, 16)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    bs._lib.bsort_set_wait_limit(0)
    try:
        s.sort_records(d_rec, d_len, n, alg=alg)
        torch.cuda.synchronize()
        assert s.status() == bs._lib.E_TIMEOUT
    finally:
        bs._lib.bsort_set_wait_limit(bs._lib.WAIT_DEFAULT)
    out_rec, out_perm, off = s.sort_records(d_rec, d_len, n, alg=alg)
    torch.cuda.synchronize()
    assert s.status() == 0
    assert_same_answer(out_rec, out_perm, off, expect, n)


def test_batched_wait_runs_out_per_list(env):
    torch, bs, orc = env
    from paper_1411_5283_gb300 import batch
    W = 16
    sizes = [5000, 3000]
    lists = [synth.list_words(70 + i, m, 50_000, W) for i, m in enumerate(sizes)]
    rec = np.concatenate([r for r, _ in lists])
    ln = np.concatenate([l for _, l in lists])
    desc = batch.record_lists(sizes)
    b = batch.BatchSorter(int(ln.size), len(sizes), W)
    b.set_lists(desc)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    bs._lib.bsort_set_wait_limit(0)
    try:
        b.run(d_rec, d_len, text=False, max_list_words=8192)
        torch.cuda.synchronize()
    finally:
        bs._lib.bsort_set_wait_limit(bs._lib.WAIT_DEFAULT)
    timed_out = b.status[:2].cpu().numpy()
    b.run(d_rec, d_len, text=False, max_list_words=8192)
    torch.cuda.synchronize()
    for i, (r, l) in enumerate(lists):
        st, out_rec, perm, off = b.result(i, desc)
        assert st == 0
        expect = orc.stable_sort(orc.Words(r, l))
        assert np.array_equal(perm, expect.out_perm) and np.array_equal(out_rec, expect.out_rec)
    # the batch's wait flag reaches every list's status word
    assert timed_out.tolist() == [bs._lib.E_TIMEOUT] * 2
