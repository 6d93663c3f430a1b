"""GPU tests of the continuous-batching server: every response equals the
oracle and the same request served alone, bit for bit; requests that do not
fit wait for memory; too-large requests are rejected; cancelled requests never
run; a malformed request fails alone."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu
W = 16


@pytest.fixture(scope="module")
def env(orc):
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import serve
    bs._lib.load()
    return torch, serve, orc


def make_requests(serve, n, seed=0, rate=2000.0, text_frac=0.25):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    for i in range(n):
        size = int(np.exp(rng.uniform(np.log(64), np.log(20_000))))
        if rng.random() < text_frac:
            reqs.append(serve.Request(i, arrival=float(t[i]),
                                      text=synth.prose(1000 + i, max(1, size // 4), 4500)))
        else:
            rec, ln = synth.list_words(1000 + i, size, 50_000, W)
            reqs.append(serve.Request(i, arrival=float(t[i]), rec=rec, ln=ln))
    return reqs


def expected(orc, r):
    if r.is_text:
        st, w, res = orc.sort_text(r.text, W, "stable")
        return st, res
    res = orc.stable_sort(orc.Words(r.rec, r.ln))
    return res.status, res


def test_served_results_match_oracle_and_alone(env):
    torch, serve, orc = env
    reqs = make_requests(serve, 40)
    srv = serve.Server(W, 256 << 20, max_list_words=1 << 16)
    stats = srv.run_trace(reqs, release=False)
    assert stats["completed"] == 40 and stats["rejected"] == 0
    for r in reqs:
        st, res = expected(orc, r)
        assert st == 0
        got = srv.result(r)
        assert got[0] == 0
        assert np.array_equal(got[3], res.off)
        assert np.array_equal(got[2], res.out_perm)
        assert np.array_equal(got[1], res.out_rec)
    # the same request served on its own gives the same bytes
    for r in reqs[::9]:
        solo = serve.Server(W, 64 << 20, max_list_words=1 << 16)
        r2 = serve.Request(r.rid, rec=r.rec, ln=r.ln, text=r.text)
        solo.run_trace([r2], release=False)
        a, b = solo.result(r2), srv.result(r)
        assert a[0] == b[0] == 0
        for x, y in zip(a[1:], b[1:]):
            assert np.array_equal(x, y)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_admission_waits_for_memory_and_rejects_oversize(env):
    torch, serve, orc = env
    srv = serve.Server(W, 4 << 20, max_list_words=1 << 16, max_batch_lists=64)
    big = srv.n_slots + 1
    reqs = make_requests(serve, 12, seed=3, text_frac=0.0)
    rec, ln = synth.list_words(7, big, 50_000, W)
    reqs.append(serve.Request(99, arrival=0.0, rec=rec, ln=ln))
    stats = srv.run_trace(reqs, release=True)
    assert stats["rejected"] == 1 and srv.rejected[0].rid == 99
    assert srv.rejected[0].status == 7  # BSORT_E_NOMEM
    assert stats["completed"] == 12
    assert srv.slots.free_total == srv.n_slots  # every slot released


def test_cancel_and_malformed(env):
    torch, serve, orc = env
    srv = serve.Server(W, 64 << 20, max_list_words=1 << 16)
    rec, ln = synth.list_words(1, 500, 50_000, W)
    bad = ln.copy()
    bad[10] = W + 3
    a = serve.Request(0, rec=rec, ln=ln)
    b = serve.Request(1, rec=rec, ln=bad)
    c = serve.Request(2, rec=rec, ln=ln)
    for r in (a, b, c):
        srv.submit(r)
    assert srv.cancel(c)
    srv.drain(release=False)
    assert {r.rid for r in srv.done} == {0, 1}
    assert a.status == 0 and b.status == 2 and c.cancelled
    st, res = expected(orc, a)
    got = srv.result(a)
    assert np.array_equal(got[2], res.out_perm)


def test_two_batches_overlap_on_the_device(env):
    """Two large requests arriving together go to the two lanes as two
    batches; the CUDA events around each batch show the second starting on
    the device before the first has finished (inputs come from pinned host
    memory, so both launches are queued at once)."""
    torch, serve, orc = env
    srv = serve.Server(W, 1 << 30, max_list_words=1 << 20, max_batch_lists=1)
    reqs, want = [], []
    for i in range(2):
        rec, ln = synth.list_words(3000 + i, 1_000_000, 50_000, W)
        want.append(orc.stable_sort(orc.Words(rec, ln)))
        reqs.append(serve.Request(i, arrival=0.0, rec=torch.from_numpy(rec).pin_memory(),
                                  ln=torch.from_numpy(ln).pin_memory()))
    ref = torch.cuda.Event(enable_timing=True)
    ref.record()
    torch.cuda.synchronize()
    stats = srv.run_trace(reqs, release=False)
    assert stats["completed"] == 2 and stats["batches"] == 2
    a, b = reqs
    assert a.ev_start is not b.ev_start
    a0, a1 = ref.elapsed_time(a.ev_start), ref.elapsed_time(a.ev_end)
    b0, b1 = ref.elapsed_time(b.ev_start), ref.elapsed_time(b.ev_end)
    assert min(a1, b1) > max(a0, b0), f"batches did not overlap: {(a0, a1)} vs {(b0, b1)}"
    for r, res in zip(reqs, want):
        got = srv.result(r)
        assert got[0] == 0
        assert np.array_equal(got[2], res.out_perm)
        assert np.array_equal(got[1], res.out_rec)
