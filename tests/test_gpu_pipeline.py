"""GPU parity of HostPipeline: jobs whose copy-in, sort and copy-out overlap
across two streams give, job by job, the oracle's answer in their own pinned
host buffers."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import need_cuda, table
from paper_1411_5283_gb300 import synth

pytestmark = pytest.mark.gpu


def test_pipelined_jobs_match_oracle(orc):
    torch = need_cuda()
    from paper_1411_5283_gb300.pipeline import HostPipeline
    W = 16
    jobs = [synth.large_records(31, 200_000, W), table(32, 5_000, W), synth.large_records(33, 90_000, W),
            table(34, 1, W), synth.large_records(35, 150_000, W)]
    pipe = HostPipeline(200_000, W, depth=2)
    outs = []
    pipe.start_after()
    for rec, ln in jobs:
        n = ln.size
        o = (torch.empty((n, W), dtype=torch.uint8).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
             torch.empty(W + 2, dtype=torch.int32).pin_memory())
        pipe.submit(torch.from_numpy(rec).pin_memory(), torch.from_numpy(ln).pin_memory(), n, *o, alg="auto")
        outs.append(o)
    pipe.wait_all()
    torch.cuda.synchronize()
    assert pipe.status() == 0
    for (rec, ln), (o_rec, o_perm, o_off) in zip(jobs, outs):
        want = orc.stable_sort(orc.Words(rec, ln))
        assert np.array_equal(o_off.numpy().view(np.uint32), want.off)
        assert np.array_equal(o_perm.numpy().view(np.uint32), want.out_perm)
        assert np.array_equal(o_rec.numpy(), want.out_rec)


def test_pipelined_packed_jobs_match_oracle(orc):
    """The same pipeline with answers read back as packed bytes, offsets and
    the permutation: each job equals the oracle's answer packed by the
    oracle."""
    torch = need_cuda()
    from paper_1411_5283_gb300.pipeline import HostPipeline
    W = 32
    jobs = [synth.large_records(51, 120_000, W), table(52, 3_000, W), synth.large_records(53, 70_000, W)]
    pipe = HostPipeline(120_000, W, depth=2)
    outs = []
    pipe.start_after()
    for rec, ln in jobs:
        n, total = ln.size, int(ln.astype(np.int64).sum())
        o = (torch.empty(total, dtype=torch.uint8).pin_memory(), torch.empty(n + 1, dtype=torch.int32).pin_memory(),
             torch.empty(n, dtype=torch.int32).pin_memory())
        pipe.submit_packed(torch.from_numpy(rec).pin_memory(), torch.from_numpy(ln).pin_memory(), n, total, *o)
        outs.append(o)
    pipe.wait_all()
    torch.cuda.synchronize()
    assert pipe.status() == 0
    for (rec, ln), (o_bytes, o_off, o_perm) in zip(jobs, outs):
        want = orc.stable_sort(orc.Words(rec, ln))
        want_bytes, want_off = orc.pack_words(want.out_rec, ln[want.out_perm])
        assert np.array_equal(o_perm.numpy().view(np.uint32), want.out_perm)
        assert np.array_equal(o_off.numpy().view(np.uint32), want_off)
        assert np.array_equal(o_bytes.numpy(), want_bytes)
