"""Helpers for the GPU parity tests: device copies and oracle comparison."""
from __future__ import annotations

import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(a: np.ndarray, torch, dtype=None):
    a = np.ascontiguousarray(a)
    if not a.flags.writeable:
        a = a.copy()
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.view(dtype)
    return t.cuda()


def u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def assert_same_answer(out_rec, out_perm, off, expect, n):
    """Bit-exact comparison of the library's answer with the oracle's."""
    got_rec = out_rec[:n].cpu().numpy()
    got_perm = u32(out_perm[:n])
    got_off = u32(off)
    assert np.array_equal(got_off, expect.off), f"off differs: {got_off} vs {expect.off}"
    if not np.array_equal(got_perm, expect.out_perm):
        bad = np.flatnonzero(got_perm != expect.out_perm)
        raise AssertionError(f"perm differs at {bad.size} ranks, first {bad[:8]}: "
                             f"{got_perm[bad[:8]]} vs {expect.out_perm[bad[:8]]}")
    assert np.array_equal(got_rec, expect.out_rec), "records differ"


def table(seed, n, W, alphabet=b"abcdefghijklmnopqrstuvwxyz", max_len=None, min_len=1):
    rng = np.random.default_rng(seed)
    max_len = W if max_len is None else max_len
    ln = rng.integers(min_len, max_len + 1, size=n).astype(np.uint8)
    a = np.frombuffer(alphabet, np.uint8)
    rec = a[rng.integers(0, a.size, size=(n, W))]
    rec[np.arange(W)[None, :] >= ln[:, None]] = 0
    return np.ascontiguousarray(rec), ln
