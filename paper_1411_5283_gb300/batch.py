"""Batched sorting of many independent word lists (``bsort_sort_many``).

:class:`BatchSorter` owns a batch workspace and output buffers, packs list
descriptors (``bsort_list``), runs the batched call on the current stream and
can capture it once in a CUDA graph for cheap replays.  Argument marshalling
and buffer management only: every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import _lib

# bsort_list, 32 bytes: text_off, text_bytes, word_off (u64), n_words, max_words (u32)
LIST_DTYPE = np.dtype([("text_off", "<u8"), ("text_bytes", "<u8"), ("word_off", "<u8"),
                       ("n_words", "<u4"), ("max_words", "<u4")])
assert LIST_DTYPE.itemsize == 32


def record_lists(sizes, capacity=None) -> np.ndarray:
    """Descriptors for record-mode lists laid out back to back."""
    sizes = np.asarray(sizes, dtype=np.int64)
    cap = sizes if capacity is None else np.asarray(capacity, dtype=np.int64)
    d = np.zeros(sizes.size, dtype=LIST_DTYPE)
    d["word_off"] = np.concatenate([[0], np.cumsum(cap)[:-1]]) if sizes.size else []
    d["n_words"] = sizes
    d["max_words"] = cap
    return d


def text_lists(text_sizes, max_words) -> np.ndarray:
    """Descriptors for text-mode lists: texts back to back, output slots too."""
    ts = np.asarray(text_sizes, dtype=np.int64)
    mw = np.asarray(max_words, dtype=np.int64)
    d = np.zeros(ts.size, dtype=LIST_DTYPE)
    d["text_off"] = np.concatenate([[0], np.cumsum(ts)[:-1]]) if ts.size else []
    d["text_bytes"] = ts
    d["word_off"] = np.concatenate([[0], np.cumsum(mw)[:-1]]) if ts.size else []
    d["max_words"] = mw
    return d


class BatchSorter:
    """Workspace and outputs for batches of up to ``n_lists`` lists holding at
    most ``total_words`` word slots (sum of max_words) of width ``W``."""

    def __init__(self, total_words: int, n_lists: int, W: int, device: str = "cuda"):
        import torch
        self.torch = torch
        self.W, self.n_lists, self.total_words, self.device = W, n_lists, total_words, device
        self.ws_bytes = _lib.bsort_sort_many_workspace_size(total_words, n_lists, W)
        if self.ws_bytes == 0:
            raise _lib.BsortError(_lib.E_INVALID, "bsort_sort_many_workspace_size")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        n = max(total_words, 1)
        self.out_rec = torch.empty((n, W), dtype=torch.uint8, device=device)
        self.out_perm = torch.empty(n, dtype=torch.int32, device=device)
        self.out_off = torch.zeros((max(n_lists, 1), W + 2), dtype=torch.int32, device=device)
        self.status = torch.zeros(max(n_lists, 1), dtype=torch.int32, device=device)
        self.lists = torch.zeros((max(n_lists, 1), LIST_DTYPE.itemsize), dtype=torch.uint8,
                                 device=device)
        self.graph = None

    def set_lists(self, desc: np.ndarray, stream=None):
        assert desc.dtype == LIST_DTYPE and desc.size <= self.n_lists
        host = self.torch.from_numpy(desc.view(np.uint8).reshape(-1, LIST_DTYPE.itemsize).copy())
        self.lists[:desc.size].copy_(host, non_blocking=False)
        self.n_active = int(desc.size)

    def run(self, data, ln, *, text: bool, max_list_words: int, alg="merge", tune=None,
            n_lists: int | None = None, stream=None):
        """One batched sort of the lists set by :meth:`set_lists`."""
        n = self.n_active if n_lists is None else n_lists
        _lib.bsort_sort_many(data, None if text else ln, self.lists, n, self.W, text,
                             max_list_words, alg, tune, self.out_rec, self.out_perm, self.out_off,
                             self.status, self.ws, self.ws_bytes, stream)

    def capture(self, data, ln, *, text: bool, max_list_words: int, alg="merge", tune=None):
        """Captures one batched sort into a CUDA graph (inputs and descriptors
        are read from the same device buffers at every replay)."""
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(data, ln, text=text, max_list_words=max_list_words, alg=alg, tune=tune)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(data, ln, text=text, max_list_words=max_list_words, alg=alg, tune=tune,
                     stream=s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def result(self, i: int, desc: np.ndarray):
        """(status, out_rec, out_perm, off) of list i as numpy arrays (syncs)."""
        st = int(self.status[i].item())
        off = self.out_off[i].cpu().numpy().view(np.uint32).copy()
        w0 = int(desc["word_off"][i])
        n = int(off[self.W + 1])
        rec = self.out_rec[w0:w0 + n].cpu().numpy()
        perm = self.out_perm[w0:w0 + n].cpu().numpy().view(np.uint32).copy()
        return st, rec, perm, off
