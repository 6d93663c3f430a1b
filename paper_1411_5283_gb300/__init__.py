"""GB300-native length-bucketed word sort (arXiv 1411.5283, §3 Methodology).

The compute path is the CUDA library ``libbsort.so`` (C ABI in
``include/bsort.h``); this package binds it with ctypes (``_lib``) and adds
:class:`Sorter`, which owns a workspace and output buffers as torch tensors.
PyTorch provides device memory and streams only.
"""
from __future__ import annotations

from . import _lib
from ._lib import (ALGS, AUTO, MERGE, ODD_EVEN, BsortError, ListDesc, Tune,  # noqa: F401
                   bsort_bucket_by_length, bsort_export_buckets, bsort_gather,
                   bsort_get_status, bsort_pack_words, bsort_profile_enable, bsort_profile_read,
                   bsort_profile_reset, bsort_reset_status, bsort_sort_buckets, bsort_sort_many,
                   bsort_sort_many_workspace_size, bsort_sort_records, bsort_sort_records_packed,
                   bsort_sort_records_whole, bsort_sort_text, bsort_sort_text_packed,
                   bsort_sort_text_whole,
                   bsort_status_string, bsort_tokenize, bsort_workspace_capacity, bsort_workspace_init,
                   bsort_workspace_size)


class Sorter:
    """A workspace for up to ``max_words`` words of width ``W`` plus output buffers.

    Methods run the library's calls on the current CUDA stream and return
    torch tensors (uint8 records, int32 permutation / offsets holding uint32
    values)."""

    def __init__(self, max_words: int, W: int, device: str = "cuda"):
        import torch
        self.torch = torch
        self.W = W
        self.max_words = max_words
        self.device = device
        self.ws_bytes = bsort_workspace_size(max_words, W)
        if self.ws_bytes == 0:
            raise BsortError(_lib.E_INVALID, "bsort_workspace_size")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        bsort_workspace_init(self.ws, self.ws_bytes)
        self.off = torch.zeros(W + 2, dtype=torch.int32, device=device)
        self.out_rec = torch.empty((max(max_words, 1), W), dtype=torch.uint8, device=device)
        self.out_perm = torch.empty(max(max_words, 1), dtype=torch.int32, device=device)
        self.rec = None

    def status(self) -> int:
        return bsort_get_status(self.ws)

    def reset(self):
        bsort_reset_status(self.ws)

    # -- phase by phase -----------------------------------------------------
    def tokenize(self, text, max_words: int | None = None):
        """Phase 1 on a uint8 CUDA tensor; returns (rec, len, src_off, n_words device tensor)."""
        torch = self.torch
        mw = self.max_words if max_words is None else max_words
        rec = torch.empty((max(mw, 1), self.W), dtype=torch.uint8, device=self.device)
        ln = torch.empty(max(mw, 1), dtype=torch.uint8, device=self.device)
        so = torch.empty(max(mw, 1), dtype=torch.int32, device=self.device)
        nw = torch.zeros(1, dtype=torch.int32, device=self.device)
        bsort_tokenize(text, text.numel(), self.W, mw, rec, ln, so, nw, self.ws, self.ws_bytes)
        return rec, ln, so, nw

    def bucket_by_length(self, rec, ln, n: int):
        bsort_bucket_by_length(rec, ln, n, self.W, self.off, self.ws, self.ws_bytes)
        return self.off

    def sort_buckets(self, n: int, alg="auto", tune=None):
        bsort_sort_buckets(n, self.W, alg, tune, self.off, self.ws, self.ws_bytes)

    def gather(self, n: int):
        bsort_gather(n, self.W, self.off, self.ws, self.ws_bytes, self.out_rec, self.out_perm)
        return self.out_rec[:n], self.out_perm[:n], self.off

    def export_buckets(self, n: int):
        torch = self.torch
        keys = torch.empty((self.W // 8, max(n, 1)), dtype=torch.int64, device=self.device)
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        bsort_export_buckets(n, self.W, self.off, self.ws, self.ws_bytes, keys, idx)
        return keys[:, :n], idx[:n]

    # -- whole path ------------------------------------------------------------
    def sort_records(self, rec, ln, n: int | None = None, alg="auto", tune=None):
        """Phases 2-3 + concatenation on a word table; returns (out_rec, out_perm, off)."""
        n = int(ln.numel()) if n is None else n
        bsort_sort_records(rec, ln, n, self.W, alg, tune, self.out_rec, self.out_perm, self.off,
                           self.ws, self.ws_bytes)
        return self.out_rec[:n], self.out_perm[:n], self.off

    def sort_records_whole(self, rec, ln, n: int | None = None, alg="auto", tune=None):
        """The unbucketed order (bytes, a proper prefix first, then input
        index) on a word table; returns (out_rec, out_perm)."""
        n = int(ln.numel()) if n is None else n
        bsort_sort_records_whole(rec, ln, n, self.W, alg, tune, self.out_rec, self.out_perm,
                                 self.ws, self.ws_bytes)
        return self.out_rec[:n], self.out_perm[:n]

    def sort_text_whole(self, text, alg="auto", tune=None, max_words: int | None = None):
        """Phase 1, then the unbucketed order; returns (out_rec, out_perm,
        n_words device tensor, rec, len, src_off)."""
        self._text_buffers(self.max_words if max_words is None else max_words)
        mw = self.max_words if max_words is None else max_words
        bsort_sort_text_whole(text, text.numel(), self.W, mw, alg, tune, self.rec, self.len,
                              self.src_off, self.n_words, self.out_rec, self.out_perm, self.ws,
                              self.ws_bytes)
        return self.out_rec, self.out_perm, self.n_words, self.rec, self.len, self.src_off

    def pack(self, n: int, bucketed: bool = True, perm=None, ln=None, out_bytes=None):
        """The sorted words in self.out_rec packed without padding (§3.1):
        returns (bytes, offsets[n + 1]) as device tensors; lengths from the
        bucket offsets (bucketed order) or from ln[perm] (any order)."""
        torch = self.torch
        cap = n * self.W
        if out_bytes is None:
            out_bytes = torch.empty(max(cap, 16), dtype=torch.uint8, device=self.device)
        offsets = torch.empty(n + 1, dtype=torch.int32, device=self.device)
        bsort_pack_words(n, self.W, self.out_rec, self.off if bucketed else None,
                         None if bucketed else perm, None if bucketed else ln, out_bytes,
                         int(out_bytes.numel()), offsets, self.ws, self.ws_bytes)
        return out_bytes, offsets

    def sort_records_packed(self, rec, ln, n: int | None = None, alg="auto", tune=None,
                            out_bytes=None, offsets=None):
        """Phases 2-3 with the answer packed without padding (§3.1) by the
        sort's last kernel; returns (bytes, offsets[n + 1], out_perm, off).
        The default byte buffer holds n W bytes."""
        torch = self.torch
        n = int(ln.numel()) if n is None else n
        if out_bytes is None:
            out_bytes = torch.empty(max(n * self.W, 16), dtype=torch.uint8, device=self.device)
        if offsets is None:
            offsets = torch.empty(n + 1, dtype=torch.int32, device=self.device)
        bsort_sort_records_packed(rec, ln, n, self.W, alg, tune, out_bytes, int(out_bytes.numel()),
                                  offsets, self.out_perm, self.off, self.ws, self.ws_bytes)
        return out_bytes, offsets, self.out_perm[:n], self.off

    def sort_text_packed(self, text, alg="auto", tune=None, max_words: int | None = None,
                         out_bytes=None, offsets=None):
        """Phases 1-3 on raw text with the packed answer; returns (bytes,
        offsets, out_perm, off, n_words device tensor).  offsets[n_words] is
        the total; entries past it are unspecified."""
        torch = self.torch
        mw = self.max_words if max_words is None else max_words
        self._text_buffers(mw)
        if out_bytes is None:
            out_bytes = torch.empty(max(mw * self.W, 16), dtype=torch.uint8, device=self.device)
        if offsets is None:
            offsets = torch.empty(mw + 1, dtype=torch.int32, device=self.device)
        bsort_sort_text_packed(text, text.numel(), self.W, mw, alg, tune, self.rec, self.len,
                               self.src_off, self.n_words, out_bytes, int(out_bytes.numel()),
                               offsets, self.out_perm, self.off, self.ws, self.ws_bytes)
        return out_bytes, offsets, self.out_perm, self.off, self.n_words

    def _text_buffers(self, mw: int):
        torch = self.torch
        if self.rec is None or self.rec.shape[0] < max(mw, 1):
            self.rec = torch.empty((max(mw, 1), self.W), dtype=torch.uint8, device=self.device)
            self.len = torch.empty(max(mw, 1), dtype=torch.uint8, device=self.device)
            self.src_off = torch.empty(max(mw, 1), dtype=torch.int32, device=self.device)
            self.n_words = torch.zeros(1, dtype=torch.int32, device=self.device)

    def sort_text(self, text, alg="auto", tune=None, max_words: int | None = None):
        """Phases 1-3 on raw text; returns (out_rec, out_perm, off, n_words device tensor,
        rec, len, src_off).  Outputs past n_words are unspecified."""
        mw = self.max_words if max_words is None else max_words
        self._text_buffers(mw)
        bsort_sort_text(text, text.numel(), self.W, mw, alg, tune, self.rec, self.len,
                        self.src_off, self.n_words, self.out_rec, self.out_perm, self.off,
                        self.ws, self.ws_bytes)
        return (self.out_rec, self.out_perm, self.off, self.n_words, self.rec, self.len,
                self.src_off)
