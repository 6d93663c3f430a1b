"""Sorting a stream of host-resident word tables with copies and sorts overlapped.

Each job is a word table in pinned host memory whose answer must come back to
pinned host memory.  A job's own copy-in, sort and copy-out cannot overlap:
the sort needs the whole table before it starts, and the answer exists only
once it ends.  Consecutive jobs can: :class:`HostPipeline` keeps ``depth``
slots, each with its own stream, device input buffers and :class:`Sorter`
(workspace and outputs), and issues job k on slot k mod depth.  On the GPU
the host-to-device copy of job k+1, the sort of job k and the device-to-host
copy of job k-1 then run at the same time (two copy directions and the SMs),
so the steady-state time per job is the largest of the three instead of their
sum.  Jobs on one slot stay in order on its stream, so a slot's buffers are
never overwritten while still in use.

Argument marshalling and stream bookkeeping only: every step of the sort runs
in the library's kernels through :meth:`Sorter.sort_records`.
"""
from __future__ import annotations

from . import Sorter


class HostPipeline:
    """``depth`` slots for tables of up to ``max_words`` words of width ``W``."""

    def __init__(self, max_words: int, W: int, depth: int = 2, device: str = "cuda"):
        import torch
        self.torch = torch
        self.W, self.max_words, self.depth = W, max_words, depth
        self.slots = []
        for _ in range(depth):
            self.slots.append({
                "stream": torch.cuda.Stream(device=device),
                "sorter": Sorter(max_words, W, device=device),
                "rec": torch.empty((max(max_words, 1), W), dtype=torch.uint8, device=device),
                "len": torch.empty(max(max_words, 1), dtype=torch.uint8, device=device),
                "done": None,
            })
        self.k = 0

    def submit(self, rec_h, len_h, n: int, out_rec_h, out_perm_h, off_h, alg="auto", tune=None):
        """Queues one job: copy the pinned host table in, sort it, copy the
        answer (records, permutation, offsets) to the pinned host buffers.
        Returns the CUDA event that marks the job's completion."""
        torch = self.torch
        s = self.slots[self.k % self.depth]
        self.k += 1
        with torch.cuda.stream(s["stream"]):
            s["rec"][:n].copy_(rec_h[:n], non_blocking=True)
            s["len"][:n].copy_(len_h[:n], non_blocking=True)
            out_rec, out_perm, off = s["sorter"].sort_records(s["rec"], s["len"], n, alg=alg, tune=tune)
            out_rec_h[:n].copy_(out_rec, non_blocking=True)
            out_perm_h[:n].copy_(out_perm, non_blocking=True)
            off_h.copy_(off, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s["stream"])
        s["done"] = ev
        return ev

    def submit_packed(self, rec_h, len_h, n: int, total_bytes: int, bytes_h, offsets_h, out_perm_h,
                      alg="auto", tune=None):
        """As submit, but the answer comes back in the paper's "vectors of
        string" form (§3.1): the sorted words packed without padding
        (total_bytes = the sum of the input lengths, known to the caller) plus
        offsets[n + 1], and the permutation."""
        torch = self.torch
        s = self.slots[self.k % self.depth]
        self.k += 1
        if "bytes" not in s:
            s["bytes"] = torch.empty(max(self.max_words * self.W, 16), dtype=torch.uint8,
                                     device=s["rec"].device)
            s["offsets"] = torch.empty(self.max_words + 1, dtype=torch.int32,
                                       device=s["rec"].device)
        with torch.cuda.stream(s["stream"]):
            s["rec"][:n].copy_(rec_h[:n], non_blocking=True)
            s["len"][:n].copy_(len_h[:n], non_blocking=True)
            b, offsets, out_perm, _ = s["sorter"].sort_records_packed(
                s["rec"], s["len"], n, alg=alg, tune=tune, out_bytes=s["bytes"],
                offsets=s["offsets"][:n + 1])
            bytes_h[:total_bytes].copy_(b[:total_bytes], non_blocking=True)
            offsets_h[:n + 1].copy_(offsets, non_blocking=True)
            out_perm_h[:n].copy_(out_perm, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s["stream"])
        s["done"] = ev
        return ev

    def wait_all(self, stream=None):
        """Makes `stream` (default: the current stream) wait for every queued job."""
        torch = self.torch
        st = stream or torch.cuda.current_stream()
        for s in self.slots:
            st.wait_stream(s["stream"])

    def start_after(self, stream=None):
        """Makes every slot's stream wait for the work queued so far on `stream`."""
        torch = self.torch
        st = stream or torch.cuda.current_stream()
        for s in self.slots:
            s["stream"].wait_stream(st)

    def status(self) -> int:
        """The largest device-detected status over the slots (syncs)."""
        return max(s["sorter"].status() for s in self.slots)
