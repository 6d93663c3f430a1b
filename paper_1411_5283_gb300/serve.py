"""Continuous-batching request loop over ``bsort_sort_many``.

Requests (a word table or a raw text) arrive over time.  The server

* admits a request when its buffers fit the free part of a fixed device budget
  (word slots for records and results, bytes for texts); a request that can
  never fit is rejected with ``BSORT_E_NOMEM``;
* keeps every admitted request's buffers resident in device arenas (a word-slot
  arena: input records, lengths, output records, permutation; a text arena);
* launches the admitted, not yet launched requests as one batch (one
  ``bsort_sort_many`` call per mode) on a free stream as soon as one is free,
  while earlier batches are still running on the other streams (work overlaps
  on the device), then frees their memory when their batch completes;
* records arrival, admission, launch and completion times for p50 / p99
  latency and throughput.

Host-side bookkeeping only; every step of the sort runs in the library's kernels.
"""
from __future__ import annotations

import bisect
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from .batch import LIST_DTYPE


@dataclass
class Request:
    """One sort request: a word table (rec [n, W], len [n]) or a raw text."""
    rid: int
    arrival: float = 0.0                     # seconds after the loop started
    rec: object = None                       # numpy array, or a (pinned) CPU tensor
    ln: object = None
    text: object = None                      # bytes, or a (pinned) uint8 CPU tensor
    max_words: int | None = None             # text mode: word slots to reserve
    # filled by the server
    status: int = -1
    t_admit: float = math.nan
    t_launch: float = math.nan
    t_done: float = math.nan
    slot: int = -1
    slots: int = 0
    text_off: int = -1
    off: np.ndarray | None = None
    cancelled: bool = False
    ev_start: object = None                  # CUDA events around the request's batch
    ev_end: object = None

    @property
    def is_text(self) -> bool:
        return self.text is not None

    @property
    def n_slots(self) -> int:
        if self.is_text:
            return self.max_words if self.max_words is not None else len(self.text) // 2 + 1
        return int(self.ln.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class RangeAllocator:
    """First-fit allocator of contiguous ranges in [0, size)."""

    def __init__(self, size: int, align: int = 1):
        self.size, self.align = size, align
        self.free = [(0, size)]  # sorted (start, length)

    def alloc(self, n: int) -> int:
        n = max(self.align, (n + self.align - 1) // self.align * self.align)
        for k, (s, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (s + n, l - n)
                return s
        return -1

    def release(self, start: int, n: int):
        n = max(self.align, (n + self.align - 1) // self.align * self.align)
        k = bisect.bisect_left(self.free, (start, 0))
        self.free.insert(k, (start, n))
        # coalesce with neighbours
        if k + 1 < len(self.free) and self.free[k][0] + self.free[k][1] == self.free[k + 1][0]:
            self.free[k] = (self.free[k][0], self.free[k][1] + self.free[k + 1][1])
            self.free.pop(k + 1)
        if k > 0 and self.free[k - 1][0] + self.free[k - 1][1] == self.free[k][0]:
            self.free[k - 1] = (self.free[k - 1][0], self.free[k - 1][1] + self.free[k][1])
            self.free.pop(k)

    @property
    def free_total(self) -> int:
        return sum(l for _, l in self.free)


class Admission:
    """Admission by free device memory (host bookkeeping only, no GPU).

    Requests wait first in, first out until their word slots (and text bytes)
    fit the free part of the arenas; a request larger than an arena, or than
    the batched call's per-list limit, is rejected with ``BSORT_E_NOMEM``."""

    def __init__(self, n_slots: int, text_bytes: int, max_list_words: int):
        self.n_slots, self.max_list_words = n_slots, max_list_words
        self.slots = RangeAllocator(n_slots, align=16)
        self.texts = RangeAllocator(max(text_bytes, 16), align=16)
        self.waiting: deque[Request] = deque()
        self.admitted: list[Request] = []
        self.rejected: list[Request] = []

    def _reject(self, req: Request, now: float):
        req.status = _lib.E_NOMEM
        req.t_done = now
        self.rejected.append(req)

    def submit(self, req: Request, now: float):
        """Queues a request (it is admitted as soon as memory allows)."""
        if req.n_slots > self.n_slots or (req.is_text and len(req.text) > self.texts.size) \
                or req.n_slots > self.max_list_words:
            self._reject(req, now)
            return
        self.waiting.append(req)

    def cancel(self, req: Request) -> bool:
        """Cancels a request not yet launched; returns whether it was."""
        if req in self.waiting:
            self.waiting.remove(req)
        elif req in self.admitted:
            self.admitted.remove(req)
            self.release(req)
        else:
            return False
        req.cancelled = True
        return True

    def admit(self, now: float):
        while self.waiting:
            req = self.waiting[0]
            slot = self.slots.alloc(req.n_slots)
            if slot < 0:
                return  # first in, first out: wait for memory
            toff = -1
            if req.is_text:
                toff = self.texts.alloc(max(1, len(req.text)))
                if toff < 0:
                    self.slots.release(slot, req.n_slots)
                    return
            self.waiting.popleft()
            req.slot, req.slots, req.text_off = slot, req.n_slots, toff
            req.t_admit = now
            self.admitted.append(req)

    def unblock(self, in_flight: bool, now: float):
        """With nothing admitted and nothing in flight, the head request waits
        for memory that only completed requests still hold (their results are
        kept): nothing will ever free it.  It is rejected with
        ``BSORT_E_NOMEM`` instead of waiting forever, and admission goes on
        with the next request."""
        while self.waiting and not self.admitted and not in_flight:
            self._reject(self.waiting.popleft(), now)
            self.admit(now)

    def release(self, req: Request):
        if req.slot >= 0:
            self.slots.release(req.slot, req.slots)
            req.slot = -1
        if req.text_off >= 0:
            self.texts.release(req.text_off, max(1, len(req.text)))
            req.text_off = -1


@dataclass
class _Lane:
    """Per-stream resources: one batch in flight at a time."""
    stream: object
    ws: object
    ws_bytes: int
    desc_dev: object
    desc_host: object
    status_dev: object
    status_host: object
    off_dev: object
    off_host: object
    event: object = None
    batch: list = field(default_factory=list)


class Server:
    """A continuous-batching sort server on one GPU.

    budget_bytes bounds all device memory the server allocates (arenas and
    per-stream workspaces); text_frac of it holds request texts."""

    def __init__(self, W: int, budget_bytes: int, *, n_streams: int = 2,
                 max_batch_lists: int = 1024, max_list_words: int = 1 << 20,
                 text_frac: float = 0.15, alg="merge", tune=None, device: str = "cuda"):
        import torch
        self.torch = torch
        self.W, self.alg, self.tune = W, alg, tune
        self.max_batch_lists, self.max_list_words = max_batch_lists, max_list_words
        text_bytes = int(budget_bytes * text_frac) // 16 * 16
        rest = budget_bytes - text_bytes
        per_slot = 2 * W + 5  # input record + length, output record + permutation

        def total(slots):
            ws = _lib.bsort_sort_many_workspace_size(slots, max_batch_lists, W)
            return per_slot * slots + n_streams * ws

        lo, hi = 0, rest // per_slot
        while lo < hi:  # largest slot count whose arenas and workspaces fit
            mid = (lo + hi + 1) // 2
            if total(mid) <= rest:
                lo = mid
            else:
                hi = mid - 1
        self.n_slots = lo // 64 * 64
        if self.n_slots == 0:
            raise _lib.BsortError(_lib.E_NOMEM, "Server budget")
        S = self.n_slots
        self.in_rec = torch.empty((S, W), dtype=torch.uint8, device=device)
        self.in_len = torch.empty(S, dtype=torch.uint8, device=device)
        self.out_rec = torch.empty((S, W), dtype=torch.uint8, device=device)
        self.out_perm = torch.empty(S, dtype=torch.int32, device=device)
        self.text = torch.empty(max(text_bytes, 16), dtype=torch.uint8, device=device)
        self.adm = Admission(S, text_bytes, max_list_words)
        self.slots, self.texts = self.adm.slots, self.adm.texts
        self.lanes = []
        for _ in range(n_streams):
            ws_bytes = _lib.bsort_sort_many_workspace_size(S, max_batch_lists, W)
            self.lanes.append(_Lane(
                stream=torch.cuda.Stream(),
                ws=torch.empty(ws_bytes, dtype=torch.uint8, device=device), ws_bytes=ws_bytes,
                desc_dev=torch.empty((max_batch_lists, LIST_DTYPE.itemsize), dtype=torch.uint8,
                                     device=device),
                desc_host=torch.empty((max_batch_lists, LIST_DTYPE.itemsize),
                                      dtype=torch.uint8).pin_memory(),
                status_dev=torch.empty(max_batch_lists, dtype=torch.int32, device=device),
                status_host=torch.empty(max_batch_lists, dtype=torch.int32).pin_memory(),
                off_dev=torch.empty((max_batch_lists, W + 2), dtype=torch.int32, device=device),
                off_host=torch.empty((max_batch_lists, W + 2), dtype=torch.int32).pin_memory()))
        self.waiting, self.admitted, self.rejected = (self.adm.waiting, self.adm.admitted,
                                                      self.adm.rejected)
        self.done: list[Request] = []
        self.batches = 0
        self.t0 = time.perf_counter()

    # -- time -------------------------------------------------------------------
    def now(self) -> float:
        return time.perf_counter() - self.t0

    # -- admission --------------------------------------------------------------
    def submit(self, req: Request):
        """Queues a request (it is admitted as soon as memory allows)."""
        self.adm.submit(req, self.now())

    def cancel(self, req: Request) -> bool:
        """Cancels a request not yet launched; returns whether it was."""
        return self.adm.cancel(req)

    def _admit(self):
        self.adm.admit(self.now())

    def _release(self, req: Request):
        self.adm.release(req)

    # -- batches ----------------------------------------------------------------
    def _launch(self, lane: _Lane):
        torch = self.torch
        batch = self.admitted[:self.max_batch_lists]
        del self.admitted[:len(batch)]
        if not batch:
            return
        lane.batch = batch
        t = self.now()
        with torch.cuda.stream(lane.stream):
            # inputs go to their resident slots on this stream, ahead of the sort
            for r in batch:
                r.t_launch = t
                if r.is_text:
                    if len(r.text):
                        # a pinned uint8 tensor is copied asynchronously; bytes are staged
                        src = r.text if torch.is_tensor(r.text) else \
                            torch.frombuffer(bytearray(r.text), dtype=torch.uint8)
                        self.text[r.text_off:r.text_off + len(r.text)].copy_(src, non_blocking=True)
                else:
                    # a pinned CPU tensor is copied asynchronously; a numpy
                    # array is staged by the driver first
                    rec = r.rec if torch.is_tensor(r.rec) else torch.from_numpy(r.rec)
                    ln = r.ln if torch.is_tensor(r.ln) else torch.from_numpy(r.ln)
                    self.in_rec[r.slot:r.slot + r.slots].copy_(rec, non_blocking=True)
                    self.in_len[r.slot:r.slot + r.slots].copy_(ln, non_blocking=True)
            start = torch.cuda.Event(enable_timing=True)
            start.record(lane.stream)
            # one call per mode; lists of a mode take consecutive descriptor rows
            order = [r for r in batch if not r.is_text] + [r for r in batch if r.is_text]
            desc = np.zeros(len(order), dtype=LIST_DTYPE)
            for k, r in enumerate(order):
                desc[k]["word_off"] = r.slot
                desc[k]["max_words"] = r.slots
                if r.is_text:
                    desc[k]["text_off"] = r.text_off
                    desc[k]["text_bytes"] = len(r.text)
                else:
                    desc[k]["n_words"] = r.slots
            lane.desc_host[:len(order)].copy_(torch.from_numpy(desc.view(np.uint8).reshape(
                -1, LIST_DTYPE.itemsize)))
            lane.desc_dev[:len(order)].copy_(lane.desc_host[:len(order)], non_blocking=True)
            n_rec = sum(1 for r in order if not r.is_text)
            n_txt = len(order) - n_rec
            sp = lane.stream.cuda_stream
            if n_rec:
                _lib.bsort_sort_many(self.in_rec, self.in_len, lane.desc_dev, n_rec, self.W, 0,
                                     self.max_list_words, self.alg, self.tune, self.out_rec,
                                     self.out_perm, lane.off_dev, lane.status_dev, lane.ws,
                                     lane.ws_bytes, sp)
            if n_txt:
                row = lane.desc_dev[n_rec:]
                _lib.bsort_sort_many(self.text, None, row, n_txt, self.W, 1,
                                     self.max_list_words, self.alg, self.tune, self.out_rec,
                                     self.out_perm, lane.off_dev[n_rec:],
                                     lane.status_dev[n_rec:], lane.ws, lane.ws_bytes, sp)
            lane.status_host[:len(order)].copy_(lane.status_dev[:len(order)], non_blocking=True)
            lane.off_host[:len(order)].copy_(lane.off_dev[:len(order)], non_blocking=True)
            lane.event = torch.cuda.Event(enable_timing=True)
            lane.event.record(lane.stream)
        for r in order:
            r.ev_start, r.ev_end = start, lane.event
        lane.batch = order
        self.batches += 1

    def _complete(self, lane: _Lane, release: bool):
        t = self.now()
        st = lane.status_host[:len(lane.batch)].numpy().copy()
        off = lane.off_host[:len(lane.batch)].numpy().view(np.uint32).copy()
        for k, r in enumerate(lane.batch):
            r.status = int(st[k])
            r.off = off[k]
            r.t_done = t
            if release:
                self._release(r)
            self.done.append(r)
        lane.batch = []
        lane.event = None

    def step(self, release: bool = True) -> bool:
        """One scheduling round; returns whether any work is still pending."""
        for lane in self.lanes:
            if lane.event is not None and lane.event.query():
                self._complete(lane, release)
        self._admit()
        busy = any(l.event is not None for l in self.lanes) or self.releases_pending()
        self.adm.unblock(busy, self.now())
        for lane in self.lanes:
            if lane.event is None and self.admitted:
                self._launch(lane)
        return bool(self.waiting or self.admitted or any(l.event is not None for l in self.lanes))

    def drain(self, release: bool = True):
        while self.step(release):
            time.sleep(0)

    # -- results ----------------------------------------------------------------
    def result(self, req: Request):
        """(status, out_rec, out_perm, off) of a completed request whose memory
        was kept (step(release=False)); copies to the host."""
        n = int(req.off[self.W + 1]) if req.status == 0 else 0
        rec = self.out_rec[req.slot:req.slot + n].cpu().numpy()
        perm = self.out_perm[req.slot:req.slot + n].cpu().numpy().view(np.uint32).copy()
        return req.status, rec, perm, req.off

    def release(self, req: Request):
        self._release(req)

    # -- driving a trace ----------------------------------------------------------
    def releases_pending(self) -> bool:
        """Whether the caller still holds completed requests it will release
        (then a request that does not fit waits instead of being rejected).
        A caller that keeps results and frees them later replaces this."""
        return False

    def run_trace(self, requests: list[Request], release: bool = True,
                  on_done=None, on_step=None) -> dict:
        """Feeds requests at their arrival times (seconds after start) and runs
        until all are done.  on_done(request) runs for every completed
        request, on_step() once per scheduling round.  Returns latency and
        throughput statistics."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        k = 0
        seen = 0
        while True:
            now = self.now()
            while k < len(reqs) and reqs[k].arrival <= now:
                self.submit(reqs[k])
                k += 1
            pending = self.step(release)
            if on_done is not None:
                while seen < len(self.done):
                    on_done(self.done[seen])
                    seen += 1
            if on_step is not None:
                on_step()
            pending = pending or self.releases_pending()
            if k >= len(reqs) and not pending:
                break
            if k < len(reqs) and not pending:
                # idle until the next arrival
                time.sleep(min(0.0005, max(0.0, reqs[k].arrival - self.now())))
        return self.stats()

    def breakdown(self) -> dict:
        """Where the latency goes (ms percentiles): waiting for admission
        (arrival -> admit), for a lane (admit -> launch), and the batch on the
        device plus its completion poll (launch -> done); and the sizes of the
        slowest 1 % of requests."""
        ok = [r for r in self.done if r.status == 0]
        if not ok:
            return {}
        a = np.array([r.t_admit - r.arrival for r in ok]) * 1e3
        q = np.array([r.t_launch - r.t_admit for r in ok]) * 1e3
        d = np.array([r.t_done - r.t_launch for r in ok]) * 1e3
        lat = np.array([r.latency for r in ok])
        slow = np.argsort(lat)[-max(1, len(ok) // 100):]
        pc = lambda x: {"p50": round(float(np.percentile(x, 50)), 3),
                        "p99": round(float(np.percentile(x, 99)), 3)}
        return {"admit_wait_ms": pc(a), "lane_wait_ms": pc(q), "run_ms": pc(d),
                "slowest_1pct_words_median": int(np.median([ok[i].n_slots for i in slow])),
                "slowest_1pct_text_share": round(float(np.mean([ok[i].is_text for i in slow])), 3),
                "slowest_1pct_arrival_s": [round(float(np.min([ok[i].arrival for i in slow])), 2),
                                           round(float(np.max([ok[i].arrival for i in slow])), 2)]}

    def stats(self) -> dict:
        ok = [r for r in self.done if r.status == 0]
        lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
        words = sum(int(r.off[self.W + 1]) for r in ok)
        span = (max(r.t_done for r in self.done) - min(r.arrival for r in self.done)) \
            if self.done else 0.0
        return {"requests": len(self.done) + len(self.rejected), "completed": len(ok),
                "rejected": len(self.rejected), "failed": len(self.done) - len(ok),
                "batches": self.batches, "words": words,
                "mwords_per_s": words / span / 1e6 if span > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "span_s": span, "slots": self.n_slots}
