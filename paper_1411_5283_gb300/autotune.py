"""Autotuner for the sort's tuning knobs (``bsort_tune``).

For a device, record width W, algorithm and size class (n rounded up to a
power of two) it times every candidate setting of tile size (bitonic),
odd-even tile size, threads per tile-sort CTA and merge-path partition size,
then, for the merge path, the bucket-size crossover below which a bucket is
sorted whole by odd-even transposition; it keeps the fastest, and caches it as JSON keyed by device name, SM count, W,
algorithm, size class and call kind (single list or batched).  Results never
depend on the knobs; only the time does.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from typing import Callable

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "bsort_tune.json")


def cache_path() -> str:
    return os.environ.get("BSORT_TUNE_CACHE", DEFAULT_CACHE)


def size_class(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(1, n))))


def tune_key(device: str, sms: int, W: int, alg: str, n: int, kind: str = "single") -> str:
    return f"{device}|sm{sms}|W{W}|{alg}|n{size_class(n)}|{kind}"


def candidates(alg: str, W: int) -> list[dict]:
    """The settings swept for an algorithm (all valid for bsort_tune)."""
    KW = W // 8
    parts = [p for p in (512, 1024, 2048, 4096) if 2 * p * (8 * KW + 4) <= 200 * 1024]
    out = []
    if alg == "odd_even":
        for oe, th in itertools.product((128, 256, 512, 1024), (256, 512)):
            for p in parts:
                if p <= 2 * oe:
                    out.append({"oddeven_max": oe, "threads_per_bucket": th, "merge_fanin": p})
    else:
        for t, th in itertools.product((1024, 2048, 4096), (256, 512, 1024)):
            for p in parts:
                if p <= 2 * t:
                    out.append({"tile": t, "threads_per_bucket": th, "merge_fanin": p})
    return out


# odd-even / merge crossovers swept for the MERGE path (words per bucket sorted
# whole by odd-even transposition; 1 = never)
CROSSOVERS = (1, 16, 32, 64, 128, 256, 512, 1024)


def crossover_candidates(base: dict) -> list[dict]:
    """The base setting with every crossover that fits its tile."""
    tile = base.get("tile", 2048)
    return [dict(base, oddeven_cross=x) for x in CROSSOVERS if x <= tile]


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(time_fn: Callable[[dict], float], cands: list[dict]) -> tuple[dict, float]:
    """The candidate with the smallest time_fn (seconds); ties keep the first."""
    best, best_t = None, float("inf")
    for c in cands:
        t = time_fn(c)
        if t < best_t:
            best, best_t = c, t
    return best, best_t


def lookup(key: str, path: str | None = None) -> dict | None:
    e = load_cache(path).get(key)
    return dict(e["tune"]) if e else None


def tune(key: str, time_fn: Callable[[dict], float], cands: list[dict],
         path: str | None = None, force: bool = False,
         refine: Callable[[dict], list[dict]] | None = None) -> dict:
    """Returns the cached setting for key, or sweeps cands with time_fn and
    caches the fastest.  refine(best) may list a second sweep around the
    first one's winner (the merge path's odd-even crossover)."""
    cache = load_cache(path)
    if not force and key in cache:
        return dict(cache[key]["tune"])
    best, t = choose(time_fn, cands)
    n = len(cands)
    if refine is not None:
        # the second sweep includes the winner's own setting (the default
        # crossover is one of its values), so its fastest entry is kept
        more = refine(best)
        best, t = choose(time_fn, more)
        n += len(more)
    cache[key] = {"tune": best, "seconds": t, "candidates": n}
    save_cache(cache, path)
    return dict(best)


# ---------------------------------------------------------------------------
# GPU timing helpers
# ---------------------------------------------------------------------------

def device_id() -> tuple[str, int]:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return p.name, p.multi_processor_count


def cuda_timer(run: Callable[[], None], reps: int = 5, warmup: int = 2) -> float:
    """Median seconds of run() measured with CUDA events on the current stream."""
    import torch
    for _ in range(warmup):
        run()
    ts = []
    s = torch.cuda.current_stream()
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        run()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    ts.sort()
    return ts[len(ts) // 2]


def tune_records(sorter, rec, ln, n: int, alg: str = "merge", path: str | None = None,
                 force: bool = False, max_candidates: int | None = None) -> dict:
    """Tunes the single-list path on this table (Sorter.sort_records)."""
    name, sms = device_id()
    cands = candidates(alg, sorter.W)[:max_candidates]
    key = tune_key(name, sms, sorter.W, alg, n, "single")
    return tune(key, lambda c: cuda_timer(lambda: sorter.sort_records(rec, ln, n, alg=alg, tune=c)),
                cands, path, force, crossover_candidates if alg != "odd_even" else None)


def tune_batch(bsorter, data, ln, *, text: bool, max_list_words: int, total_words: int,
               alg: str = "merge", path: str | None = None, force: bool = False,
               max_candidates: int | None = None) -> dict:
    """Tunes the batched path (BatchSorter.run) on this batch."""
    name, sms = device_id()
    cands = candidates(alg, bsorter.W)[:max_candidates]
    key = tune_key(name, sms, bsorter.W, alg, total_words, "batched")
    return tune(key, lambda c: cuda_timer(lambda: bsorter.run(
        data, ln, text=text, max_list_words=max_list_words, alg=alg, tune=c)), cands, path, force,
        crossover_candidates if alg != "odd_even" else None)
