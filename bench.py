#!/usr/bin/env python
"""Throughput benchmark of the length-bucketed word sort on GB300.

One step = the whole path (bucket by length -> per-bucket sort -> gather) over
the 16,777,216-word pre-tokenised table (32-byte records, lengths 1..32,
30 % Zipf words), the largest single-GPU workload.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--alg auto|merge|odd_even] [--words N]

N > 1 runs under torchrun as independent replicas (one full workload per
GPU; the path has no exchange step), value = all words sorted / slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mwords/s sorted end-to-end (tokenise/bucket/sort/gather)"
WORKLOAD = "large: 16,777,216 pre-tokenised words, W=32, seed 2"
N_WORDS = 16_777_216
W = 32
SEED = 2

# DRAM bytes per full-size launch from the committed ncu summaries (profiles/),
# by kernel, with the SHA-1 prefix of the kernel sources they were taken on:
# reported only while the sources still match (else null).
NCU_TRAFFIC = {
    # dram__bytes_read + dram__bytes_write of one launch on the 4,194,304-word
    # cut of the table, x4 for 16,777,216 words; a lower bound: at 4M words
    # part of each kernel's output is still in L2 when the next one reads it
    "auto_segsort": {"bytes": 4 * (60.71e6 + 126.42e6),
                     "sources": {"paper_1411_5283_gb300/csrc/auto.cu": "19ced58c997d",
                                 "paper_1411_5283_gb300/csrc/common.cuh": "401ac195dfb3",
                                 "paper_1411_5283_gb300/csrc/sort_impl.cuh": "8244b70a0067",
                                 "paper_1411_5283_gb300/csrc/block_scan.cuh": "8b681f3332d2"}},
    "auto_partition": {"bytes": 4 * (55.05e6 + 2.42e6),
                       "sources": {"paper_1411_5283_gb300/csrc/auto.cu": "19ced58c997d",
                                   "paper_1411_5283_gb300/csrc/common.cuh": "401ac195dfb3",
                                   "paper_1411_5283_gb300/csrc/block_scan.cuh": "8b681f3332d2"}},
    "auto_bucket": {"bytes": 4 * (138.86e6 + 23.33e6),
                    "sources": {"paper_1411_5283_gb300/csrc/auto.cu": "19ced58c997d",
                                "paper_1411_5283_gb300/csrc/common.cuh": "401ac195dfb3",
                                "paper_1411_5283_gb300/csrc/block_scan.cuh": "8b681f3332d2"}},
}


def ncu_traffic(kernel: str):
    """Committed DRAM traffic of kernel's launch, or None when its sources changed."""
    import hashlib
    e = NCU_TRAFFIC.get(kernel)
    if not e:
        return None
    for path, want in e["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest()[:len(want)] != want:
                return None
    return round(e["bytes"])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--alg", default="auto")
    ap.add_argument("--words", type=int, default=N_WORDS)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--e2e-depth", type=int, default=3, help="slots of the end-to-end host pipeline")
    ap.add_argument("--workload", choices=["large", "batched", "served", "text", "whole", "packed"],
                    default="large",
                    help="large: 16.7M pre-tokenised words (default, the headline line); "
                         "batched: 4,096 lists in one graph-captured batched call vs per-list "
                         "calls; served: Poisson requests through the continuous-batching "
                         "server; text: the 240,000-word raw text end to end; whole: the "
                         "unbucketed order of the large table; packed: the large table's answer "
                         "as packed bytes plus offsets")
    ap.add_argument("--pack-form", choices=["one-call", "two-call"], default="one-call",
                    help="packed: the sort writes the packed answer itself (one call), or "
                         "writes records that bsort_pack_words then packs (two calls)")
    ap.add_argument("--lists", type=int, default=4096)
    ap.add_argument("--served-check", choices=["inline", "replay"], default="replay",
                    help="served: compare every response with the oracle during the timed "
                         "run (inline) or in an untimed replay of the same trace")
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="served: requests per second")
    ap.add_argument("--profile-run", action="store_true",
                    help="warm-up and timed steps only (for ncu captures): no e2e, no CPU "
                         "baseline, no clock sampling; prints the device time only")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, the active
    clock-event reasons) for the device with the given UUID; None fields when
    the library or the device is not found."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str | None, index: int):
        import ctypes
        self.ok = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            r = lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) if uuid else 1
            if r != 0 and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                return
            self.lib, self.h, self.c = lib, h, ctypes
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            self.ok = self.sample() is not None
        except Exception:
            self.ok = False

    def sample(self):
        try:
            c = self.c
            mhz, mx, rs = c.c_uint(), c.c_uint(), c.c_ulonglong()
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, c.byref(mhz)) != 0:  # 1: SM clock
                return None
            self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, c.byref(mx))
            if self.reasons_fn is not None:
                self.reasons_fn(self.h, c.byref(rs))
            return time.perf_counter(), float(mhz.value), float(mx.value), int(rs.value)
        except Exception:
            return None


class Clocks:
    """Samples clocks and throttle reasons during the timed region: nvidia-smi
    every 200 ms (the recipe's query) and, where NVML loads, an in-process
    sampler every 2 ms, so that a region of a few tens of milliseconds still
    gets a dozen samples; begin() / end() bracket the region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        import threading
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(index).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            uuid = None
        self.nvml = _Nvml(uuid, index)
        self.samples, self.t0, self.t1 = [], None, None
        self.stop_flag = threading.Event()
        self.thread = threading.Thread(target=self._poll, daemon=True) if self.nvml.ok else None

    def _poll(self):
        while not self.stop_flag.is_set():
            smp = self.nvml.sample()
            if smp is not None:
                self.samples.append(smp)
            time.sleep(0.002)

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        if self.thread is not None:
            self.thread.start()
        time.sleep(0.3)

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def _smi(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}

    def stop(self) -> dict:
        smi = self._smi()
        if self.thread is None:
            return dict(smi, source="nvidia-smi")
        self.stop_flag.set()
        self.thread.join(timeout=5)
        t0 = self.t0 if self.t0 is not None else -1e30
        t1 = self.t1 if self.t1 is not None else 1e30
        win = [x for x in self.samples if t0 <= x[0] <= t1]
        if not win:
            return dict(smi, source="nvidia-smi")
        reasons = set()
        for _, _, _, bits in win:
            for b, nm in _Nvml.REASONS.items():
                if bits & b:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(x[1] for x in win), "sm_max_mhz": max(x[2] for x in win),
                "reasons": sorted(reasons), "samples": len(win), "source": "nvml every 2 ms in the timed region",
                "nvidia_smi": smi}


def kernel_bytes(hist: np.ndarray, n: int, Wd: int, tile: int) -> dict:
    """Algorithmic bytes of one step, per kernel, from the length histogram.

    Elements are (ceil(L/8) uint64 keys, uint32 index)."""
    L = np.arange(hist.size)
    K = (L + 7) // 8
    elem = (8 * K + 4) * hist  # bytes of all elements of each bucket
    # between partition and segment sort a one-key element travels as one
    # 8-byte item (code 2^ib + index) when that fits 64 bits, as it does for
    # every one-key segment of the large table
    seg_elem = np.where(K == 1, 8, 8 * K + 4) * hist
    kb = {
        "hist": n,                                            # read len
        "scatter": n * (Wd + 1) + int(elem.sum()),            # read rec+len, write keys+idx
        "tile_bitonic": 2 * int(elem.sum()),                  # read + write every element
        "tile_odd_even": 2 * int(elem.sum()),
        "gather": int(elem.sum()) + n * (Wd + 4),             # read keys+idx, write rec+perm
        # sample sort: the bucket pass reads rec+len and writes the staged
        # elements; partition reads them and writes them into segments; segsort
        # reads the segments and writes the final records + permutation
        "auto_bucket": n * (Wd + 1) + int(elem.sum()),
        "auto_partition": int(elem.sum()) + int(seg_elem.sum()),
        "auto_segsort": int(seg_elem.sum()) + n * (Wd + 4),
    }
    merge = 0
    R = tile
    while R < n:
        merge += 2 * int(elem[hist > R].sum())
        R *= 2
    kb["merge_pass"] = merge
    return kb


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import replicas, synth

    bs._lib.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.words
    rec_np, len_np = synth.large_records(SEED, n, W)
    rec_h = torch.from_numpy(rec_np).pin_memory()
    len_h = torch.from_numpy(len_np).pin_memory()
    rec = rec_h.to(dev)
    ln = len_h.to(dev)
    s = bs.Sorter(n, W, device=str(dev))
    stream = torch.cuda.current_stream()

    def step():
        s.sort_records(rec, ln, n, alg=args.alg)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = s.status()
    if st != 0:
        raise RuntimeError(f"device status {bs.bsort_status_string(st)}")

    if args.profile_run:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "words": n, "alg": args.alg,
                          "ms_per_step": e0.elapsed_time(e1) / args.steps,
                          "status": s.status()}), flush=True)
        return None

    # ---- device-resident timed region --------------------------------------
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.begin()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    # the same steps again with the library's per-kernel events (they add a
    # little time between launches, so the step time above is taken without)
    bs.bsort_profile_reset()
    bs.bsort_profile_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    bs.bsort_profile_enable(False)
    prof = bs.bsort_profile_read()

    # ---- end to end through the C ABI with host buffers -------------------
    # every step copies its input table in from pinned host memory and its
    # answer (records, permutation, offsets) back out; consecutive steps run
    # on --e2e-depth slots (streams, buffers, workspaces), so one step's
    # copy-in, an earlier step's sort and another's copy-out overlap on the GPU
    from paper_1411_5283_gb300.pipeline import HostPipeline
    depth = args.e2e_depth
    pipe = HostPipeline(n, W, depth=depth, device=str(dev))
    outs_h = [(torch.empty((n, W), dtype=torch.uint8).pin_memory(),
               torch.empty(n, dtype=torch.int32).pin_memory(),
               torch.empty(W + 2, dtype=torch.int32).pin_memory()) for _ in range(depth)]
    k2 = args.e2e_steps or max(3, min(args.steps, 10))

    def e2e_run(k):
        pipe.start_after()
        for j in range(k):
            o = outs_h[j % depth]
            pipe.submit(rec_h, len_h, n, o[0], o[1], o[2], alg=args.alg)
        pipe.wait_all()

    e2e_run(depth)
    torch.cuda.synchronize()
    if pipe.status() != 0:
        raise RuntimeError("device status after the end-to-end warm-up")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    e2e_run(k2)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = replicas.max_over_ranks(e0.elapsed_time(e1) / k2, dev)
    # the same, with the answer in the packed "vectors of string" form
    total_bytes = int(len_np.astype(np.int64).sum())
    outs_p = [(torch.empty(max(total_bytes, 16), dtype=torch.uint8).pin_memory(),
               torch.empty(n + 1, dtype=torch.int32).pin_memory(),
               torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(depth)]

    def e2e_packed_run(k):
        pipe.start_after()
        for j in range(k):
            o = outs_p[j % depth]
            pipe.submit_packed(rec_h, len_h, n, total_bytes, o[0], o[1], o[2], alg=args.alg)
        pipe.wait_all()

    e2e_packed_run(depth)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0.record(stream)
    e2e_packed_run(k2)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_packed_ms = replicas.max_over_ranks(e0.elapsed_time(e1) / k2, dev)
    d2h_packed = total_bytes + 4 * (n + 1) + 4 * n
    del pipe

    # ---- roofline of the dominant kernel ----------------------------------
    off = s.off.cpu().numpy().view(np.uint32).astype(np.int64)
    hist = np.diff(off)[: W + 1]  # hist[L] = words of length L (index 0 empty)
    hist = np.concatenate([[0], hist[1:]]) if hist.size else hist
    tile = 2048 if args.alg != "odd_even" else 512
    kb = kernel_bytes(hist, n, W, tile)
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (1, 1.0))
    name, (launches, tot_ms) = dom
    steps_prof = args.steps
    bytes_step = kb.get(name, 0)
    ms_step_kernel = tot_ms / steps_prof
    achieved = bytes_step / (ms_step_kernel * 1e-3) / 1e9 if ms_step_kernel > 0 else 0.0
    peak, peak_kind = peaks()
    compulsory = n * (W + 1) + n * (W + 4)
    path_gbs = compulsory / (ms * 1e-3) / 1e9
    # the timed step's output, kept for the oracle check of the CPU-baseline leg
    out_perm_np = s.out_perm[:n].cpu().numpy().view(np.uint32).copy()
    out_rec_np = s.out_rec[:n].cpu().numpy()
    return {
        "out": (out_rec_np, out_perm_np, off, len_np),
        "ms": ms, "e2e_ms": e2e_ms, "e2e_packed_ms": e2e_packed_ms, "d2h_packed": d2h_packed,
        "n": n, "prof": prof, "clk": clk,
        "roofline": {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": ncu_traffic(name), "peak_kind": peak_kind,
                     "launches_per_step": launches / steps_prof,
                     "algorithmic_bytes_per_step": bytes_step},
        "path_roofline": {"compulsory_bytes_per_word": W + 1 + W + 4,
                          "achieved": round(path_gbs, 1), "peak": peak, "unit": "GB/s",
                          "frac": round(path_gbs / peak, 4)},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "h2d": n * (W + 1), "d2h": n * (W + 4) + 4 * (W + 2),
    }


def cpu_baseline(out=None):
    """The oracle, as it stands, on bounded samples of the same workload.

    With ``out`` (the timed step's records, permutation, offsets and the input
    lengths) it also checks that output against the oracle: restricted to the
    words of the first 1,048,576 indices, the output must be exactly the
    oracle's answer on that prefix (the sort order is a strict total order,
    so a subset of a sorted sequence is the subset sorted), and the offsets
    must be the prefix sums of the length histogram."""
    import oracle
    from paper_1411_5283_gb300 import synth
    oracle.build()
    rec, ln = synth.large_records(SEED, 1 << 20, W)
    out_parity = None
    # the paper's method (bubble sort per length) on a 65,536-word sample
    m = 65_536
    t0 = time.perf_counter()
    res = oracle.bubble_sort(oracle.Words(rec[:m], ln[:m]))
    tb = time.perf_counter() - t0
    assert res.status == 0
    # the stable-sort formulation on a 1,048,576-word sample
    t0 = time.perf_counter()
    res = oracle.stable_sort(oracle.Words(rec, ln))
    ts = time.perf_counter() - t0
    assert res.status == 0
    if out is not None:
        out_rec, out_perm, off, len_all = out
        S = rec.shape[0]
        keep = out_perm < S
        sub = out_perm[keep]
        mism = int(np.count_nonzero(sub != res.out_perm)) if sub.size == S else abs(int(sub.size) - S)
        rec_ok = sub.size == S and bool(np.array_equal(out_rec[keep], res.out_rec))
        hist = np.bincount(len_all, minlength=W + 1)[: W + 1]
        want_off = np.concatenate([[0], np.cumsum(hist)]).astype(np.int64)
        off_ok = bool(np.array_equal(off, want_off))
        out_parity = {"checked_words": S, "perm_mismatches": mism, "records_equal": rec_ok,
                      "offsets_equal": off_ok, "ok": mism == 0 and rec_ok and off_ok,
                      "how": f"the benchmarked call's output (last step) restricted to input "
                             f"indices < {S:,} vs the oracle's stable sort of that prefix; "
                             "offsets vs the length histogram's prefix sums"}
    base = {"value": round(m / tb / 1e6, 6), "unit": "Mwords/s", "cores": 1, "kind": "oracle",
            "sample": f"bubble sort per length (paper's method) on the first {m:,} words of the "
                      f"workload: {tb:.2f} s; stable-sort oracle on the first "
                      f"{rec.shape[0]:,} words: {ts:.2f} s = "
                      f"{rec.shape[0] / ts / 1e6:.3f} Mwords/s",
            "stable_sort_mwords_s": round(rec.shape[0] / ts / 1e6, 4)}
    return base, out_parity


def run_reference(args):
    """Reference arm: the CPU oracle on the host cores (bounded sample per step)."""
    import oracle
    from paper_1411_5283_gb300 import synth
    oracle.build()
    m = 65_536
    rec, ln = synth.large_records(SEED, m, W)
    w = oracle.Words(rec, ln)
    for _ in range(args.warmup):
        oracle.bubble_sort(w)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.bubble_sort(w)
        times.append(time.perf_counter() - t0)
        assert r.status == 0
    sec = sum(times) / len(times)
    v = m / sec / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "Mwords/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_words": m, "algorithm": "bubble sort",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(v, 6), "unit": "Mwords/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"bubble sort per length on the first {m:,} words of "
                                       f"the workload, per step"},
            "e2e": {"value": round(v, 6), "unit": "Mwords/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """4,096 independent lists (seed i, log-uniform 64..65,536 words, W = 16) in
    one graph-replayed bsort_sort_many, against one plain call per list.
    Under torchrun the host router splits the lists over the ranks (each rank
    sorts its share; no data crosses GPUs), value = all words / slowest rank."""
    import torch

    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import autotune, batch, replicas, synth
    bs._lib.load()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    Wb = 16
    rec_all, ln_all, sizes_all = synth.batch_lists(args.lists, V=50_000, width=Wb, seed0=0)
    ids, starts = replicas.shard_lists(sizes_all, world, rank)
    rec, ln, sizes = replicas.gather_shard(rec_all, ln_all, sizes_all, ids, starts)
    n_all = int(ln_all.size)
    n = int(ln.size)
    desc = batch.record_lists(sizes)
    b = batch.BatchSorter(n, len(sizes), Wb)
    b.set_lists(desc)
    d_rec, d_len = torch.from_numpy(rec).cuda(), torch.from_numpy(ln).cuda()
    if args.profile_run:  # warm-up and timed calls only, default knobs (for ncu captures)
        for _ in range(args.warmup + args.steps):
            b.run(d_rec, d_len, text=False, max_list_words=65_536, alg="merge")
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "lists": len(sizes), "words": n,
                          "status": int(b.status[:len(sizes)].abs().sum())}), flush=True)
        return
    tune = autotune.tune_batch(b, d_rec, d_len, text=False, max_list_words=65_536,
                               total_words=n, alg="merge", max_candidates=12)
    b.capture(d_rec, d_len, text=False, max_list_words=65_536, alg="merge", tune=tune)
    for _ in range(args.warmup):
        b.replay()
    torch.cuda.synchronize()
    assert int(b.status[:len(sizes)].abs().sum()) == 0
    stream = torch.cuda.current_stream()
    bs.bsort_profile_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    # one profiled direct call for the per-kernel split
    bs.bsort_profile_enable(True)
    b.run(d_rec, d_len, text=False, max_list_words=65_536, alg="merge", tune=tune)
    torch.cuda.synchronize()
    bs.bsort_profile_enable(False)
    prof = bs.bsort_profile_read()
    # plain per-list calls on the same GPU, same lists
    s = bs.Sorter(int(sizes.max()), Wb)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    def plain():
        for i in range(len(sizes)):
            a, z = int(starts[i]), int(starts[i + 1])
            s.sort_records(d_rec[a:z], d_len[a:z], z - a, alg="merge", tune=tune)
    plain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    plain()
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    plain_wall = (time.perf_counter() - t0) * 1e3
    peak, kind = peaks()
    compulsory = n_all * (2 * Wb + 5)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": "Mwords/s sorted, batched lists", "value": round(n_all / ms / 1e3, 2),
            "unit": "Mwords/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"batched: {len(sizes_all)} lists, {n_all:,} words, W=16, "
                                   "seeds 0..", "graph": True, "tune": tune,
                       "parallelism": f"lists routed over {world} rank(s), no exchange"},
            "plain_per_list": {"ms": round(plain_ms, 3), "wall_ms": round(plain_wall, 3),
                               "mwords_per_s": round(n / plain_ms / 1e3, 2)},
            "path_roofline": {"achieved": round(compulsory / ms / 1e6, 1), "peak": peak,
                              "unit": "GB/s", "frac": round(compulsory / ms / 1e6 / peak, 4)},
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()}}
    print(json.dumps(line), flush=True)


def served_cpu_baseline(pool, Ws):
    """The served workload's CPU-baseline leg: the oracle (stable-sort
    formulation, one core) on every pooled payload, timed; its answers are
    kept to check every served response."""
    import oracle
    oracle.build()
    answers, words = [], 0
    t0 = time.perf_counter()
    for p in pool:
        if p[0] == "text":
            st, w, exp = oracle.sort_text(p[1], Ws, "stable")
            words += w.n
        else:
            exp = oracle.stable_sort(oracle.Words(p[1], p[2]))
            st = exp.status
            words += int(p[2].size)
        assert st == 0
        answers.append(exp)
    sec = time.perf_counter() - t0
    base = {"value": round(words / sec / 1e6, 4), "unit": "Mwords/s", "cores": 1,
            "kind": "oracle",
            "sample": f"stable-sort oracle (text payloads tokenised first) on the {len(pool)} "
                      f"pooled payloads, {words:,} words: {sec:.2f} s"}
    return base, answers


def run_served(args):
    """Poisson arrivals (rate x duration) of requests log-uniform in 1,024..1,048,576
    words (10 % raw text of the same word count), through the continuous-batching
    server (64 GB budget).  Payloads come from a pool of 128 generated requests
    (request i uses payload i mod 128).  Every completed response is compared
    with the oracle's answer for its payload, then released."""
    import torch

    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import serve, synth
    bs._lib.load()
    Ws = 16
    t, sizes, is_text = synth.request_stream(4, args.rate, args.duration)
    P = 128
    pool = []
    for i in range(P):
        m = int(sizes[i % len(sizes)])
        if is_text[i % len(sizes)]:
            pool.append(("text", synth.prose(10_000 + i, m, 12_000), m))
        else:
            pool.append(("rec",) + synth.list_words(10_000 + i, m, 50_000, Ws))
    base, answers = served_cpu_baseline(pool, Ws)
    srv = serve.Server(Ws, 64 << 30, max_list_words=1 << 20, max_batch_lists=1024)

    # payloads in pinned host memory: requests copy in asynchronously, as a
    # server receiving into pinned buffers would
    pinned = [("text", torch.from_numpy(np.frombuffer(p[1], np.uint8).copy()).pin_memory(), p[2])
              if p[0] == "text" else
              ("rec", torch.from_numpy(p[1]).pin_memory(), torch.from_numpy(p[2]).pin_memory())
              for p in pool]

    def request(rid, p, arrival=0.0):
        if p[0] == "text":
            return serve.Request(rid, arrival=arrival, text=p[1], max_words=p[2])
        return serve.Request(rid, arrival=arrival, rec=p[1], ln=p[2])

    # the oracle's answers, resident on the device (all payloads back to back)
    # so that responses are compared element by element without host copies
    e_sizes = [int(a.out_perm.size) for a in answers]
    e_start = np.concatenate([[0], np.cumsum(e_sizes)[:-1]]).astype(np.int64)
    E_rec = torch.from_numpy(np.concatenate([a.out_rec for a in answers])).cuda()
    E_perm = torch.from_numpy(np.concatenate([a.out_perm for a in answers]).view(np.int32)).cuda()
    reqs = [request(i, pinned[i % P], float(t[i])) for i in range(len(t))]
    # warm up the kernels on one request of each mode
    srv.run_trace([request(-1, pinned[0]), request(-2, next(p for p in pinned if p[0] == "text"))])
    srv.done.clear()
    srv.batches = 0
    # every response is compared with its payload's answer on the device, in
    # groups (one set of kernels per group, on a stream of its own, no host
    # sync); a response's memory is released once its group's comparison ran
    check_stream = torch.cuda.Stream()
    bad_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    group, pending = [], []
    checked = host_bad = 0

    def flush_checks():
        if not group:
            return
        dev_ = torch.device("cuda")
        total = int(sum(int(r.off[Ws + 1]) if r.status == 0 else 0 for r in group))
        for r in group:
            check_stream.wait_event(r.ev_end)
        # every tensor of the check is made and used on the check stream (the
        # caching allocator then reuses its memory only in that stream's order)
        meta = torch.tensor([[int(r.off[Ws + 1]) if r.status == 0 else 0 for r in group],
                             [int(r.slot) for r in group],
                             [int(e_start[r.rid % P]) for r in group]], dtype=torch.int64).pin_memory()
        with torch.cuda.stream(check_stream):
            md = meta.to(dev_, non_blocking=True)  # no host wait; the pinned block outlives the copy
            ns, slots, es = md[0], md[1], md[2]
            if total:
                which = torch.repeat_interleave(torch.arange(len(group), device=dev_), ns,
                                                output_size=total)
                first = torch.cumsum(ns, 0) - ns
                j = torch.arange(total, device=dev_) - first[which]
                oi, ei = slots[which] + j, es[which] + j
                bad = (srv.out_perm[oi] != E_perm[ei]).sum() + \
                    (srv.out_rec[oi] != E_rec[ei]).any(dim=1).sum()
                bad_dev.add_(bad)
            ev = torch.cuda.Event()
            ev.record(check_stream)
        pending.append((ev, list(group)))
        group.clear()

    def retire(block: bool):
        while pending and (block or pending[0][0].query()):
            ev, rs = pending.pop(0)
            ev.synchronize()
            for r in rs:
                srv.release(r)

    def on_done(r):
        nonlocal checked, host_bad
        exp = answers[r.rid % P]
        ok = r.status == 0 and np.array_equal(r.off, exp.off) and \
            int(r.off[Ws + 1]) == int(exp.out_perm.size)
        host_bad += 0 if ok else 1
        group.append(r)
        checked += 1

    def on_step():
        if len(group) >= 16 or (group and srv.now() - group[0].t_done > 0.002):
            flush_checks()
        retire(False)

    srv.releases_pending = lambda: bool(pending or group)
    if args.served_check == "inline":
        stats = srv.run_trace(reqs, release=False, on_done=on_done, on_step=on_step)
        flush_checks()
        retire(True)
    else:
        stats = srv.run_trace(reqs, release=True)
    stats["breakdown"] = srv.breakdown()
    if args.served_check == "replay":
        # the same trace once more, every response checked (this pass is not timed)
        srv.done.clear()
        srv.batches = 0
        srv.run_trace([request(i, pinned[i % P], float(t[i])) for i in range(len(t))],
                      release=False, on_done=on_done, on_step=on_step)
        flush_checks()
        retire(True)
    torch.cuda.synchronize()
    stats["oracle_checked"] = checked
    stats["oracle_mismatches"] = host_bad + int(bad_dev.item())
    stats["requests_per_batch"] = round(len(srv.done) / max(1, stats["batches"]), 3)
    line = {"metric": "served Mwords/s and p50/p99 latency", "value": round(stats["mwords_per_s"], 2),
            "unit": "Mwords/s", "n_gpus": 1, "higher_is_better": True, "dtype": "u8",
            "data": "synthetic", "config": {"workload": f"served: Poisson {args.rate}/s for "
                                            f"{args.duration}s, sizes 1024..1048576, 10% text",
                                            "budget_gb": 64, "pool": P},
            "p50_ms": round(stats["p50_ms"], 3), "p99_ms": round(stats["p99_ms"], 3),
            "stats": stats, "cpu_baseline": base,
            "check": args.served_check,
            "note": "every response is compared with the oracle's answer on the device as it "
                    "completes (in groups, on a stream of its own, no host sync), inside the "
                    "timed run (inline) or in an untimed replay of the same trace (replay)"}
    print(json.dumps(line), flush=True)


def run_variant(args):
    """The large table through the paper's other two forms: `whole` is the
    unbucketed order (Table 2, second row: every word by its bytes), `packed`
    the bucketed order written as packed bytes plus offsets (the "vectors of
    string" of §3.1) by the sort's last kernel (or, with --pack-form two-call,
    records packed by a second call).  One step = one pass of the form's path."""
    import torch

    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import synth
    bs._lib.load()
    n = args.words
    rec_np, len_np = synth.large_records(SEED, n, W)
    rec, ln = torch.from_numpy(rec_np).cuda(), torch.from_numpy(len_np).cuda()
    s = bs.Sorter(n, W)
    out_bytes = torch.empty(n * W, dtype=torch.uint8, device="cuda")
    if args.workload == "whole":
        def step():
            s.sort_records_whole(rec, ln, n, alg=args.alg)
    elif args.pack_form == "two-call":
        def step():
            s.sort_records(rec, ln, n, alg=args.alg)
            s.pack(n, bucketed=True, out_bytes=out_bytes)
    else:
        offsets = torch.empty(n + 1, dtype=torch.int32, device="cuda")

        def step():
            s.sort_records_packed(rec, ln, n, alg=args.alg, out_bytes=out_bytes, offsets=offsets)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert s.status() == 0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if args.profile_run:
        print(json.dumps({"profile_run": True, "workload": args.workload, "ms_per_step": ms}), flush=True)
        return
    bs.bsort_profile_reset()
    bs.bsort_profile_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    bs.bsort_profile_enable(False)
    prof = bs.bsort_profile_read()
    total_bytes = int(len_np.astype(np.int64).sum())
    line = {"metric": f"Mwords/s sorted, {args.workload} form", "value": round(n / ms / 1e3, 2),
            "unit": "Mwords/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD}", "alg": args.alg,
                       **({"pack_form": args.pack_form} if args.workload == "packed" else {})},
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()}}
    if args.workload == "packed":
        line["packed_output_bytes_per_word"] = round((total_bytes + 4 * (n + 1) + 4 * n) / n, 2)
        line["record_output_bytes_per_word"] = W + 4
    print(json.dumps(line), flush=True)


def run_text(args):
    """Raw text end to end (tokenise, bucket, sort, gather in one call): the
    32,768-word text of seed 0 (vocabulary 4,500) and the 240,000-word text of
    seed 1 (vocabulary 12,000), every algorithm.  These sizes are latency
    bound, so the line reports microseconds per call beside Mwords/s."""
    import torch

    import paper_1411_5283_gb300 as bs
    from paper_1411_5283_gb300 import synth
    bs._lib.load()
    Wt = 16
    stream = torch.cuda.current_stream()
    results = {}
    for name, seed, nw, V in (("small", 0, 32_768, 4_500), ("medium", 1, 240_000, 12_000)):
        text = synth.prose(seed, nw, V)
        d_text = torch.from_numpy(np.frombuffer(text, np.uint8).copy()).cuda()
        s = bs.Sorter(len(text) // 2 + 1, Wt)
        for alg in ("odd_even", "merge", "auto"):
            def step():
                s.sort_text(d_text, alg=alg)
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            assert s.status() == 0
            assert int(s.n_words.item()) == nw
            bs.bsort_profile_reset()
            bs.bsort_profile_enable(True)
            step()
            torch.cuda.synchronize()
            bs.bsort_profile_enable(False)
            prof = bs.bsort_profile_read()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            results[f"{name}/{alg}"] = {
                "words": nw, "text_bytes": len(text), "us_per_call": round(ms * 1e3, 2),
                "mwords_per_s": round(nw / ms / 1e3, 2),
                "launches_per_call": int(sum(v[0] for v in prof.values())),
                "kernels_us": {k: round(v[1] * 1e3, 2) for k, v in prof.items()}}
    head = results["medium/odd_even"]
    line = {"metric": "Mwords/s sorted end-to-end from raw text (tokenise/bucket/sort/gather)",
            "value": head["mwords_per_s"], "unit": "Mwords/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(head["us_per_call"] / 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "text: 240,000-word prose (seed 1, V=12,000), W=16, "
                                   "odd_even; also 32,768 words (seed 0) and every algorithm",
                       "l2": "inputs smaller than L2: latency-bound, no flush"},
            "runs": results}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "text":
        return run_text(args)
    if args.workload in ("whole", "packed"):
        return run_variant(args)
    if args.workload == "served":
        return run_served(args)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world, local_rank)
    if r is not None and rank == 0:
        from paper_1411_5283_gb300 import replicas
        n_total = r["n"] * world
        value = replicas.throughput(n_total, r["ms"])
        e2e_value = replicas.throughput(n_total, r["e2e_ms"])
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mwords/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "words": r["n"], "W": W, "alg": args.alg,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs (553 MB) larger than L2 (129 MB); no flush"},
            "e2e": {"value": round(e2e_value, 2), "unit": "Mwords/s",
                    "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                    "ms_per_step": round(r["e2e_ms"], 4),
                    "how": "pinned host table in, answer out, every step; consecutive steps "
                           f"on {args.e2e_depth} slots (HostPipeline streams) so copies and sorts overlap"},
            "e2e_packed": {"value": round(replicas.throughput(n_total, r["e2e_packed_ms"]), 2),
                           "unit": "Mwords/s", "h2d_bytes_per_step": r["h2d"],
                           "d2h_bytes_per_step": r["d2h_packed"],
                           "ms_per_step": round(r["e2e_packed_ms"], 4),
                           "how": "as e2e, the answer read back as packed bytes + offsets[n+1] + "
                                  "permutation (the paper's vectors-of-string form)"},
            "roofline": r["roofline"],
            "path_roofline": r["path_roofline"],
            "gpu_launches": r["gpu_launches"],
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in r["prof"].items()},
            "clocks": r["clk"],
        }
        if world == 1:
            line["cpu_baseline"], line["parity"] = cpu_baseline(r["out"])
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
