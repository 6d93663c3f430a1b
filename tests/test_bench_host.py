"""Host-side arithmetic of bench.py (no GPU): the algorithmic bytes that the
roofline figures divide by, worked out by hand on a tiny length histogram."""
from __future__ import annotations

import numpy as np

import bench


def test_kernel_bytes_by_hand():
    # three 1-letter words (one key word: 8 + 4 bytes per element) and five
    # 9-letter words (two key words: 16 + 4), W = 16, tiles of 2
    hist = np.zeros(17, dtype=np.int64)
    hist[1], hist[9] = 3, 5
    kb = bench.kernel_bytes(hist, 8, 16, 2)
    elem = 3 * 12 + 5 * 20                       # 136
    assert kb["hist"] == 8
    assert kb["scatter"] == 8 * 17 + elem        # records + lengths in, elements out
    assert kb["tile_bitonic"] == 2 * elem
    assert kb["gather"] == elem + 8 * 20         # elements in, records + permutation out
    assert kb["auto_bucket"] == 8 * 17 + elem
    # one-key elements travel as 8-byte items between partition and segment sort
    assert kb["auto_partition"] == elem + (3 * 8 + 5 * 20)
    assert kb["auto_segsort"] == (3 * 8 + 5 * 20) + 8 * 20
    # merge passes: runs of 2 (both buckets longer), runs of 4 (the 5-word
    # bucket); runs of 8 reach n = 8
    assert kb["merge_pass"] == 2 * elem + 2 * (5 * 20)


def test_clock_sampler_degrades_without_a_gpu():
    c = bench.Clocks(0)
    c.start()
    c.begin()
    c.end()
    out = c.stop()
    assert set(out) >= {"sm_mhz", "sm_max_mhz", "reasons", "samples"}
    if not c.nvml.ok:
        assert out["source"] == "nvidia-smi"


def test_nvml_reason_bits_are_distinct():
    bits = list(bench._Nvml.REASONS)
    assert len(set(bits)) == len(bits) and all(b & (b - 1) == 0 for b in bits)
    assert {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"} <= set(
        bench._Nvml.REASONS.values())
