"""The C ABI library loads on the CPU and exports every symbol bsort.h declares.

No compute call is made here (no GPU): only symbol presence and the pure
host-side size arithmetic.
"""
from __future__ import annotations

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bsort.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1411_5283_gb300 import _lib, build
    build.build()
    return _lib


def declared() -> list[str]:
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(bsort_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi():
    names = declared()
    for want in ["bsort_tokenize", "bsort_bucket_by_length", "bsort_sort_buckets",
                 "bsort_gather", "bsort_sort_many", "bsort_workspace_size",
                 "bsort_get_status", "bsort_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (bsort_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_the_header(lib):
    assert sorted(lib.exported_symbols()) == declared()
    lib.load()  # every binding resolves


def test_workspace_size_roundtrip(lib):
    L = lib.load()
    for W in (8, 16, 24, 32):
        for n in (0, 1, 63, 64, 1000, 32768, 16_777_216):
            b = L.bsort_workspace_size(n, W, 2)
            assert b > 0 and b % 256 == 0
            assert L.bsort_workspace_capacity(b, W) >= n
            # one byte less may not hold more
            assert L.bsort_workspace_capacity(b - 1, W) <= L.bsort_workspace_capacity(b, W)
    assert L.bsort_workspace_size(10, 12, 2) == 0   # W not a multiple of 8
    assert L.bsort_workspace_size(10, 40, 2) == 0   # W above 32
    assert L.bsort_workspace_capacity(1 << 20, 7) == 0


def test_status_strings(lib):
    for c in range(8):
        assert lib.status_string(c) and "unknown" not in lib.status_string(c)


def test_list_descriptor_layout():
    import ctypes
    from paper_1411_5283_gb300 import _lib as L, batch
    assert batch.LIST_DTYPE.itemsize == ctypes.sizeof(L.ListDesc) == 32
    d = batch.record_lists([3, 0, 5], capacity=[4, 1, 5])
    assert d["word_off"].tolist() == [0, 4, 5]
    assert d["n_words"].tolist() == [3, 0, 5] and d["max_words"].tolist() == [4, 1, 5]
    t = batch.text_lists([10, 0, 7], [6, 1, 4])
    assert t["text_off"].tolist() == [0, 10, 10] and t["word_off"].tolist() == [0, 6, 7]


def test_sort_many_workspace_size(lib):
    L = lib.load()
    b = L.bsort_sort_many_workspace_size(1000, 10, 16)
    assert b > 0 and L.bsort_sort_many_workspace_size(1000, 10, 12) == 0
    assert L.bsort_sort_many_workspace_size(2000, 10, 16) > b


def test_packed_calls_refuse_bad_sizes_before_any_work(lib):
    """The packed calls check W, the offsets pointer and the 2^28-word /
    2^32-byte limits on the host and return before touching the device (the
    pointers below are never dereferenced)."""
    L = lib.load()
    fake = 1 << 20  # 16-byte aligned, never read
    E_INVALID, E_CAPACITY = 1, 3
    rec_call = L.bsort_sort_records_packed
    # n W at 2^32 bytes, and n above 2^28 words
    assert rec_call(fake, fake, 1 << 28, 16, 2, None, fake, 64, fake, fake, fake, fake, 1 << 20,
                    None) == E_CAPACITY
    assert rec_call(fake, fake, (1 << 28) + 1, 8, 2, None, fake, 64, fake, fake, fake, fake,
                    1 << 20, None) == E_CAPACITY
    # W not a multiple of 8, offsets missing, bytes missing for a non-empty call
    assert rec_call(fake, fake, 10, 12, 2, None, fake, 64, fake, fake, fake, fake, 1 << 20,
                    None) == E_INVALID
    assert rec_call(fake, fake, 10, 16, 2, None, fake, 64, None, fake, fake, fake, 1 << 20,
                    None) == E_INVALID
    assert rec_call(fake, fake, 10, 16, 2, None, None, 64, fake, fake, fake, fake, 1 << 20,
                    None) == E_INVALID
    text_call = L.bsort_sort_text_packed
    assert text_call(fake, 100, 16, 1 << 28, 2, None, fake, fake, fake, fake, fake, 64, fake, fake,
                     fake, fake, 1 << 20, None) == E_CAPACITY
    assert text_call(fake, 100, 16, 1000, 2, None, fake, fake, fake, fake, fake, 64, None, fake,
                     fake, fake, 1 << 20, None) == E_INVALID
