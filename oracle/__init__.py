"""Python handle on the CPU oracle -- TEST INFRASTRUCTURE ONLY.

The oracle (``bsort_oracle.cpp``) restates the paper's method (arXiv 1411.5283,
§3 Methodology, "Pre-processing", phases 1-3; bubble sort as described in §2 and
§3.2) as plain single-threaded C++.  This module compiles it with g++ and wraps
its entry points with ctypes, taking and returning numpy arrays.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never touches the CUDA library and
the CUDA library never touches it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsort_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, E_INVALID, E_WORD_TOO_LONG, E_CAPACITY = 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/liboracle.so`` (host code only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def bind(path: str):
    """Loads an oracle build from ``path`` and declares its C signatures."""
    lib = ctypes.CDLL(path)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.orc_tokenize.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 u8p, u8p, u32p, u32p]
    lib.orc_split_by_length.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint32, u32p, u32p]
    lib.orc_bubble_sort.argtypes = [u8p, u8p, ctypes.c_uint32, ctypes.c_uint32,
                                    u8p, u32p, u32p, u64p]
    lib.orc_stable_sort.argtypes = [u8p, u8p, ctypes.c_uint32, ctypes.c_uint32,
                                    u8p, u32p, u32p]
    lib.orc_bubble_sort_whole.argtypes = [u8p, u8p, ctypes.c_uint32, ctypes.c_uint32,
                                          u8p, u32p, u64p]
    lib.orc_stable_sort_whole.argtypes = [u8p, u8p, ctypes.c_uint32, ctypes.c_uint32,
                                          u8p, u32p]
    for f in (lib.orc_tokenize, lib.orc_split_by_length, lib.orc_bubble_sort,
              lib.orc_stable_sort, lib.orc_bubble_sort_whole, lib.orc_stable_sort_whole):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _p(a: np.ndarray | None, ct):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Words:
    """A table of words: ``rec[n, W]`` zero-padded letters, ``len[n]``."""
    rec: np.ndarray
    len: np.ndarray
    src_off: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.len.shape[0])

    @property
    def W(self) -> int:
        return int(self.rec.shape[1])


@dataclass
class Sorted:
    """The method's answer: words in (length, alphabetic, input index) order."""
    status: int
    out_rec: np.ndarray
    out_perm: np.ndarray
    off: np.ndarray          # off[L] = number of words shorter than L, L = 0..W+1
    swaps: np.ndarray | None = None   # bubble-sort exchanges per length (index L)


def tokenize(text: bytes | np.ndarray, W: int, max_words: int | None = None):
    """Phase 1: returns ``(status, Words, n_found)``."""
    lib = _load()
    t = np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) \
        else np.ascontiguousarray(text, dtype=np.uint8)
    if max_words is None:
        max_words = int(t.size // 2 + 1)
    rec = np.zeros((max(max_words, 1), W), dtype=np.uint8)
    ln = np.zeros(max(max_words, 1), dtype=np.uint8)
    so = np.zeros(max(max_words, 1), dtype=np.uint32)
    nw = np.zeros(1, dtype=np.uint32)
    st = lib.orc_tokenize(_p(t, ctypes.c_uint8) if t.size else None, t.size, W, max_words,
                          _p(rec, ctypes.c_uint8), _p(ln, ctypes.c_uint8),
                          _p(so, ctypes.c_uint32), _p(nw, ctypes.c_uint32))
    n = min(int(nw[0]), max_words)
    return st, Words(rec[:n].copy(), ln[:n].copy(), so[:n].copy()), int(nw[0])


def split_by_length(ln: np.ndarray, W: int):
    """Phase 2 alone: ``(status, off[W+2], ids grouped by length in input order)``."""
    lib = _load()
    ln = np.ascontiguousarray(ln, dtype=np.uint8)
    n = ln.size
    off = np.zeros(W + 2, dtype=np.uint32)
    ids = np.zeros(max(n, 1), dtype=np.uint32)
    st = lib.orc_split_by_length(_p(ln, ctypes.c_uint8) if n else None, n, W,
                                 _p(off, ctypes.c_uint32), _p(ids, ctypes.c_uint32))
    return st, off, ids[:n]


def _sort(fn: str, w: Words, with_swaps: bool) -> Sorted:
    lib = _load()
    rec = np.ascontiguousarray(w.rec, dtype=np.uint8)
    ln = np.ascontiguousarray(w.len, dtype=np.uint8)
    n, W = ln.size, rec.shape[1]
    out_rec = np.zeros((max(n, 1), W), dtype=np.uint8)
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    off = np.zeros(W + 2, dtype=np.uint32)
    args = [_p(rec, ctypes.c_uint8) if n else None, _p(ln, ctypes.c_uint8) if n else None,
            n, W, _p(out_rec, ctypes.c_uint8), _p(perm, ctypes.c_uint32),
            _p(off, ctypes.c_uint32)]
    swaps = None
    if with_swaps:
        swaps = np.zeros(W + 1, dtype=np.uint64)
        args.append(_p(swaps, ctypes.c_uint64))
    st = getattr(lib, fn)(*args)
    return Sorted(st, out_rec[:n], perm[:n], off, swaps)


def bubble_sort(w: Words) -> Sorted:
    """Phases 2-3 and concatenation, bubble sort per length (O1)."""
    return _sort("orc_bubble_sort", w, True)


def stable_sort(w: Words) -> Sorted:
    """The same answer by one stable library sort on (length, bytes) (O2)."""
    return _sort("orc_stable_sort", w, False)


def sort_text(text: bytes, W: int, method: str = "bubble") -> tuple[int, Words, Sorted | None]:
    """Phase 1 then phases 2-3: returns ``(status, tokenised words, answer)``."""
    st, w, _ = tokenize(text, W)
    if st != OK:
        return st, w, None
    res = bubble_sort(w) if method == "bubble" else stable_sort(w)
    return res.status, w, res


@dataclass
class SortedWhole:
    """Every word in (bytes, input index) order, without length buckets."""
    status: int
    out_rec: np.ndarray
    out_perm: np.ndarray
    swaps: int | None = None


def _sort_whole(fn: str, w: Words, with_swaps: bool) -> SortedWhole:
    lib = _load()
    rec = np.ascontiguousarray(w.rec, dtype=np.uint8)
    ln = np.ascontiguousarray(w.len, dtype=np.uint8)
    n, W = ln.size, rec.shape[1]
    out_rec = np.zeros((max(n, 1), W), dtype=np.uint8)
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    args = [_p(rec, ctypes.c_uint8) if n else None, _p(ln, ctypes.c_uint8) if n else None,
            n, W, _p(out_rec, ctypes.c_uint8), _p(perm, ctypes.c_uint32)]
    swaps = None
    if with_swaps:
        sw = np.zeros(1, dtype=np.uint64)
        args.append(_p(sw, ctypes.c_uint64))
    st = getattr(lib, fn)(*args)
    if with_swaps:
        swaps = int(sw[0])
    return SortedWhole(st, out_rec[:n], perm[:n], swaps)


def bubble_sort_whole(w: Words) -> SortedWhole:
    """The whole file's words by bubble sort, no length sub-arrays (Table 2,
    second row)."""
    return _sort_whole("orc_bubble_sort_whole", w, True)


def stable_sort_whole(w: Words) -> SortedWhole:
    """The same answer by one stable library sort on the byte strings."""
    return _sort_whole("orc_stable_sort_whole", w, False)


def pack_words(out_rec: np.ndarray, lengths: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The paper's other data structure (§3.1, "vectors of string"): the sorted
    words as one packed byte buffer without padding, and offsets[n + 1] with
    word r at bytes[offsets[r]:offsets[r + 1]].  out_rec holds the sorted
    records and lengths their lengths in the same (output) order."""
    n = int(lengths.size)
    offsets = np.zeros(n + 1, dtype=np.uint32)
    parts = []
    for r in range(n):
        L = int(lengths[r])
        parts.append(bytes(out_rec[r, :L]))
        offsets[r + 1] = offsets[r] + L
    return np.frombuffer(b"".join(parts), dtype=np.uint8).copy(), offsets
