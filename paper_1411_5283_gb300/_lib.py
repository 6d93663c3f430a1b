"""ctypes binding of ``libbsort.so``: the C ABI of ``include/bsort.h``, same names.

Argument marshalling only: every function takes CUDA tensors (or raw device
pointers), passes their addresses and the current CUDA stream to the library,
and raises :class:`BsortError` on a non-OK status.  There is no fallback: if
the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbsort.so")

OK, E_INVALID, E_WORD_TOO_LONG, E_CAPACITY, E_WORKSPACE, E_CUDA, E_TIMEOUT, E_NOMEM = range(8)
ODD_EVEN, MERGE, AUTO = 0, 1, 2
ALGS = {"odd_even": ODD_EVEN, "merge": MERGE, "auto": AUTO}

_lib = None

c_u8p = ctypes.c_void_p
c_size = ctypes.c_size_t


class BsortError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class Tune(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_uint32), ("oddeven_max", ctypes.c_uint32),
                ("threads_per_bucket", ctypes.c_uint32), ("merge_fanin", ctypes.c_uint32),
                ("oddeven_cross", ctypes.c_uint32)]


class ListDesc(ctypes.Structure):
    _fields_ = [("text_off", ctypes.c_uint64), ("text_bytes", ctypes.c_uint64),
                ("word_off", ctypes.c_uint64), ("n_words", ctypes.c_uint32),
                ("max_words", ctypes.c_uint32)]


_SIGS = {
    "bsort_workspace_size": (c_size, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int]),
    "bsort_workspace_capacity": (ctypes.c_uint64, [c_size, ctypes.c_uint32]),
    "bsort_workspace_init": (ctypes.c_int, [c_u8p, c_size, c_u8p]),
    "bsort_tokenize": (ctypes.c_int, [c_u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      c_u8p, c_u8p, c_u8p, c_u8p, c_u8p, c_size, c_u8p]),
    "bsort_bucket_by_length": (ctypes.c_int, [c_u8p, c_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                              c_u8p, c_u8p, c_size, c_u8p]),
    "bsort_sort_buckets": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                          ctypes.POINTER(Tune), c_u8p, c_u8p, c_size, c_u8p]),
    "bsort_gather": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, c_u8p, c_u8p, c_size,
                                    c_u8p, c_u8p, c_u8p]),
    "bsort_sort_records": (ctypes.c_int, [c_u8p, c_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int, ctypes.POINTER(Tune), c_u8p, c_u8p,
                                          c_u8p, c_u8p, c_size, c_u8p]),
    "bsort_sort_text": (ctypes.c_int, [c_u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int, ctypes.POINTER(Tune), c_u8p, c_u8p, c_u8p,
                                       c_u8p, c_u8p, c_u8p, c_u8p, c_u8p, c_size, c_u8p]),
    "bsort_sort_records_whole": (ctypes.c_int, [c_u8p, c_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                                ctypes.c_int, ctypes.POINTER(Tune), c_u8p, c_u8p,
                                                c_u8p, c_size, c_u8p]),
    "bsort_sort_text_whole": (ctypes.c_int, [c_u8p, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(Tune),
                                             c_u8p, c_u8p, c_u8p, c_u8p, c_u8p, c_u8p, c_u8p,
                                             c_size, c_u8p]),
    "bsort_pack_words": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, c_u8p, c_u8p, c_u8p,
                                        c_u8p, c_u8p, ctypes.c_uint64, c_u8p, c_u8p, c_size,
                                        c_u8p]),
    "bsort_sort_records_packed": (ctypes.c_int, [c_u8p, c_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                                 ctypes.c_int, ctypes.POINTER(Tune), c_u8p,
                                                 ctypes.c_uint64, c_u8p, c_u8p, c_u8p, c_u8p,
                                                 c_size, c_u8p]),
    "bsort_sort_text_packed": (ctypes.c_int, [c_u8p, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(Tune),
                                              c_u8p, c_u8p, c_u8p, c_u8p, c_u8p, ctypes.c_uint64,
                                              c_u8p, c_u8p, c_u8p, c_u8p, c_size, c_u8p]),
    "bsort_sort_records_noalloc": (ctypes.c_int, [c_u8p, c_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                                  ctypes.c_int, ctypes.POINTER(Tune), c_u8p,
                                                  c_u8p, c_u8p, c_u8p, c_u8p]),
    "bsort_sort_many_workspace_size": (c_size, [ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32]),
    "bsort_sort_many": (ctypes.c_int, [c_u8p, c_u8p, c_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                       ctypes.POINTER(Tune), c_u8p, c_u8p, c_u8p, c_u8p, c_u8p,
                                       c_size, c_u8p]),
    "bsort_export_buckets": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, c_u8p, c_u8p,
                                            c_size, c_u8p, c_u8p, c_u8p]),
    "bsort_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "bsort_profile_reset": (ctypes.c_int, []),
    "bsort_profile_read": (ctypes.c_uint32, [ctypes.c_char_p, c_size,
                                             ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_uint32]),
    "bsort_set_wait_limit": (ctypes.c_int, [ctypes.c_uint32]),
    "bsort_get_status": (ctypes.c_int, [c_u8p, c_u8p]),
    "bsort_reset_status": (ctypes.c_int, [c_u8p, c_u8p]),
    "bsort_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str = LIB_PATH):
    """Loads the compiled library (raises if it is missing) and declares signatures."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbsort.so not built at {path}: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def status_string(st: int) -> str:
    try:
        return load().bsort_status_string(int(st)).decode()
    except ImportError:
        return f"status {st}"


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _tune(tune) -> Optional[ctypes.POINTER(Tune)]:
    if tune is None:
        return None
    if isinstance(tune, dict):
        tune = Tune(**tune)
    return ctypes.pointer(tune)


def _alg(alg) -> int:
    return ALGS[alg] if isinstance(alg, str) else int(alg)


def _check(st: int, where: str):
    if st != OK:
        raise BsortError(st, where)


# ---------------------------------------------------------------------------
# The C ABI, one function each
# ---------------------------------------------------------------------------

def bsort_workspace_size(max_words: int, W: int, alg=AUTO) -> int:
    return int(load().bsort_workspace_size(max_words, W, _alg(alg)))


def bsort_workspace_capacity(ws_bytes: int, W: int) -> int:
    return int(load().bsort_workspace_capacity(ws_bytes, W))


def bsort_workspace_init(ws, ws_bytes: int, stream=None):
    _check(load().bsort_workspace_init(_ptr(ws), ws_bytes, _stream(stream)),
           "bsort_workspace_init")


def bsort_tokenize(text, n_bytes, W, max_words, rec, ln, src_off, n_words, ws, ws_bytes,
                   stream=None):
    _check(load().bsort_tokenize(_ptr(text), n_bytes, W, max_words, _ptr(rec), _ptr(ln),
                                 _ptr(src_off), _ptr(n_words), _ptr(ws), ws_bytes,
                                 _stream(stream)), "bsort_tokenize")


def bsort_bucket_by_length(rec, ln, n, W, off, ws, ws_bytes, stream=None):
    _check(load().bsort_bucket_by_length(_ptr(rec), _ptr(ln), n, W, _ptr(off), _ptr(ws),
                                         ws_bytes, _stream(stream)), "bsort_bucket_by_length")


def bsort_sort_buckets(n, W, alg, tune, off, ws, ws_bytes, stream=None):
    _check(load().bsort_sort_buckets(n, W, _alg(alg), _tune(tune), _ptr(off), _ptr(ws),
                                     ws_bytes, _stream(stream)), "bsort_sort_buckets")


def bsort_gather(n, W, off, ws, ws_bytes, out_rec, out_perm, stream=None):
    _check(load().bsort_gather(n, W, _ptr(off), _ptr(ws), ws_bytes, _ptr(out_rec),
                               _ptr(out_perm), _stream(stream)), "bsort_gather")


def bsort_sort_records(rec, ln, n, W, alg, tune, out_rec, out_perm, off, ws, ws_bytes,
                       stream=None):
    _check(load().bsort_sort_records(_ptr(rec), _ptr(ln), n, W, _alg(alg), _tune(tune),
                                     _ptr(out_rec), _ptr(out_perm), _ptr(off), _ptr(ws),
                                     ws_bytes, _stream(stream)), "bsort_sort_records")


def bsort_sort_text(text, n_bytes, W, max_words, alg, tune, rec, ln, src_off, n_words, out_rec,
                    out_perm, off, ws, ws_bytes, stream=None):
    _check(load().bsort_sort_text(_ptr(text), n_bytes, W, max_words, _alg(alg), _tune(tune),
                                  _ptr(rec), _ptr(ln), _ptr(src_off), _ptr(n_words),
                                  _ptr(out_rec), _ptr(out_perm), _ptr(off), _ptr(ws), ws_bytes,
                                  _stream(stream)), "bsort_sort_text")


def bsort_sort_records_whole(rec, ln, n, W, alg, tune, out_rec, out_perm, ws, ws_bytes,
                             stream=None):
    _check(load().bsort_sort_records_whole(_ptr(rec), _ptr(ln), n, W, _alg(alg), _tune(tune),
                                           _ptr(out_rec), _ptr(out_perm), _ptr(ws), ws_bytes,
                                           _stream(stream)), "bsort_sort_records_whole")


def bsort_sort_text_whole(text, n_bytes, W, max_words, alg, tune, rec, ln, src_off, n_words,
                          out_rec, out_perm, ws, ws_bytes, stream=None):
    _check(load().bsort_sort_text_whole(_ptr(text), n_bytes, W, max_words, _alg(alg),
                                        _tune(tune), _ptr(rec), _ptr(ln), _ptr(src_off),
                                        _ptr(n_words), _ptr(out_rec), _ptr(out_perm), _ptr(ws),
                                        ws_bytes, _stream(stream)), "bsort_sort_text_whole")


def bsort_pack_words(n, W, rec, off, perm, ln, out_bytes, bytes_cap, offsets, ws, ws_bytes,
                     stream=None):
    _check(load().bsort_pack_words(n, W, _ptr(rec), _ptr(off), _ptr(perm), _ptr(ln),
                                   _ptr(out_bytes), bytes_cap, _ptr(offsets), _ptr(ws), ws_bytes,
                                   _stream(stream)), "bsort_pack_words")


def bsort_sort_records_packed(rec, ln, n, W, alg, tune, out_bytes, bytes_cap, offsets, out_perm,
                              off, ws, ws_bytes, stream=None):
    _check(load().bsort_sort_records_packed(_ptr(rec), _ptr(ln), n, W, _alg(alg), _tune(tune),
                                            _ptr(out_bytes), bytes_cap, _ptr(offsets),
                                            _ptr(out_perm), _ptr(off), _ptr(ws), ws_bytes,
                                            _stream(stream)), "bsort_sort_records_packed")


def bsort_sort_text_packed(text, n_bytes, W, max_words, alg, tune, rec, ln, src_off, n_words,
                           out_bytes, bytes_cap, offsets, out_perm, off, ws, ws_bytes,
                           stream=None):
    _check(load().bsort_sort_text_packed(_ptr(text), n_bytes, W, max_words, _alg(alg),
                                         _tune(tune), _ptr(rec), _ptr(ln), _ptr(src_off),
                                         _ptr(n_words), _ptr(out_bytes), bytes_cap,
                                         _ptr(offsets), _ptr(out_perm), _ptr(off), _ptr(ws),
                                         ws_bytes, _stream(stream)), "bsort_sort_text_packed")


def bsort_sort_many_workspace_size(total_words: int, n_lists: int, W: int) -> int:
    return int(load().bsort_sort_many_workspace_size(total_words, n_lists, W))


def bsort_sort_many(text_or_rec, ln, lists, n_lists, W, lists_are_text, max_list_words, alg,
                    tune, out_rec, out_perm, out_off, list_status, ws, ws_bytes, stream=None):
    _check(load().bsort_sort_many(_ptr(text_or_rec), _ptr(ln), _ptr(lists), n_lists, W,
                                  int(lists_are_text), max_list_words, _alg(alg), _tune(tune),
                                  _ptr(out_rec), _ptr(out_perm), _ptr(out_off),
                                  _ptr(list_status), _ptr(ws), ws_bytes, _stream(stream)),
           "bsort_sort_many")


def bsort_sort_records_noalloc(rec, ln, n, W, alg, tune, out_rec, out_perm, off, status=None,
                               stream=None):
    """Whole record sort with the library's static scratch (no workspace)."""
    _check(load().bsort_sort_records_noalloc(_ptr(rec), _ptr(ln), n, W, _alg(alg), _tune(tune),
                                             _ptr(out_rec), _ptr(out_perm), _ptr(off),
                                             _ptr(status), _stream(stream)),
           "bsort_sort_records_noalloc")


def bsort_export_buckets(n, W, off, ws, ws_bytes, keys, idx, stream=None):
    _check(load().bsort_export_buckets(n, W, _ptr(off), _ptr(ws), ws_bytes, _ptr(keys),
                                       _ptr(idx), _stream(stream)), "bsort_export_buckets")


def bsort_profile_enable(on: bool = True):
    _check(load().bsort_profile_enable(1 if on else 0), "bsort_profile_enable")


def bsort_profile_reset():
    _check(load().bsort_profile_reset(), "bsort_profile_reset")


def bsort_profile_read() -> dict:
    """{kernel name: (launches, total device ms)} since the last reset."""
    lib = load()
    cap = 64
    names = ctypes.create_string_buffer(64 * cap)
    launches = (ctypes.c_uint64 * cap)()
    ms = (ctypes.c_double * cap)()
    n = lib.bsort_profile_read(names, 64 * cap, launches, ms, cap)
    parts = names.raw.split(b"\0")
    return {parts[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(n, cap))}


WAIT_DEFAULT = 0xFFFFFFFF


def bsort_set_wait_limit(polls: int):
    """Polls of the kernels' first wait for a bulk copy (WAIT_DEFAULT restores
    the default; 0 makes every such wait give up at once)."""
    _check(load().bsort_set_wait_limit(int(polls)), "bsort_set_wait_limit")


def bsort_get_status(ws, stream=None) -> int:
    return int(load().bsort_get_status(_ptr(ws), _stream(stream)))


def bsort_reset_status(ws, stream=None):
    _check(load().bsort_reset_status(_ptr(ws), _stream(stream)), "bsort_reset_status")


def bsort_status_string(st: int) -> str:
    return status_string(st)
