// C ABI of the bsort library: argument checks, workspace views and launches.
// Every operation runs in the kernels of this directory; nothing here touches
// the data.
#include <cstring>

#include "common.cuh"
#include "kernels.h"

using namespace bsort;

namespace bsort {

namespace {
std::atomic<uint32_t> g_first_wait_polls{kSpinLimit};
}  // namespace

uint32_t first_wait_polls() { return g_first_wait_polls.load(std::memory_order_relaxed); }

}  // namespace bsort

namespace {

bool valid_W(uint32_t W) { return W >= 8 && W <= kMaxW && W % 8 == 0; }

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

bsort_status cuda_status(cudaError_t e) { return e == cudaSuccess ? BSORT_OK : BSORT_E_CUDA; }

bsort_status check_ws(const void* d_ws, size_t ws_bytes, uint32_t W, uint64_t need_words) {
  if (!d_ws || !aligned(d_ws, 256)) return BSORT_E_WORKSPACE;
  if (ws_capacity(ws_bytes, W) < need_words) return BSORT_E_WORKSPACE;
  return BSORT_OK;
}

}  // namespace

namespace bsort {

namespace {

// One set per host thread and device keeps concurrent calls from different
// threads from sharing events; calls on one thread are ordered by their
// streams, so reusing the events is safe.
struct SideSlot {
  SideStream s{};
  bool failed = false;
};
thread_local SideSlot t_side[kMaxDevices];

}  // namespace

SideStream* side_stream() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  SideSlot& t = t_side[dev];
  if (t.failed) return nullptr;
  if (!t.s.side) {
    if (cudaStreamCreateWithFlags(&t.s.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&t.s.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t.s.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();  // run without the helper stream
      t.failed = true;
      return nullptr;
    }
  }
  return &t.s;
}

}  // namespace bsort

bool bsort::resolve_params(bsort_alg alg, const bsort_tune* tune, uint32_t W, SortParams* p) {
  bsort_tune t{};
  if (tune) t = *tune;
  (void)W;  // every record width takes the same defaults
  p->alg = alg == BSORT_ODD_EVEN ? BSORT_ODD_EVEN : BSORT_MERGE;
  if (p->alg == BSORT_ODD_EVEN) {
    p->tile = t.oddeven_max ? t.oddeven_max : 512;
    if (!pow2(p->tile) || p->tile < 64 || p->tile > 2048) return false;
  } else {
    p->tile = t.tile ? t.tile : 2048;
    if (!pow2(p->tile) || p->tile < 256 || p->tile > 4096) return false;
  }
  // bitonic tiles sort four positions per thread in registers by default
  p->threads = t.threads_per_bucket ? t.threads_per_bucket
                                    : (p->alg == BSORT_ODD_EVEN ? 256u : (p->tile / 4 < 64 ? 64u : p->tile / 4));
  if (p->threads < 64 || p->threads > 1024 || p->threads % 32) return false;
  // partitions of one-key elements; wider elements take part / 2 or part / 4
  // (merge_part_for), so one shared-memory size serves every W
  p->part = t.merge_fanin ? t.merge_fanin : 2048u;
  if (!pow2(p->part) || p->part < 256 || p->part > 4096) return false;
  if (2ull * p->part * 12 > 200 * 1024) return false;  // merge CTA shared memory (one-key partitions)
  if (p->part > 2 * p->tile) p->part = 2 * p->tile;  // a partition never spans two run pairs
  if (p->alg == BSORT_ODD_EVEN) {
    p->cross = 0xFFFFFFFFu;  // every tile by odd-even transposition
  } else {
    p->cross = t.oddeven_cross ? t.oddeven_cross : kDefaultCross;
    if (p->cross > p->tile) return false;
  }
  return true;
}

namespace {

bool resolve(bsort_alg alg, const bsort_tune* tune, uint32_t W, SortParams* p) {
  return resolve_params(alg, tune, W, p);
}

}  // namespace

extern "C" {

size_t bsort_workspace_size(uint64_t max_words, uint32_t W, bsort_alg alg) {
  (void)alg;
  if (!valid_W(W) || max_words > 0xFFFFFFFEull) return 0;
  return ws_layout(max_words, W).total;
}

uint64_t bsort_workspace_capacity(size_t ws_bytes, uint32_t W) {
  if (!valid_W(W)) return 0;
  return ws_capacity(ws_bytes, W);
}

bsort_status bsort_workspace_init(void* d_ws, size_t ws_bytes, cudaStream_t s) {
  if (!d_ws || !aligned(d_ws, 256) || ws_bytes < sizeof(WsHeader)) return BSORT_E_WORKSPACE;
  return cuda_status(cudaMemsetAsync(d_ws, 0, 4096, s));
}

bsort_status bsort_reset_status(void* d_ws, cudaStream_t s) {
  if (!d_ws || !aligned(d_ws, 256)) return BSORT_E_WORKSPACE;
  return cuda_status(cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s));
}

bsort_status bsort_get_status(const void* d_ws, cudaStream_t s) {
  if (!d_ws || !aligned(d_ws, 256)) return BSORT_E_WORKSPACE;
  uint32_t flags = 0;
  if (cudaMemcpyAsync(&flags, d_ws, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BSORT_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return BSORT_E_CUDA;
  for (int c = 1; c < 32; ++c)
    if (flags & (1u << c)) return static_cast<bsort_status>(c);
  return BSORT_OK;
}

bsort_status bsort_set_wait_limit(uint32_t polls) {
  g_first_wait_polls.store(polls == BSORT_WAIT_DEFAULT ? kSpinLimit : polls,
                           std::memory_order_relaxed);
  return BSORT_OK;
}

const char* bsort_status_string(bsort_status st) {
  switch (st) {
    case BSORT_OK: return "ok";
    case BSORT_E_INVALID: return "invalid argument";
    case BSORT_E_WORD_TOO_LONG: return "word longer than the record width";
    case BSORT_E_CAPACITY: return "more words than the capacity";
    case BSORT_E_WORKSPACE: return "workspace missing, misaligned or too small";
    case BSORT_E_CUDA: return "CUDA error";
    case BSORT_E_TIMEOUT: return "device-side wait timed out";
    case BSORT_E_NOMEM: return "not enough device memory";
  }
  return "unknown status";
}

bsort_status bsort_tokenize(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                            uint32_t max_words, uint8_t* d_rec, uint8_t* d_len,
                            uint32_t* d_src_off, uint32_t* d_n_words, void* d_ws,
                            size_t ws_bytes, cudaStream_t s) {
  if (!valid_W(W) || n_bytes > 0xFFFF0000ull || (n_bytes && !d_text)) return BSORT_E_INVALID;
  if (max_words > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (max_words && (!d_rec || !d_len || !d_src_off || !aligned(d_rec, 16))) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, 0)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  return cuda_status(launch_tokenize(d_text, static_cast<uint32_t>(n_bytes), W, max_words, d_rec,
                                     d_len, d_src_off, d_n_words, ws, s));
}

bsort_status bsort_bucket_by_length(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                    uint32_t W, uint32_t* d_off, void* d_ws, size_t ws_bytes,
                                    cudaStream_t s) {
  if (!valid_W(W) || !d_off || n > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (n && (!d_rec || !d_len || !aligned(d_rec, 16))) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, n)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  return cuda_status(launch_bucket(d_rec, d_len, n, nullptr, W, d_off, ws, s));
}

bsort_status bsort_sort_buckets(uint32_t n, uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                const uint32_t* d_off, void* d_ws, size_t ws_bytes,
                                cudaStream_t s) {
  if (!valid_W(W) || !d_off || n > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (alg != BSORT_ODD_EVEN && alg != BSORT_MERGE && alg != BSORT_AUTO) return BSORT_E_INVALID;
  SortParams p;
  if (!resolve(alg, tune, W, &p)) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, n)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  return cuda_status(launch_sort(n, W, p, d_off, ws, s));
}

bsort_status bsort_gather(uint32_t n, uint32_t W, const uint32_t* d_off, const void* d_ws,
                          size_t ws_bytes, uint8_t* d_out_rec, uint32_t* d_out_perm,
                          cudaStream_t s) {
  if (!valid_W(W) || !d_off || n > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (n && (!d_out_rec || !d_out_perm || !aligned(d_out_rec, 16))) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, n)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  return cuda_status(launch_gather(n, nullptr, W, d_off, ws, d_out_rec, d_out_perm, s));
}

}  // extern "C"

namespace {

// The one-call paths, with the bucket offsets at d_off; whole = true adds the
// merge of the buckets into the unbucketed order.  With pk the final write
// packs the words (bucketed order only; d_out_rec is then unused).
bsort_status sort_records_impl(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n, uint32_t W,
                               bsort_alg alg, const bsort_tune* tune, uint8_t* d_out_rec,
                               uint32_t* d_out_perm, uint32_t* d_off, void* d_ws, size_t ws_bytes,
                               bool whole, cudaStream_t s, const PackOut* pk = nullptr) {
  if (!valid_W(W) || !d_off || n > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (n && (!d_rec || !d_len || (!pk && !d_out_rec) || !d_out_perm)) return BSORT_E_INVALID;
  if (n && (!aligned(d_rec, 16) || (!pk && !aligned(d_out_rec, 16)))) return BSORT_E_INVALID;
  if (alg != BSORT_ODD_EVEN && alg != BSORT_MERGE && alg != BSORT_AUTO) return BSORT_E_INVALID;
  SortParams p;
  if (!resolve(alg, tune, W, &p)) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, n)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  if (cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) != cudaSuccess) return BSORT_E_CUDA;
  cudaError_t e;
  if (alg == BSORT_AUTO && auto_applies(n, ws, W)) {
    e = launch_auto(d_rec, d_len, n, nullptr, W, d_off, ws, d_out_rec, d_out_perm, s, pk);
  } else {
    e = launch_bucket(d_rec, d_len, n, nullptr, W, d_off, ws, s);
    if (e == cudaSuccess) e = launch_sort(n, W, p, d_off, ws, s);
    if (e == cudaSuccess) e = launch_gather(n, nullptr, W, d_off, ws, d_out_rec, d_out_perm, s, pk);
  }
  if (e == cudaSuccess && whole) e = launch_whole(n, W, d_off, ws, d_out_rec, d_out_perm, s);
  return cuda_status(e);
}

bsort_status sort_text_impl(const uint8_t* d_text, uint64_t n_bytes, uint32_t W, uint32_t max_words,
                            bsort_alg alg, const bsort_tune* tune, uint8_t* d_rec, uint8_t* d_len,
                            uint32_t* d_src_off, uint32_t* d_n_words, uint8_t* d_out_rec,
                            uint32_t* d_out_perm, uint32_t* d_off, void* d_ws, size_t ws_bytes,
                            bool whole, cudaStream_t s, const PackOut* pk = nullptr) {
  if (!valid_W(W) || n_bytes > 0xFFFF0000ull || (n_bytes && !d_text) || !d_off || !d_n_words)
    return BSORT_E_INVALID;
  if (max_words > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (max_words && (!d_rec || !d_len || !d_src_off || (!pk && !d_out_rec) || !d_out_perm))
    return BSORT_E_INVALID;
  if (max_words && (!aligned(d_rec, 16) || (!pk && !aligned(d_out_rec, 16)))) return BSORT_E_INVALID;
  if (alg != BSORT_ODD_EVEN && alg != BSORT_MERGE && alg != BSORT_AUTO) return BSORT_E_INVALID;
  SortParams p;
  if (!resolve(alg, tune, W, &p)) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, max_words)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  if (cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) != cudaSuccess) return BSORT_E_CUDA;
  cudaError_t e = launch_tokenize(d_text, static_cast<uint32_t>(n_bytes), W, max_words, d_rec,
                                  d_len, d_src_off, d_n_words, ws, s);
  if (e == cudaSuccess && alg == BSORT_AUTO && auto_applies(max_words, ws, W)) {
    e = launch_auto(d_rec, d_len, max_words, d_n_words, W, d_off, ws, d_out_rec, d_out_perm, s, pk);
  } else {
    if (e == cudaSuccess) e = launch_bucket(d_rec, d_len, max_words, d_n_words, W, d_off, ws, s);
    if (e == cudaSuccess) e = launch_sort(max_words, W, p, d_off, ws, s);
    if (e == cudaSuccess)
      e = launch_gather(max_words, d_n_words, W, d_off, ws, d_out_rec, d_out_perm, s, pk);
  }
  if (e == cudaSuccess && whole) e = launch_whole(max_words, W, d_off, ws, d_out_rec, d_out_perm, s);
  return cuda_status(e);
}

// Bucket offsets of the unbucketed calls live in the workspace.
uint32_t* internal_off(void* d_ws, size_t ws_bytes, uint32_t W) {
  if (!valid_W(W) || !d_ws || !aligned(d_ws, 256)) return nullptr;
  return ws_view(d_ws, ws_bytes, W).misc;
}

// Arguments of the packed calls: n words at most (n_max), bytes[cap].
bsort_status packed_args(uint32_t n_max, uint32_t W, uint8_t* d_bytes, uint64_t bytes_cap,
                         uint32_t* d_offsets, PackOut* pk) {
  if (!valid_W(W) || !d_offsets) return BSORT_E_INVALID;
  if (n_max > pack_max_words() || static_cast<uint64_t>(n_max) * W > 0xFFFFFFFFull)
    return BSORT_E_CAPACITY;
  if (n_max && !d_bytes) return BSORT_E_INVALID;
  *pk = PackOut{d_bytes, d_offsets, bytes_cap};
  return BSORT_OK;
}

}  // namespace

extern "C" {

bsort_status bsort_sort_records(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                uint8_t* d_out_rec, uint32_t* d_out_perm, uint32_t* d_off,
                                void* d_ws, size_t ws_bytes, cudaStream_t s) {
  return sort_records_impl(d_rec, d_len, n, W, alg, tune, d_out_rec, d_out_perm, d_off, d_ws,
                           ws_bytes, false, s);
}

bsort_status bsort_sort_text(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                             uint32_t max_words, bsort_alg alg, const bsort_tune* tune,
                             uint8_t* d_rec, uint8_t* d_len, uint32_t* d_src_off,
                             uint32_t* d_n_words, uint8_t* d_out_rec, uint32_t* d_out_perm,
                             uint32_t* d_off, void* d_ws, size_t ws_bytes, cudaStream_t s) {
  return sort_text_impl(d_text, n_bytes, W, max_words, alg, tune, d_rec, d_len, d_src_off,
                        d_n_words, d_out_rec, d_out_perm, d_off, d_ws, ws_bytes, false, s);
}

bsort_status bsort_sort_records_whole(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                      uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                      uint8_t* d_out_rec, uint32_t* d_out_perm, void* d_ws,
                                      size_t ws_bytes, cudaStream_t s) {
  uint32_t* off = internal_off(d_ws, ws_bytes, W);
  if (!off) return valid_W(W) ? BSORT_E_WORKSPACE : BSORT_E_INVALID;
  return sort_records_impl(d_rec, d_len, n, W, alg, tune, d_out_rec, d_out_perm, off, d_ws,
                           ws_bytes, true, s);
}

bsort_status bsort_sort_text_whole(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                                   uint32_t max_words, bsort_alg alg, const bsort_tune* tune,
                                   uint8_t* d_rec, uint8_t* d_len, uint32_t* d_src_off,
                                   uint32_t* d_n_words, uint8_t* d_out_rec, uint32_t* d_out_perm,
                                   void* d_ws, size_t ws_bytes, cudaStream_t s) {
  uint32_t* off = internal_off(d_ws, ws_bytes, W);
  if (!off) return valid_W(W) ? BSORT_E_WORKSPACE : BSORT_E_INVALID;
  return sort_text_impl(d_text, n_bytes, W, max_words, alg, tune, d_rec, d_len, d_src_off,
                        d_n_words, d_out_rec, d_out_perm, off, d_ws, ws_bytes, true, s);
}

bsort_status bsort_sort_records_packed(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                       uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                       uint8_t* d_bytes, uint64_t bytes_cap, uint32_t* d_offsets,
                                       uint32_t* d_out_perm, uint32_t* d_off, void* d_ws,
                                       size_t ws_bytes, cudaStream_t s) {
  PackOut pk;
  if (const bsort_status e = packed_args(n, W, d_bytes, bytes_cap, d_offsets, &pk)) return e;
  return sort_records_impl(d_rec, d_len, n, W, alg, tune, nullptr, d_out_perm, d_off, d_ws,
                           ws_bytes, false, s, &pk);
}

bsort_status bsort_sort_text_packed(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                                    uint32_t max_words, bsort_alg alg, const bsort_tune* tune,
                                    uint8_t* d_rec, uint8_t* d_len, uint32_t* d_src_off,
                                    uint32_t* d_n_words, uint8_t* d_bytes, uint64_t bytes_cap,
                                    uint32_t* d_offsets, uint32_t* d_out_perm, uint32_t* d_off,
                                    void* d_ws, size_t ws_bytes, cudaStream_t s) {
  PackOut pk;
  if (const bsort_status e = packed_args(max_words, W, d_bytes, bytes_cap, d_offsets, &pk)) return e;
  return sort_text_impl(d_text, n_bytes, W, max_words, alg, tune, d_rec, d_len, d_src_off,
                        d_n_words, nullptr, d_out_perm, d_off, d_ws, ws_bytes, false, s, &pk);
}

bsort_status bsort_pack_words(uint32_t n, uint32_t W, const uint8_t* d_rec, const uint32_t* d_off,
                              const uint32_t* d_perm, const uint8_t* d_len, uint8_t* d_bytes,
                              uint64_t bytes_cap, uint32_t* d_offsets, void* d_ws,
                              size_t ws_bytes, cudaStream_t s) {
  if (!valid_W(W) || !d_offsets) return BSORT_E_INVALID;
  if (n > pack_max_words() || static_cast<uint64_t>(n) * W > 0xFFFFFFFFull) return BSORT_E_CAPACITY;
  if (n && (!d_rec || !aligned(d_rec, 16) || !d_bytes)) return BSORT_E_INVALID;
  if (n && !d_off && (!d_perm || !d_len)) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, 0)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  return cuda_status(launch_pack(n, W, d_rec, d_off, d_perm, d_len, d_bytes, bytes_cap, d_offsets,
                                 ws, s));
}

size_t bsort_sort_many_workspace_size(uint64_t total_words, uint32_t n_lists, uint32_t W) {
  if (!valid_W(W) || total_words > 0xFFFFFFF0ull) return 0;
  return many_workspace_size(total_words, n_lists, W);
}

bsort_status bsort_sort_many(const uint8_t* d_text_or_rec, const uint8_t* d_len,
                             const bsort_list* d_lists, uint32_t n_lists, uint32_t W,
                             int lists_are_text, uint32_t max_list_words, bsort_alg alg,
                             const bsort_tune* tune, uint8_t* d_out_rec, uint32_t* d_out_perm,
                             uint32_t* d_out_off, int32_t* d_list_status, void* d_ws,
                             size_t ws_bytes, cudaStream_t s) {
  if (!valid_W(W)) return BSORT_E_INVALID;
  if (n_lists == 0) return BSORT_OK;
  if (!d_lists || !d_out_off || !d_list_status || !d_out_rec || !d_out_perm || !d_text_or_rec)
    return BSORT_E_INVALID;
  if (lists_are_text ? d_len != nullptr : d_len == nullptr) return BSORT_E_INVALID;
  if (!aligned(d_out_rec, 16) || (!lists_are_text && !aligned(d_text_or_rec, 16)))
    return BSORT_E_INVALID;
  if (alg != BSORT_ODD_EVEN && alg != BSORT_MERGE && alg != BSORT_AUTO) return BSORT_E_INVALID;
  if (max_list_words == 0) return BSORT_E_INVALID;
  SortParams p;
  if (!resolve(alg, tune, W, &p)) return BSORT_E_INVALID;
  if (!d_ws || !aligned(d_ws, 256) || many_capacity(ws_bytes, W, n_lists) == 0)
    return BSORT_E_WORKSPACE;
  return cuda_status(launch_many(d_text_or_rec, d_len, d_lists, n_lists, W, lists_are_text != 0,
                                 max_list_words, p, d_out_off, d_out_rec, d_out_perm,
                                 d_list_status, d_ws, ws_bytes, s));
}

bsort_status bsort_export_buckets(uint32_t n, uint32_t W, const uint32_t* d_off,
                                  const void* d_ws, size_t ws_bytes, uint64_t* d_keys,
                                  uint32_t* d_idx, cudaStream_t s) {
  if (!valid_W(W) || !d_off || n > 0xFFFFFFFEu) return BSORT_E_INVALID;
  if (n && (!d_keys || !d_idx)) return BSORT_E_INVALID;
  if (const bsort_status e = check_ws(d_ws, ws_bytes, W, n)) return e;
  const Ws ws = ws_view(d_ws, ws_bytes, W);
  return cuda_status(launch_export(n, W, d_off, ws, d_keys, d_idx, s));
}

}  // extern "C"
