// Shared device helpers and the workspace layout of the bsort library.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "bsort.h"

namespace bsort {

constexpr uint32_t kMaxW = 32;          // widest record (bytes)
constexpr uint32_t kMaxK = kMaxW / 8;   // most uint64 key words per word
constexpr uint32_t kBins = kMaxW + 1;   // length bins 0..W (0 stays empty)
constexpr uint32_t kHistBlocksMax = 2048;  // blocks of the histogram / scatter grid
constexpr uint32_t kTextBlocksMax = 4096;  // blocks of the tokeniser grid
constexpr uint32_t kScanThreads = 1024;
constexpr uint32_t kSpinLimit = 1u << 26;  // bound on every device-side wait loop

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
// [header 4 KB][block table][keys A][keys B][idx A][idx B][misc]
// keys X: kK planes of `cap` uint64 (plane k at k*cap); idx X: `cap` uint32.
// Bucket L occupies positions off[L]..off[L+1]-1 of every plane.
struct WsHeader {
  uint32_t status_flags;            // bit c set: error code c was seen
  uint32_t n_words;                 // device-side word count of the last tokenise
  uint32_t final_buf[kMaxW + 2];    // per bucket: 0 = sorted data in A, 1 = in B
  uint32_t tile;                    // tile size used by the last sort
  uint32_t magic;
  uint32_t counters[16];            // work-queue counters of persistent kernels
};
static_assert(sizeof(WsHeader) <= 4096, "header too large");

constexpr uint32_t kWsMagic = 0x42534f52u;

struct WsLayout {
  size_t header, table, keys_a, keys_b, keys_c, idx_a, idx_b, idx_c, misc, splits, autoa, total;
  uint64_t cap;       // element capacity of each plane (>= max_words + 64)
  uint32_t K;         // key planes
};

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---- sample-sort (AUTO) constants --------------------------------------
// Per key count K (1..4): shared-memory segment capacity, expected segment
// size, and the most samples one bucket keeps for choosing its splitters.
__host__ __device__ constexpr uint32_t auto_seg_cap(uint32_t K) {
  return K <= 1 ? 8192u : K == 2 ? 4096u : 2048u;
}
__host__ __device__ constexpr uint32_t auto_target(uint32_t K) {
  return auto_seg_cap(K) / 3;  // regions hold 3x the expected count
}
__host__ __device__ constexpr uint32_t auto_sample_max(uint32_t K) {
  return K <= 1 ? 16384u : K == 2 ? 8192u : 4096u;
}
constexpr uint32_t kAutoSampleEvery = 32;      // one stratified sample position per 32 words
constexpr uint32_t kAutoMinWords = 65536;      // smaller inputs take the merge path
constexpr uint64_t kAutoSlack = 1u << 18;      // extra elements of the third region
// splitter directory per bucket: (kAutoDir2Max + 1) u16 entries, enough for
// two-byte codes of mixed-case letters (65 byte classes)
constexpr uint32_t kAutoDir2Max = 65 * 65;
constexpr uint32_t kAutoDirBytes = 8464;

__host__ __device__ constexpr uint32_t auto_sample_cap(uint32_t K, uint64_t cap) {
  return static_cast<uint32_t>(
      ((auto_sample_max(K) < (cap / 64 < 256 ? 256 : cap / 64)) ? auto_sample_max(K)
                                                                 : (cap / 64 < 256 ? 256 : cap / 64)) /
      64 * 64);
}
// Per-segment byte code record of the sample sort: 16 position fields (lo |
// offset << 8 | width << 16), the code width, the index width and the
// one-key shape (packed smallest bytes, two words; p0, w0, wl, n).
constexpr uint32_t kSegFWords = 21;
__host__ __device__ constexpr uint64_t auto_max_segments(uint64_t cap) {
  return cap / 1024 + 2 * kBins + 1;
}
constexpr size_t auto_bytes(uint64_t cap, uint32_t W) {
  size_t samples = 0;
  for (uint32_t L = 1; L <= W; ++L) {
    const uint32_t K = (L + 7) / 8;
    samples += static_cast<size_t>(auto_sample_cap(K, cap)) * (8 * K + 4);
  }
  // splitters (8 KW + 4), cursors (one 128-byte line each), four u32 and two
  // u64 tables and the 18-word byte code record per segment
  const size_t tables = auto_max_segments(cap) * (8 * (W / 8) + 4 + 128 + 4 * 4 + 8 * 2 + 4 * kSegFWords);
  // staging planes of the length buckets (keys, indices), in workspaces the
  // sample sort runs in
  const size_t stage = cap >= kAutoMinWords + 64 ? (cap + 64) * (8 * (W / 8) + 4) : 0;
  return align_up(4096 + samples + tables + (16 + kAutoDirBytes) * kBins + 4096 + stage + 512, 256);
}

// Layout for a plane capacity of `cap` elements (a multiple of 64).
constexpr WsLayout ws_layout_cap(uint64_t cap, uint32_t W) {
  WsLayout l{};
  l.K = W / 8;
  l.cap = cap;
  size_t o = 0;
  l.header = o;
  o += 4096;
  l.table = o;
  o += align_up(sizeof(uint32_t) * static_cast<size_t>(kBins) * kHistBlocksMax * 2 + 64 * 1024, 256);
  l.keys_a = o;
  o += align_up(8 * l.cap * l.K, 256);
  l.keys_b = o;
  o += align_up(8 * l.cap * l.K, 256);
  // third region: sample-sort room, only in workspaces large enough for it
  const uint64_t third = cap >= kAutoMinWords + 64 ? cap + kAutoSlack : 0;
  l.keys_c = o;
  o += align_up(8 * third * l.K, 256);
  l.idx_a = o;
  o += align_up(4 * l.cap, 256);
  l.idx_b = o;
  o += align_up(4 * l.cap, 256);
  l.idx_c = o;
  o += align_up(4 * third, 256);
  l.misc = o;
  o += 64 * 1024;
  // merge-path splits of one merge pass: one per partition, partitions of at
  // least 64 elements (the smallest partition of the widest words) plus a
  // partial one per bucket
  l.splits = o;
  o += align_up(4 * (cap / 64 + 2 * static_cast<size_t>(kBins) + 1), 256);
  l.autoa = o;
  o += auto_bytes(cap, W);
  l.total = o;
  return l;
}

// Smallest layout holding max_words words (64 elements of slack per plane).
constexpr WsLayout ws_layout(uint64_t max_words, uint32_t W) {
  return ws_layout_cap(align_up(max_words + 64, 64), W);
}

// The layout is a pure function of (ws_bytes, W): the largest capacity that
// fits, so every call on the same workspace agrees on where things live.
inline WsLayout ws_layout_bytes(size_t ws_bytes, uint32_t W) {
  const uint32_t K = W / 8;
  const size_t fixed = ws_layout_cap(0, W).total;
  if (ws_bytes <= fixed) return ws_layout_cap(0, W);
  // total(cap) is increasing in cap: binary search the largest cap (a multiple of 64) that fits
  uint64_t lo = 0, hi = (ws_bytes - fixed) / (16ull * K + 8ull) / 64 + 1;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;
    if (ws_layout_cap(mid * 64, W).total <= ws_bytes) lo = mid;
    else hi = mid - 1;
  }
  return ws_layout_cap(lo * 64, W);
}

// Words a workspace of ws_bytes can hold.
inline uint64_t ws_capacity(size_t ws_bytes, uint32_t W) {
  const uint64_t cap = ws_layout_bytes(ws_bytes, W).cap;
  return cap > 64 ? cap - 64 : 0;
}

// Polls of the first wait for a bulk copy before it gives up (host side; set
// by bsort_set_wait_limit, read when a call is issued).
uint32_t first_wait_polls();

// Device-side view of the workspace.
struct Ws {
  WsHeader* hdr;
  uint32_t* table;
  uint8_t* autoa;     // sample-sort area (samples, splitters, segment tables)
  uint32_t* misc;     // 64 KB of small per-call state (e.g. internal bucket offsets)
  uint32_t* splits;   // merge-path splits of the current merge pass, one per partition
  uint64_t* keys[2];
  uint32_t* idx[2];
  uint64_t cap;
  uint32_t K;
  uint32_t wait_polls;  // bound of the first wait for a bulk copy (drains use kSpinLimit)
};

inline Ws ws_view(const void* base, size_t ws_bytes, uint32_t W) {
  WsLayout l = ws_layout_bytes(ws_bytes, W);
  char* b = static_cast<char*>(const_cast<void*>(base));
  Ws w;
  w.hdr = reinterpret_cast<WsHeader*>(b + l.header);
  w.table = reinterpret_cast<uint32_t*>(b + l.table);
  w.keys[0] = reinterpret_cast<uint64_t*>(b + l.keys_a);
  w.keys[1] = reinterpret_cast<uint64_t*>(b + l.keys_b);
  w.idx[0] = reinterpret_cast<uint32_t*>(b + l.idx_a);
  w.idx[1] = reinterpret_cast<uint32_t*>(b + l.idx_b);
  w.autoa = reinterpret_cast<uint8_t*>(b + l.autoa);
  w.misc = reinterpret_cast<uint32_t*>(b + l.misc);
  w.splits = reinterpret_cast<uint32_t*>(b + l.splits);
  w.cap = l.cap;
  w.K = l.K;
  w.wait_polls = first_wait_polls();
  return w;
}

// Devices a process may drive; per-device host caches hold this many entries.
constexpr int kMaxDevices = 64;

// The dynamic shared-memory limit already set for one kernel, per device.
// cudaFuncSetAttribute acts on the current device only, so a process that
// launches on several devices must opt in on each; the entries are atomics,
// so host threads may launch concurrently.  Static storage starts at zero.
struct SmemOptIn {
  std::atomic<size_t> cur[kMaxDevices];
};

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (host).
template <typename Kernel>
inline cudaError_t ensure_smem(Kernel k, size_t bytes, SmemOptIn* o) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // always opt in: static shared memory counts against the 48 KB default too
  if (bytes <= o->cur[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e != cudaSuccess) return e;
  size_t c = o->cur[dev].load(std::memory_order_relaxed);
  while (c < bytes && !o->cur[dev].compare_exchange_weak(c, bytes, std::memory_order_release)) {
  }
  return cudaSuccess;
}

// Streaming multiprocessors of the current device (cached per device).
inline int device_sm_count() {
  static std::atomic<int> sms[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 148;
  int n = sms[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 148;
  sms[dev].store(n, std::memory_order_relaxed);
  return n;
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_error(WsHeader* h, int code) {
  atomicOr(&h->status_flags, 1u << code);
}

__device__ __forceinline__ bool is_letter(uint32_t b) {
  return ((b | 0x20u) - 'a') < 26u;
}

// Byte-reverses a uint64 so that the first byte in memory becomes the most
// significant: integer order of the result is lexicographic byte order.
__device__ __forceinline__ uint64_t bswap64(uint64_t x) {
  uint32_t lo = static_cast<uint32_t>(x), hi = static_cast<uint32_t>(x >> 32);
  uint32_t nlo = __byte_perm(hi, 0, 0x0123), nhi = __byte_perm(lo, 0, 0x0123);
  return (static_cast<uint64_t>(nhi) << 32) | nlo;
}

// Big-endian key word k of a word of length L: keeps its bytes 8k..min(L,8k+8)-1.
__device__ __forceinline__ uint64_t key_mask(uint32_t L, uint32_t k) {
  int c = static_cast<int>(L) - static_cast<int>(8 * k);
  if (c <= 0) return 0ull;
  if (c >= 8) return ~0ull;
  return ~0ull << (64 - 8 * c);
}

__device__ __forceinline__ uint32_t keys_for_len(uint32_t L) { return (L + 7) >> 3; }

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Element of a bucket: K key words then the input index; a strict total order.
template <int K>
struct Elem {
  uint64_t k[K];
  uint32_t idx;
};

template <int K>
__device__ __forceinline__ bool elem_less(const Elem<K>& a, const Elem<K>& b) {
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (a.k[i] != b.k[i]) return a.k[i] < b.k[i];
  return a.idx < b.idx;
}

// Packed output of the bucketed order (§3.1, "vectors of string"): every word
// of bucket L is L bytes long, so word r of bucket L starts at byte
// P_L + (r - off[L]) L, P_L being the bytes of all shorter words.  Writes
// base[L] = P_L - off[L] L (mod 2^32) for L = 1..W, so that the start is
// base[L] + r L, and base[W + 1] = the total, which it returns.  With
// n W < 2^32 every start and the total fit 32 bits.  One thread.
__device__ __forceinline__ uint32_t packed_bases(const uint32_t* off, uint32_t W, uint32_t* base) {
  uint32_t p = 0;
  for (uint32_t L = 1; L <= W; ++L) {
    const uint32_t lo = off[L], hi = off[L + 1];
    base[L] = p - lo * L;
    p += (hi - lo) * L;
  }
  base[W + 1] = p;
  return p;
}

// The L bytes of a word (key words k[0..K-1], big-endian, K = ceil(L / 8)) to
// dst, any alignment.
template <int K>
__device__ __forceinline__ void put_word_bytes(uint8_t* dst, uint32_t L, const uint64_t (&k)[K]) {
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const uint32_t m = min(8u, L - 8u * q);
    for (uint32_t j = 0; j < m; ++j) dst[8 * q + j] = static_cast<uint8_t>(k[q] >> (56 - 8 * j));
  }
}

// Shared-memory structure-of-arrays tile: planes of keys then idx.
template <int K>
struct SmemTile {
  uint64_t* k[K];
  uint32_t* idx;
  __device__ __forceinline__ Elem<K> get(uint32_t i) const {
    Elem<K> e;
#pragma unroll
    for (int j = 0; j < K; ++j) e.k[j] = k[j][i];
    e.idx = idx[i];
    return e;
  }
  __device__ __forceinline__ void put(uint32_t i, const Elem<K>& e) const {
#pragma unroll
    for (int j = 0; j < K; ++j) k[j][i] = e.k[j];
    idx[i] = e.idx;
  }
};

template <int K>
__device__ __forceinline__ Elem<K> load_elem(const Ws& ws, int buf, uint64_t pos) {
  Elem<K> e;
#pragma unroll
  for (int j = 0; j < K; ++j) e.k[j] = ws.keys[buf][j * ws.cap + pos];
  e.idx = ws.idx[buf][pos];
  return e;
}

template <int K>
__device__ __forceinline__ void store_elem(const Ws& ws, int buf, uint64_t pos, const Elem<K>& e) {
#pragma unroll
  for (int j = 0; j < K; ++j) ws.keys[buf][j * ws.cap + pos] = e.k[j];
  ws.idx[buf][pos] = e.idx;
}

// ---------------------------------------------------------------------------
// Bulk-copy (TMA engine) staging of global ranges into shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 1-D bulk copy global -> shared; dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier; gives up after `polls` polls
// (kSpinLimit by default; 0 gives up at once).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t polls = kSpinLimit) {
  for (uint32_t it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace bsort
