// Phase 2 of the method (§3 Methodology, "Pre-processing", second phase, and
// the abstract: sub-arrays by character count, each sized by the number of
// words of that length, shorter lengths first).
//
//   hist_kernel     per-block length histogram: each warp aggregates equal
//                   lengths with __match_any_sync, one shared-memory counter
//                   row per warp, then a block reduction -> table[L][b]
//   scan_kernel     exclusive scan of the L-major table (chunks read and
//                   written coalesced through shared memory): base[L][b] is the
//                   first output slot of block b's words of length L
//   off_kernel      bucket offsets off[L] = base[L][0], off[W+1] = n
//   scatter_kernel  stable scatter: word i goes to base[L][b] + (number of
//                   earlier words of length L in block b); its letters are
//                   packed into ceil(L/8) big-endian uint64 keys
#include "block_scan.cuh"
#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kWarps = kThreads / 32;
constexpr uint32_t kItems = 4;  // words per lane per scatter iteration

__device__ __forceinline__ uint32_t word_count(uint32_t n_cap, const uint32_t* d_n) {
  return d_n ? min(*d_n, n_cap) : n_cap;
}

__global__ void __launch_bounds__(kThreads)
hist_kernel(const uint8_t* __restrict__ len, uint32_t n_cap, const uint32_t* __restrict__ d_n,
            uint32_t W, uint32_t wpb, uint32_t G, uint32_t* __restrict__ table, WsHeader* hdr) {
  __shared__ uint32_t cnt[kWarps][kBins];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  for (uint32_t i = threadIdx.x; i < kWarps * kBins; i += kThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t n = word_count(n_cap, d_n);
  const uint32_t start = blockIdx.x * wpb;
  const uint32_t end = min(n, start + wpb);
  bool bad_zero = false, bad_long = false;
  for (uint32_t b = start; b < end; b += kThreads) {
    const uint32_t i = b + threadIdx.x;
    uint32_t L = i < end ? len[i] : 0u;
    if (i < end) {
      bad_zero |= L == 0;
      bad_long |= L > W;
    }
    if (L > W) L = 0;  // bin 0 collects nothing: invalid words are left out
    const uint32_t peers = __match_any_sync(0xffffffffu, L);
    if (L != 0 && lane == __ffs(peers) - 1) cnt[warp][L] += __popc(peers);
  }
  __syncthreads();
  for (uint32_t L = threadIdx.x; L <= W; L += kThreads) {
    uint32_t s = 0;
#pragma unroll
    for (uint32_t w = 0; w < kWarps; ++w) s += cnt[w][L];
    table[L * G + blockIdx.x] = s;
  }
  if (bad_zero) set_error(hdr, BSORT_E_INVALID);
  if (bad_long) set_error(hdr, BSORT_E_WORD_TOO_LONG);
}

__global__ void off_kernel(const uint32_t* __restrict__ table, const uint32_t* __restrict__ total,
                           uint32_t W, uint32_t G, uint32_t* __restrict__ off, WsHeader* hdr) {
  const uint32_t L = threadIdx.x;
  if (L <= W) off[L] = L == 0 ? 0u : table[L * G];
  if (L == W + 1) off[L] = *total;
  if (L < kMaxW + 2) hdr->final_buf[L] = 0;
}

__global__ void __launch_bounds__(kThreads)
scatter_kernel(const uint8_t* __restrict__ rec, const uint8_t* __restrict__ len, uint32_t n_cap,
               const uint32_t* __restrict__ d_n, uint32_t W, uint32_t wpb, uint32_t G,
               const uint32_t* __restrict__ base_tab, Ws ws) {
  __shared__ uint32_t cursor[kBins];
  __shared__ uint32_t wcnt[kWarps][kBins];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t n = word_count(n_cap, d_n);
  const uint32_t start = blockIdx.x * wpb;
  const uint32_t end = min(n, start + wpb);
  if (threadIdx.x <= W) cursor[threadIdx.x] = base_tab[threadIdx.x * G + blockIdx.x];
  for (uint32_t c = start; c < end; c += kThreads * kItems) {
    for (uint32_t i = lane; i < kBins; i += 32) wcnt[warp][i] = 0;
    __syncwarp();
    uint32_t Ls[kItems], rank[kItems];
    // warp `warp` owns words [c + warp*32*kItems, +32*kItems), kItems steps of
    // 32; the lengths, then the record words, are all loaded before the
    // ranking, so the loads are in flight together
    uint64_t words[kItems][kMaxW / 8];
#pragma unroll
    for (uint32_t it = 0; it < kItems; ++it) {
      const uint32_t i = c + warp * 32 * kItems + it * 32 + lane;
      const uint32_t L = i < end ? len[i] : 0u;
      Ls[it] = L > W ? 0u : L;
    }
#pragma unroll
    for (uint32_t it = 0; it < kItems; ++it) {
      const uint32_t i = c + warp * 32 * kItems + it * 32 + lane;
      const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + static_cast<uint64_t>(i) * W);
      const uint32_t K = Ls[it] ? keys_for_len(Ls[it]) : 0u;
#pragma unroll
      for (uint32_t k = 0; k < kMaxW / 8; ++k) words[it][k] = k < K ? __ldg(src + k) : 0ull;
    }
#pragma unroll
    for (uint32_t it = 0; it < kItems; ++it) {
      const uint32_t L = Ls[it];
      const uint32_t peers = __match_any_sync(0xffffffffu, L);
      rank[it] = wcnt[warp][L] + __popc(peers & lanemask_lt());
      __syncwarp();
      if (lane == __ffs(peers) - 1) wcnt[warp][L] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x <= W) {
      uint32_t run = cursor[threadIdx.x];
#pragma unroll
      for (uint32_t w = 0; w < kWarps; ++w) {
        const uint32_t t = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = run;
        run += t;
      }
      cursor[threadIdx.x] = run;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t it = 0; it < kItems; ++it) {
      const uint32_t L = Ls[it];
      if (L == 0) continue;
      const uint32_t i = c + warp * 32 * kItems + it * 32 + lane;
      const uint32_t pos = wcnt[warp][L] + rank[it];
      const uint32_t K = keys_for_len(L);
#pragma unroll
      for (uint32_t k = 0; k < kMaxW / 8; ++k)
        if (k < K) ws.keys[0][k * ws.cap + pos] = bswap64(words[it][k]) & key_mask(L, k);
      ws.idx[0][pos] = i;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024)
scan_kernel(uint32_t* data, uint32_t n, uint32_t* __restrict__ total) {
  block_scan_into(n, [&](uint32_t i) { return data[i]; }, data, total);
}

}  // namespace

HistGeom hist_geom(uint32_t n_cap) {
  uint64_t wpb = (static_cast<uint64_t>(n_cap) + kHistBlocksMax - 1) / kHistBlocksMax;
  if (wpb < 4096) wpb = 4096;
  wpb = (wpb + kThreads * kItems - 1) / (kThreads * kItems) * (kThreads * kItems);
  uint32_t G = static_cast<uint32_t>((static_cast<uint64_t>(n_cap) + wpb - 1) / wpb);
  if (G == 0) G = 1;
  return {static_cast<uint32_t>(wpb), G};
}

void launch_scan(uint32_t* data, uint32_t n, uint32_t* total, cudaStream_t s) {
  BSORT_LAUNCH("scan", scan_kernel, 1, 1024, 0, s, data, n, total);
}

cudaError_t launch_hist(const uint8_t* len, uint32_t n_cap, const uint32_t* d_n, uint32_t W,
                        uint32_t* d_off, const Ws& ws, cudaStream_t s) {
  const HistGeom g = hist_geom(n_cap);
  uint32_t* table = ws.table;
  uint32_t* total = ws.table + kBins * kHistBlocksMax;
  BSORT_LAUNCH("hist", hist_kernel, g.G, kThreads, 0, s, len, n_cap, d_n, W, g.wpb, g.G, table,
               ws.hdr);
  launch_scan(table, (W + 1) * g.G, total, s);
  BSORT_LAUNCH("offsets", off_kernel, 1, 64, 0, s, table, total, W, g.G, d_off, ws.hdr);
  return cudaGetLastError();
}

cudaError_t launch_bucket(const uint8_t* rec, const uint8_t* len, uint32_t n_cap,
                          const uint32_t* d_n, uint32_t W, uint32_t* d_off, const Ws& ws,
                          cudaStream_t s) {
  const HistGeom g = hist_geom(n_cap);
  uint32_t* table = ws.table;
  cudaError_t e = launch_hist(len, n_cap, d_n, W, d_off, ws, s);
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("scatter", scatter_kernel, g.G, kThreads, 0, s, rec, len, n_cap, d_n, W, g.wpb,
               g.G, table, ws);
  return cudaGetLastError();
}

}  // namespace bsort
