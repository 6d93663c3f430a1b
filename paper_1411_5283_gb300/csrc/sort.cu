// Phase 3 of the method (§3 Methodology, "Pre-processing", third phase):
// every length bucket is sorted alphabetically.
//
// The paper sorts each sub-array with bubble sort (§2, §3.2) and, under MPI,
// has every process bubble-sort one chunk before the master merges the sorted
// chunks (§4 "MPI Implementation", §5).  The GPU form keeps that shape:
//   tile_sort_kernel   one CTA per tile of a bucket; the tile is staged into
//                      shared memory by the bulk-copy (TMA) engine and sorted
//                      by odd-even transposition (bubble sort's data-parallel
//                      form: alternate even / odd neighbour exchanges, stop
//                      after an even and an odd phase without exchange) or by
//                      a bitonic network;
//   merge_split_kernel the merge-path splits of a pass over long runs, one
//                      warp per partition, all at once;
//   merge_pass_kernel  merge-path merging of neighbouring sorted runs, run
//                      length doubling each pass, until each bucket is one run
//                      (a producer warp per CTA finds or reads the splits and
//                      stages the inputs by bulk copies, consumer warps merge).
// Elements are (key words..., input index); comparing the tuple is a strict
// total order, so every algorithm and tile size gives the same result.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "sort_impl.cuh"

namespace bsort {

namespace {

// Tiles of bucket L are numbered from the prefix sum of ceil(cnt_L / T) over
// shorter lengths.
__device__ TileRef find_tile(const uint32_t* s_off, uint32_t W, uint32_t T, uint32_t t) {
  TileRef r{0, 0, 0, false};
  uint32_t acc = 0;
  for (uint32_t L = 1; L <= W; ++L) {
    const uint32_t cnt = s_off[L + 1] - s_off[L];
    const uint32_t nt = (cnt + T - 1) / T;
    if (t < acc + nt) {
      r.L = L;
      r.start = s_off[L] + (t - acc) * T;
      r.len = min(T, s_off[L + 1] - r.start);
      r.valid = true;
      return r;
    }
    acc += nt;
  }
  return r;
}

// A bucket of at most `cross` words is sorted whole by odd-even
// transposition (it fits one tile); a larger one by bitonic tiles, merged
// afterwards.  cross = 0xFFFFFFFF makes every tile odd-even.
__global__ void __launch_bounds__(1024) tile_sort_kernel(const uint32_t* __restrict__ d_off, uint32_t W, uint32_t T,
                                 uint32_t cross, Ws ws) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_off[kMaxW + 2];
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x <= W + 1) {
    // record where each bucket's sorted run ends up after the merge passes
    const uint32_t L = threadIdx.x;
    const uint32_t cnt = (L >= 1 && L <= W) ? s_off[L + 1] - s_off[L] : 0u;
    ws.hdr->final_buf[L] = merge_passes(cnt, T) & 1u;
    if (L == 0) ws.hdr->tile = T;
  }
  const TileRef tr = find_tile(s_off, W, T, blockIdx.x);
  if (!tr.valid) return;
  uint8_t* sm = align128(smem);
  const bool odd_even = s_off[tr.L + 1] - s_off[tr.L] <= cross;
  switch (keys_for_len(tr.L)) {
    case 1: sort_one_tile<1>(sm, T, tr, odd_even, ws); break;
    case 2: sort_one_tile<2>(sm, T, tr, odd_even, ws); break;
    case 3: sort_one_tile<3>(sm, T, tr, odd_even, ws); break;
    default: sort_one_tile<4>(sm, T, tr, odd_even, ws); break;
  }
}

// Partitions of one merge pass over every bucket longer than R (prefix over
// the buckets in s_pre; thread 0 writes it).
__device__ void pass_partitions(const uint32_t* s_off, uint32_t W, uint32_t R, uint32_t part, uint32_t* s_pre) {
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t l = 0; l <= W + 1; ++l) {
      s_pre[l] = acc;
      if (l >= 1 && l <= W) {
        const uint32_t cnt = s_off[l + 1] - s_off[l], P = merge_part_for(part, keys_for_len(l));
        if (cnt > R) acc += (cnt + P - 1) / P;
      }
    }
  }
}

// The split of every partition of one merge pass, one warp per partition,
// all at once: splits[q] at partition q's first output.
__global__ void __launch_bounds__(256)
merge_split_kernel(const uint32_t* __restrict__ d_off, uint32_t W, uint32_t R, uint32_t part, int src,
                   Ws ws) {
  __shared__ uint32_t s_off[kMaxW + 2], s_pre[kMaxW + 2];
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  pass_partitions(s_off, W, R, part, s_pre);
  __syncthreads();
  const uint32_t total = s_pre[W + 1];
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); q < total; q += warps) {
    uint32_t L = 1;
    while (L < W && s_pre[L + 1] <= q) ++L;  // warp-uniform
    const uint32_t K = keys_for_len(L), P = merge_part_for(part, K);
    const uint32_t o0 = (q - s_pre[L]) * P, bstart = s_off[L], cnt = s_off[L + 1] - s_off[L];
    uint32_t* out = ws.splits + q;
    switch (K) {
      case 1: merge_split_warp<1>(bstart, cnt, R, o0, src, ws, out); break;
      case 2: merge_split_warp<2>(bstart, cnt, R, o0, src, ws, out); break;
      case 3: merge_split_warp<3>(bstart, cnt, R, o0, src, ws, out); break;
      default: merge_split_warp<4>(bstart, cnt, R, o0, src, ws, out); break;
    }
  }
}

// One merge pass over every bucket longer than R: output ranges of each
// bucket cut into partitions (merge_part_for(part, K) elements, so that one
// shared-memory size fits every key count), numbered over all buckets and
// handed to persistent CTAs in contiguous chunks (merge_pass_ws: a producer
// warp finds the splits and stages the inputs by bulk copies, the consumer
// warps merge).
__global__ void __launch_bounds__(kMergeThreads) merge_pass_kernel(const uint32_t* __restrict__ d_off, uint32_t W,
                                                                   uint32_t R, uint32_t part, int src, Ws ws,
                                                                   int presplit) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_off[kMaxW + 2], s_pre[kMaxW + 2];
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  pass_partitions(s_off, W, R, part, s_pre);
  __syncthreads();
  const uint32_t total = s_pre[W + 1];
  // a thread walks its partitions in increasing order, so the length search
  // only moves forward
  uint32_t L = 1;
  const auto part_of = [&](uint32_t q, uint32_t* K, uint32_t* P, uint32_t* bstart, uint32_t* cnt, uint32_t* o0) {
    while (L < W && s_pre[L + 1] <= q) ++L;
    *K = keys_for_len(L);
    *P = merge_part_for(part, *K);
    *o0 = (q - s_pre[L]) * *P;
    *bstart = s_off[L];
    *cnt = s_off[L + 1] - s_off[L];
  };
  merge_pass_ws(align128(smem), part, total, R, src, ws, presplit ? ws.splits : nullptr, part_of);
}

}  // namespace

cudaError_t launch_sort(uint32_t n_cap, uint32_t W, const SortParams& p, const uint32_t* d_off,
                        const Ws& ws, cudaStream_t s) {
  const uint32_t KW = W / 8;
  const uint32_t T = p.tile;
  const size_t tsm = tile_smem_bytes(KW, T);
  static SmemOptIn tile_smem_set, merge_smem_set;
  const uint32_t part = p.part;
  const size_t msm = merge_staged_smem_bytes(part) + 128;  // partitions shrink with the key count
  cudaError_t e = ensure_smem(tile_sort_kernel, tsm, &tile_smem_set);
  if (e == cudaSuccess) e = ensure_smem(merge_pass_kernel, msm, &merge_smem_set);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (n_cap + T - 1) / T + W;
  BSORT_LAUNCH(p.alg == BSORT_ODD_EVEN ? "tile_odd_even" : "tile_bitonic", tile_sort_kernel, tiles,
               p.threads, tsm, s, d_off, W, T, p.cross, ws);
  // persistent merge CTAs: as many as fit the SMs
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, merge_pass_kernel, kMergeThreads, msm);
  if (e != cudaSuccess) return e;
  const uint32_t per_sm = occ < 1 ? 1u : occ > 8 ? 8u : static_cast<uint32_t>(occ);
  const uint32_t need = (n_cap + part - 1) / part * 4 + W;  // partitions are at most part / 4
  const uint32_t fit = static_cast<uint32_t>(device_sm_count()) * per_sm;
  const uint32_t parts = need < fit ? need : fit;
  int src = 0;
  const uint32_t split_ctas = (need + 7) / 8 < static_cast<uint32_t>(device_sm_count()) * 8
                                  ? (need + 7) / 8 : static_cast<uint32_t>(device_sm_count()) * 8;
  for (uint64_t R = T; R < n_cap; R <<= 1) {
    const int presplit = n_cap >= kPresplitMinWords && R >= kPresplitMinRun;
    if (presplit)
      BSORT_LAUNCH("merge_split", merge_split_kernel, split_ctas, 256, 0, s, d_off, W, static_cast<uint32_t>(R),
                   part, src, ws);
    BSORT_LAUNCH("merge_pass", merge_pass_kernel, parts, kMergeThreads, msm, s, d_off, W,
                 static_cast<uint32_t>(R), part, src, ws, presplit);
    src ^= 1;
  }
  return cudaGetLastError();
}

}  // namespace bsort
