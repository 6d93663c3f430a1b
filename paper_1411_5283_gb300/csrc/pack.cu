// The paper's other output data structure (§3.1, "vectors of string"; the
// abstract contrasts it with the 3-D char array): the sorted words back to
// back without padding, plus offsets[n + 1] with word r at
// bytes[offsets[r] .. offsets[r+1]-1].
//
//   pack_sum_kernel    bytes of every tile of kPackTile words
//   pack_scan_kernel   exclusive scan of the tile sums (one block); the
//                      total goes to offsets[n] and is checked against the
//                      buffer's capacity
//   pack_write_kernel  per tile: the words' offsets (block scan of their
//                      lengths), then the bytes staged in shared memory at
//                      the destination's 16-byte phase and written out in
//                      aligned 16-byte pieces (byte stores only at a tile's
//                      two ragged ends, which it shares with its neighbours)
//
// A word's length comes from the bucket offsets when the order is the
// bucketed one (word r has the length L with off[L] <= r < off[L+1]), else
// from the input lengths through the permutation.
#include "block_scan.cuh"
#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

constexpr uint32_t kPackThreads = 256;
constexpr uint32_t kPackPer = 8;
constexpr uint32_t kPackTile = kPackThreads * kPackPer;  // 2,048 words
// tile sums (then the fit flag) live in the workspace's block table
constexpr uint32_t kPackMaxTiles = 128 * 1024;  // 268,435,456 words
static_assert((kPackMaxTiles + 1) * 4 <= 4 * kBins * kHistBlocksMax * 2, "tile sums fit the block table");

struct PackArgs {
  uint32_t n_cap, W;
  const uint32_t* off;   // bucket offsets (W + 2), or null
  const uint32_t* perm;  // output -> input index (with len), when off is null
  const uint8_t* len;
  const uint8_t* rec;
  uint8_t* bytes;
  uint64_t cap;
  uint32_t* offsets;
  uint32_t* sums;        // per tile, then the total and a flag
  uint32_t tiles_max;
  WsHeader* hdr;
};

__device__ __forceinline__ uint32_t pack_count(const PackArgs& a) {
  return a.off ? min(a.off[a.W + 1], a.n_cap) : a.n_cap;
}

// length of output word r (r < n)
__device__ __forceinline__ uint32_t word_len(const PackArgs& a, const uint32_t* s_off, uint32_t r) {
  if (a.off) {
    uint32_t lo = 1, hi = a.W;  // largest L with off[L] <= r
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= r) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
  return a.len[a.perm[r]];
}

__device__ __forceinline__ void load_off(const PackArgs& a, uint32_t* s_off) {
  if (a.off && threadIdx.x < a.W + 2) s_off[threadIdx.x] = a.off[threadIdx.x];
  __syncthreads();
}

__global__ void __launch_bounds__(kPackThreads) pack_sum_kernel(PackArgs a) {
  __shared__ uint32_t s_off[kMaxW + 2], tmp[kPackThreads / 32 + 1];
  load_off(a, s_off);
  const uint32_t n = pack_count(a);
  const uint32_t tiles = (n + kPackTile - 1) / kPackTile;
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    uint32_t sum = 0;
    for (uint32_t k = 0; k < kPackPer; ++k) {
      const uint32_t r = t * kPackTile + k * kPackThreads + threadIdx.x;
      if (r < n) sum += word_len(a, s_off, r);
    }
    uint32_t tot;
    block_exclusive_scan(sum, tmp, &tot);
    if (threadIdx.x == 0) a.sums[t] = tot;
  }
}

__global__ void __launch_bounds__(1024) pack_scan_kernel(PackArgs a) {
  __shared__ uint32_t tmp[1024 / 32 + 1];
  __shared__ uint32_t s_off[kMaxW + 2];
  load_off(a, s_off);
  const uint32_t n = pack_count(a);
  const uint32_t tiles = (n + kPackTile - 1) / kPackTile;
  const uint32_t per = (tiles + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = min(tiles, b + per);
  // n W < 2^32 (checked by the caller), so no sum overflows 32 bits
  uint32_t s = 0;
  for (uint32_t i = b; i < e; ++i) s += a.sums[i];
  uint32_t tot;
  uint32_t run = block_exclusive_scan(s, tmp, &tot);
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t v = a.sums[i];
    a.sums[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) {
    const bool fits = tot <= a.cap;
    a.sums[a.tiles_max] = fits ? 1u : 0u;
    if (!fits) set_error(a.hdr, BSORT_E_CAPACITY);
    a.offsets[n] = fits ? tot : 0u;
  }
}

__global__ void __launch_bounds__(kPackThreads) pack_write_kernel(PackArgs a) {
  extern __shared__ __align__(16) uint8_t stage[];  // 16 + kPackTile W bytes
  __shared__ uint32_t s_off[kMaxW + 2], tmp[kPackThreads / 32 + 1];
  load_off(a, s_off);
  const uint32_t n = pack_count(a);
  const uint32_t tiles = (n + kPackTile - 1) / kPackTile;
  const bool fits = a.sums[a.tiles_max] != 0;
  const uint32_t W = a.W;
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t r0 = t * kPackTile + threadIdx.x * kPackPer;  // a thread's words are consecutive
    uint32_t L[kPackPer], sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPackPer; ++k) {
      L[k] = r0 + k < n ? word_len(a, s_off, r0 + k) : 0u;
      sum += L[k];
    }
    uint32_t tot;
    const uint32_t mine = block_exclusive_scan(sum, tmp, &tot);
    const uint32_t base = a.sums[t];  // first byte of the tile
    uint32_t o = mine;
#pragma unroll
    for (uint32_t k = 0; k < kPackPer; ++k) {
      if (r0 + k < n) a.offsets[r0 + k] = base + o;
      o += L[k];
    }
    if (!fits) continue;  // block-uniform
    // stage the bytes at the destination's 16-byte phase
    const uint32_t phase = base & 15u;
    o = mine;
#pragma unroll
    for (uint32_t k = 0; k < kPackPer; ++k) {
      if (L[k]) {
        const uint8_t* src = a.rec + static_cast<uint64_t>(r0 + k) * W;
        uint8_t* dst = stage + phase + o;
        for (uint32_t q = 0; q < L[k]; q += 8) {
          const uint64_t w = *reinterpret_cast<const uint64_t*>(src + q);  // records are 8-byte aligned
          const uint32_t m = min(8u, L[k] - q);
          for (uint32_t j = 0; j < m; ++j) dst[q + j] = static_cast<uint8_t>(w >> (8 * j));
        }
      }
      o += L[k];
    }
    __syncthreads();
    // copy out: 16-byte pieces of the aligned span [base - phase, base + tot)
    uint8_t* gdst = a.bytes + (base - phase);
    const uint32_t end = phase + tot, pieces = (end + 15) / 16;
    for (uint32_t p = threadIdx.x; p < pieces; p += blockDim.x) {
      const uint32_t lo = p * 16, hi = lo + 16;
      if (lo >= phase && hi <= end) {
        *reinterpret_cast<uint4*>(gdst + lo) = *reinterpret_cast<const uint4*>(stage + lo);
      } else {
        for (uint32_t j = max(lo, phase); j < min(hi, end); ++j) gdst[j] = stage[j];
      }
    }
    __syncthreads();  // the stage is reused by the next tile
  }
}

}  // namespace

size_t pack_smem_bytes(uint32_t W) { return 16 + static_cast<size_t>(kPackTile) * W; }

cudaError_t launch_pack(uint32_t n_cap, uint32_t W, const uint8_t* rec, const uint32_t* d_off,
                        const uint32_t* perm, const uint8_t* len, uint8_t* bytes, uint64_t cap,
                        uint32_t* offsets, const Ws& ws, cudaStream_t s) {
  static SmemOptIn set;
  const size_t sm = pack_smem_bytes(W);
  cudaError_t e = ensure_smem(pack_write_kernel, sm, &set);
  if (e != cudaSuccess) return e;
  PackArgs a{};
  a.n_cap = n_cap;
  a.W = W;
  a.off = d_off;
  a.perm = perm;
  a.len = len;
  a.rec = rec;
  a.bytes = bytes;
  a.cap = cap;
  a.offsets = offsets;
  a.sums = ws.table;
  a.tiles_max = kPackMaxTiles;
  a.hdr = ws.hdr;
  const uint32_t tiles = (n_cap + kPackTile - 1) / kPackTile;
  const uint32_t cap_grid = static_cast<uint32_t>(device_sm_count()) * 8;
  const uint32_t grid = tiles == 0 ? 1u : (tiles < cap_grid ? tiles : cap_grid);
  BSORT_LAUNCH("pack_sum", pack_sum_kernel, grid, kPackThreads, 0, s, a);
  BSORT_LAUNCH("pack_scan", pack_scan_kernel, 1, 1024, 0, s, a);
  BSORT_LAUNCH("pack_write", pack_write_kernel, grid, kPackThreads, sm, s, a);
  return cudaGetLastError();
}

uint32_t pack_max_words() { return kPackMaxTiles * kPackTile; }

}  // namespace bsort
