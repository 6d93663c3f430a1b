// Block-wide scans built from warp shuffles.
#pragma once

#include <cstdint>

namespace bsort {

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31u) >= static_cast<uint32_t>(d)) v += t;
  }
  return v;
}

// Exclusive prefix sum of v over the block (threads in order); *total gets the
// block sum.  warp_tmp must hold blockDim.x / 32 + 1 words.  All threads call.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tmp,
                                                         uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t nwarps = (blockDim.x + 31) >> 5;
  uint32_t inc = warp_inclusive_scan(v);
  if (lane == 31) warp_tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nwarps ? warp_tmp[lane] : 0u;
    uint32_t wi = warp_inclusive_scan(w);
    if (lane < nwarps) warp_tmp[lane] = wi - w;
    if (lane == 31) warp_tmp[nwarps] = wi;
  }
  __syncthreads();
  uint32_t r = warp_tmp[warp] + inc - v;
  *total = warp_tmp[nwarps];
  __syncthreads();
  return r;
}

}  // namespace bsort
