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


// Exclusive scan of f(0..n-1) by one block of 1,024 threads into
// out[0..n-1], the total to *total_at (when given) and returned.  out may be
// the array f reads: each chunk is read whole before it is written.
template <typename F>
__device__ uint32_t block_scan_into(uint32_t n, F f, uint32_t* out, uint32_t* total_at) {
  // chunks of kScanChunk values: read with coalesced accesses (all of a
  // thread's reads in flight together) into shared memory, scanned there,
  // written back coalesced; a running carry joins the chunks
  constexpr uint32_t kScanChunk = 8192;
  constexpr uint32_t kPer = kScanChunk / 1024;
  __shared__ uint32_t tmp[1024 / 32 + 1];
  __shared__ uint32_t chunk[kScanChunk];
  uint32_t carry = 0;
  for (uint32_t c0 = 0; c0 < n; c0 += kScanChunk) {
    const uint32_t m = min(kScanChunk, n - c0);
    uint32_t vals[kPer];
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint32_t i = k * blockDim.x + threadIdx.x;
      vals[k] = i < m ? f(c0 + i) : 0u;
    }
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint32_t i = k * blockDim.x + threadIdx.x;
      if (i < kScanChunk) chunk[i] = vals[k];
    }
    __syncthreads();
    // thread t scans positions t kPer .. t kPer + kPer - 1 of the chunk
    uint32_t mine[kPer], s = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint32_t i = threadIdx.x * kPer + k;
      mine[k] = i < kScanChunk ? chunk[i] : 0u;
      s += mine[k];
    }
    uint32_t tot;
    uint32_t run = carry + block_exclusive_scan(s, tmp, &tot);
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint32_t i = threadIdx.x * kPer + k;
      if (i < kScanChunk) chunk[i] = run;
      run += mine[k];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) out[c0 + i] = chunk[i];
    carry += tot;
    __syncthreads();  // the chunk is reused
  }
  if (threadIdx.x == 0 && total_at) *total_at = carry;
  return carry;
}

}  // namespace bsort
