// Concatenation of the sorted buckets in ascending length (§3 Methodology,
// "Pre-processing", second phase: shorter words before longer ones).
//
// Bucket L already sits at ranks off[L]..off[L+1]-1 of the key planes, so
// output rank r reads its keys at position r of the buffer that holds bucket
// L's final run.  The record is rebuilt from the big-endian keys (bytes past
// the word are zero in the keys), so the input records are not read again.
// The packed form (§3.1, "vectors of string") writes the word's L bytes at
// its offset instead of the record.
#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

constexpr uint32_t kThreads = 256;

__device__ __forceinline__ uint32_t bucket_of(const uint32_t* s_off, uint32_t W, uint32_t r) {
  // largest L in 1..W with off[L] <= r
  uint32_t lo = 1, hi = W;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (s_off[mid] <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <bool kPacked>
__global__ void __launch_bounds__(kThreads)
gather_kernel(const uint32_t* __restrict__ d_off, uint32_t n_cap, const uint32_t* __restrict__ d_n,
              uint32_t W, Ws ws, uint8_t* __restrict__ out_rec, uint32_t* __restrict__ out_perm,
              PackOut pk) {
  __shared__ uint32_t s_off[kMaxW + 2];
  __shared__ uint32_t s_buf[kMaxW + 2];
  __shared__ uint32_t s_base[kMaxW + 2];
  __shared__ bool s_fits;
  if (threadIdx.x < W + 2) {
    s_off[threadIdx.x] = d_off[threadIdx.x];
    s_buf[threadIdx.x] = ws.hdr->final_buf[threadIdx.x];
  }
  __syncthreads();
  const uint32_t n = min(s_off[W + 1], d_n ? min(*d_n, n_cap) : n_cap);
  const uint32_t KW = W / 8;
  if constexpr (kPacked) {
    if (threadIdx.x == 0) {
      const uint32_t total = packed_bases(s_off, W, s_base);
      s_fits = total <= pk.cap;
      if (blockIdx.x == 0) {
        pk.offsets[n] = s_fits ? total : 0u;
        if (!s_fits) set_error(ws.hdr, BSORT_E_CAPACITY);
      }
    }
    __syncthreads();
  }
  for (uint32_t r = blockIdx.x * kThreads + threadIdx.x; r < n; r += gridDim.x * kThreads) {
    const uint32_t L = bucket_of(s_off, W, r);
    const uint32_t K = keys_for_len(L);
    const int buf = static_cast<int>(s_buf[L]);
    if constexpr (kPacked) {
      const uint32_t o = s_base[L] + r * L;
      pk.offsets[r] = o;
      if (s_fits) {
        for (uint32_t q = 0; q < K; ++q) {
          const uint64_t key = ws.keys[buf][q * ws.cap + r];
          const uint32_t m = min(8u, L - 8u * q);
          for (uint32_t j = 0; j < m; ++j)
            pk.bytes[o + 8 * q + j] = static_cast<uint8_t>(key >> (56 - 8 * j));
        }
      }
      out_perm[r] = ws.idx[buf][r];
      continue;
    }
    uint64_t* dst = reinterpret_cast<uint64_t*>(out_rec + static_cast<uint64_t>(r) * W);
    for (uint32_t k = 0; k < KW; k += 2) {
      const uint64_t a = k < K ? bswap64(ws.keys[buf][k * ws.cap + r]) : 0ull;
      if (k + 1 < KW) {
        const uint64_t b = k + 1 < K ? bswap64(ws.keys[buf][(k + 1) * ws.cap + r]) : 0ull;
        // W = 16 or 32 records are 16-byte aligned: one vector store per key pair
        if ((W & 15u) == 0) {
          reinterpret_cast<ulonglong2*>(dst)[k / 2] = make_ulonglong2(a, b);
        } else {
          dst[k] = a;
          dst[k + 1] = b;
        }
      } else {
        dst[k] = a;
      }
    }
    out_perm[r] = ws.idx[buf][r];
  }
}

__global__ void __launch_bounds__(kThreads)
export_kernel(const uint32_t* __restrict__ d_off, uint32_t n, uint32_t W, Ws ws,
              uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  __shared__ uint32_t s_off[kMaxW + 2];
  __shared__ uint32_t s_buf[kMaxW + 2];
  if (threadIdx.x < W + 2) {
    s_off[threadIdx.x] = d_off[threadIdx.x];
    s_buf[threadIdx.x] = ws.hdr->final_buf[threadIdx.x];
  }
  __syncthreads();
  const uint32_t m = min(n, s_off[W + 1]);
  const uint32_t KW = W / 8;
  for (uint32_t r = blockIdx.x * kThreads + threadIdx.x; r < m; r += gridDim.x * kThreads) {
    const uint32_t L = bucket_of(s_off, W, r);
    const uint32_t K = keys_for_len(L);
    const int buf = static_cast<int>(s_buf[L]);
    for (uint32_t k = 0; k < KW; ++k)
      keys[static_cast<uint64_t>(k) * n + r] = k < K ? ws.keys[buf][k * ws.cap + r] : 0ull;
    idx[r] = ws.idx[buf][r];
  }
}

uint32_t grid_for(uint32_t n) {
  uint32_t g = (n + kThreads - 1) / kThreads;
  if (g == 0) g = 1;
  if (g > 152u * 64u) g = 152u * 64u;
  return g;
}

}  // namespace

cudaError_t launch_gather(uint32_t n_cap, const uint32_t* d_n, uint32_t W, const uint32_t* d_off,
                          const Ws& ws, uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s,
                          const PackOut* pk) {
  if (pk) {
    BSORT_LAUNCH("gather_packed", gather_kernel<true>, grid_for(n_cap), kThreads, 0, s, d_off, n_cap,
                 d_n, W, ws, out_rec, out_perm, *pk);
  } else {
    BSORT_LAUNCH("gather", gather_kernel<false>, grid_for(n_cap), kThreads, 0, s, d_off, n_cap, d_n,
                 W, ws, out_rec, out_perm, PackOut{});
  }
  return cudaGetLastError();
}

cudaError_t launch_export(uint32_t n, uint32_t W, const uint32_t* d_off, const Ws& ws,
                          uint64_t* keys, uint32_t* idx, cudaStream_t s) {
  BSORT_LAUNCH("export", export_kernel, grid_for(n), kThreads, 0, s, d_off, n, W, ws, keys, idx);
  return cudaGetLastError();
}

}  // namespace bsort
