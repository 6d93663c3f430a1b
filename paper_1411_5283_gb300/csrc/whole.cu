// The paper's unbucketed variant (Table 2, second row: the whole file sorted
// alphabetically without the length sub-arrays): every word ordered by its
// bytes, a proper prefix before the longer word, equal words by input index.
//
// The GPU form reaches that order from the length-bucketed answer.  Inside a
// length bucket the bucketed order and the whole-file order agree (same
// length: bytes, then index).  Across buckets, a record's zero-padded bytes
// order words as byte strings except that a word and the same word followed
// by zero bytes pad to the same record; the shorter one is the proper prefix
// and comes first.  So merging the sorted buckets in length order, pairwise
// and stably (on equal records the run of shorter lengths wins), gives the
// whole-file order:
//
//   whole_merge_kernel  one level: runs of `span` consecutive lengths merged
//                       in pairs by merge path (partitions of kWholePart
//                       outputs; a partition may cross pairs), records
//                       compared as big-endian 64-bit words in shared memory
//   whole_copy_kernel   after an odd number of levels, the answer moves from
//                       the scratch planes back to the caller's outputs
//
// ceil(log2 W) levels: 3 for W = 8, 4 for W = 16, 5 for W = 24 or 32.
#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

constexpr uint32_t kWholeThreads = 256;
constexpr uint32_t kWholePart = 1024;  // outputs per partition
constexpr uint32_t kWholePer = kWholePart / kWholeThreads;

// Shared memory of a merge CTA: input and output tiles of kWholePart
// elements, KW key planes and a permutation plane each.
__host__ __device__ constexpr size_t whole_smem_bytes(uint32_t KW) {
  return 2ull * kWholePart * (8 * KW + 4);
}

template <int KW>
struct RecTile {
  uint64_t* k[KW];
  uint32_t* p;
  // b before a?  (records compared as big-endian words)
  __device__ __forceinline__ bool less(uint32_t b, const RecTile& o, uint32_t a) const {
#pragma unroll
    for (int j = 0; j < KW; ++j)
      if (k[j][b] != o.k[j][a]) return k[j][b] < o.k[j][a];
    return false;
  }
};

template <int KW>
__device__ __forceinline__ void load_key(const uint8_t* rec, uint64_t i, uint64_t (&key)[KW]) {
  const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + i * (8 * KW));
#pragma unroll
  for (int j = 0; j < KW; ++j) key[j] = bswap64(src[j]);
}

template <int KW>
__device__ __forceinline__ bool key_less(const uint64_t (&a)[KW], const uint64_t (&b)[KW]) {
#pragma unroll
  for (int j = 0; j < KW; ++j)
    if (a[j] != b[j]) return a[j] < b[j];
  return false;
}

// Splits: the number of elements of run A among the first d outputs of the
// stable merge of A (na records at a) and B (nb records at b), equal records
// taken from A first.
// The same split found by one warp, 32 candidates a round: the predicate "A[i]
// comes after B[d-1-i]" is false then true along i (merge_path_warp's scheme;
// every lane of the warp calls and gets the split).
template <int KW>
__device__ uint32_t split_global_warp(const uint8_t* rec, uint64_t a, uint32_t na, uint64_t b, uint32_t nb,
                                      uint32_t d) {
  uint32_t lo = d > nb ? d - nb : 0u, hi = min(d, na);
  const uint32_t lane = threadIdx.x & 31u;
  while (lo < hi) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t q = lo + lane * step;
    bool holds = q >= hi;
    if (!holds) {
      uint64_t ka[KW], kb[KW];
      load_key<KW>(rec, a + q, ka);
      load_key<KW>(rec, b + d - 1 - q, kb);
      holds = key_less<KW>(kb, ka);
    }
    const uint32_t m = __ballot_sync(0xffffffffu, holds);
    if (m == 0) {
      lo += 31 * step + 1;
      continue;
    }
    const uint32_t f = __ffs(m) - 1;
    hi = min(lo + f * step, hi);
    lo = f ? lo + (f - 1) * step + 1 : lo;
  }
  return lo;
}

// The same split inside shared memory: A at positions [0, ca), B at [ca, ca + cb).
template <int KW>
__device__ uint32_t split_smem(const RecTile<KW>& t, uint32_t ca, uint32_t cb, uint32_t d) {
  uint32_t lo = d > cb ? d - cb : 0u, hi = min(d, ca);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (!t.less(ca + d - 1 - mid, t, mid)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Outputs [d0, d1) (relative to the pair's start at global position g0) of
// the stable merge of A = [g0, g0 + na) and B = [g0 + na, g0 + na + nb).
template <int KW>
__device__ void merge_range(uint8_t* smem, const uint8_t* src_rec, const uint32_t* src_perm,
                            uint8_t* dst_rec, uint32_t* dst_perm, uint64_t g0, uint32_t na,
                            uint32_t nb, uint32_t d0, uint32_t d1) {
  __shared__ uint32_t s_split[2];
  if (threadIdx.x < 64) {  // warps 0 and 1: the two splits
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t sp = split_global_warp<KW>(src_rec, g0, na, g0 + na, nb, w == 0 ? d0 : d1);
    if ((threadIdx.x & 31u) == 0) s_split[w] = sp;
  }
  __syncthreads();
  // sorted runs give i0 <= i1 <= i0 + (d1 - d0); clamping keeps every access
  // inside the runs should an earlier error have left them unsorted
  const uint32_t i0 = s_split[0];
  const uint32_t lo1 = d1 > nb ? d1 - nb : 0u;
  const uint32_t i1 = min(max(s_split[1], max(i0, lo1)), min(i0 + (d1 - d0), na));
  const uint32_t j0 = d0 - i0, j1 = d1 - i1;
  const uint32_t ca = i1 - i0, cb = j1 - j0, tot = ca + cb;
  RecTile<KW> in, out;
  uint64_t* kp = reinterpret_cast<uint64_t*>(smem);
#pragma unroll
  for (int j = 0; j < KW; ++j) {
    in.k[j] = kp + j * kWholePart;
    out.k[j] = kp + (KW + j) * kWholePart;
  }
  in.p = reinterpret_cast<uint32_t*>(kp + 2 * KW * kWholePart);
  out.p = in.p + kWholePart;
  // stage: record words of consecutive elements are consecutive in memory
  for (uint32_t q = threadIdx.x; q < tot * KW; q += blockDim.x) {
    const uint32_t e = q / KW, j = q % KW;
    const uint64_t g = e < ca ? g0 + i0 + e : g0 + na + j0 + (e - ca);
    in.k[j][e] = bswap64(reinterpret_cast<const uint64_t*>(src_rec)[g * KW + j]);
  }
  for (uint32_t e = threadIdx.x; e < tot; e += blockDim.x)
    in.p[e] = src_perm[e < ca ? g0 + i0 + e : g0 + na + j0 + (e - ca)];
  __syncthreads();
  const uint32_t o0 = min(tot, threadIdx.x * kWholePer), o1 = min(tot, o0 + kWholePer);
  uint32_t ia = split_smem<KW>(in, ca, cb, o0), ib = o0 - ia;
  for (uint32_t o = o0; o < o1; ++o) {
    const bool takeA = ia < ca && (ib >= cb || !in.less(ca + ib, in, ia));
    const uint32_t from = takeA ? ia++ : ca + ib++;
#pragma unroll
    for (int j = 0; j < KW; ++j) out.k[j][o] = in.k[j][from];
    out.p[o] = in.p[from];
  }
  __syncthreads();
  const uint64_t base = g0 + d0;
  for (uint32_t q = threadIdx.x; q < tot * KW; q += blockDim.x) {
    const uint32_t e = q / KW, j = q % KW;
    reinterpret_cast<uint64_t*>(dst_rec)[(base + e) * KW + j] = bswap64(out.k[j][e]);
  }
  for (uint32_t e = threadIdx.x; e < tot; e += blockDim.x) dst_perm[base + e] = out.p[e];
  __syncthreads();  // shared tiles and splits are reused by the next range
}

template <int KW>
__global__ void __launch_bounds__(kWholeThreads)
whole_merge_kernel(const uint32_t* __restrict__ d_off, uint32_t W, uint32_t span,
                   const uint8_t* __restrict__ src_rec, const uint32_t* __restrict__ src_perm,
                   uint8_t* __restrict__ dst_rec, uint32_t* __restrict__ dst_perm) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_off[kMaxW + 2];
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  const uint32_t n = s_off[W + 1];
  // length index -> position of its bucket (lengths past W end at n)
  const auto pos = [&](uint32_t L) { return L <= W ? s_off[L] : n; };
  for (uint32_t o0 = blockIdx.x * kWholePart; o0 < n; o0 += gridDim.x * kWholePart) {
    const uint32_t o1 = min(n, o0 + kWholePart);
    // pairs of runs at this level: lengths [a, a + span) and [a + span, a + 2 span)
    for (uint32_t a = 1; a <= W; a += 2 * span) {
      const uint32_t p0 = pos(a), pm = pos(a + span), p1 = pos(a + 2 * span);
      if (p1 <= o0 || p0 >= o1) continue;  // block-uniform
      const uint32_t lo = max(o0, p0), hi = min(o1, p1);
      merge_range<KW>(smem, src_rec, src_perm, dst_rec, dst_perm, p0, pm - p0, p1 - pm, lo - p0,
                      hi - p0);
    }
  }
}

__global__ void __launch_bounds__(kWholeThreads)
whole_copy_kernel(const uint32_t* __restrict__ d_off, uint32_t W, const uint4* __restrict__ src_rec,
                  const uint32_t* __restrict__ src_perm, uint4* __restrict__ dst_rec,
                  uint32_t* __restrict__ dst_perm) {
  const uint32_t n = d_off[W + 1];
  const uint64_t vecs = static_cast<uint64_t>(n) * W / 16;  // W is a multiple of 8; n W / 8 words
  const uint64_t step = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < vecs; i += step) dst_rec[i] = src_rec[i];
  if ((static_cast<uint64_t>(n) * W) & 15u) {  // an odd number of 8-byte words: the last one
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const uint64_t w = static_cast<uint64_t>(n) * W / 8 - 1;
      reinterpret_cast<uint64_t*>(dst_rec)[w] = reinterpret_cast<const uint64_t*>(src_rec)[w];
    }
  }
  for (uint64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) dst_perm[i] = src_perm[i];
}

template <int KW>
cudaError_t whole_levels(uint32_t n_cap, uint32_t W, const uint32_t* d_off, const Ws& ws,
                         uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s) {
  static SmemOptIn set;
  const size_t sm = whole_smem_bytes(KW);
  cudaError_t e = ensure_smem(whole_merge_kernel<KW>, sm, &set);
  if (e != cudaSuccess) return e;
  uint8_t* scr_rec = reinterpret_cast<uint8_t*>(ws.keys[0]);  // n W bytes fit K planes of cap words
  uint32_t* scr_perm = ws.idx[0];
  const uint32_t parts = (n_cap + kWholePart - 1) / kWholePart;
  const uint32_t cap_grid = static_cast<uint32_t>(device_sm_count()) * 8;
  const uint32_t grid = parts == 0 ? 1u : (parts < cap_grid ? parts : cap_grid);
  bool in_out = true;  // the current answer is in the caller's outputs
  for (uint32_t span = 1; span < W; span *= 2) {
    const uint8_t* sr = in_out ? out_rec : scr_rec;
    const uint32_t* sp = in_out ? out_perm : scr_perm;
    uint8_t* dr = in_out ? scr_rec : out_rec;
    uint32_t* dp = in_out ? scr_perm : out_perm;
    BSORT_LAUNCH("whole_merge", whole_merge_kernel<KW>, grid, kWholeThreads, sm, s, d_off, W, span, sr, sp,
                 dr, dp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    in_out = !in_out;
  }
  if (!in_out) {
    BSORT_LAUNCH("whole_copy", whole_copy_kernel, grid, kWholeThreads, 0, s, d_off, W,
                 reinterpret_cast<const uint4*>(scr_rec), scr_perm, reinterpret_cast<uint4*>(out_rec),
                 out_perm);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

cudaError_t launch_whole(uint32_t n_cap, uint32_t W, const uint32_t* d_off, const Ws& ws,
                         uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s) {
  switch (W / 8) {
    case 1: return whole_levels<1>(n_cap, W, d_off, ws, out_rec, out_perm, s);
    case 2: return whole_levels<2>(n_cap, W, d_off, ws, out_rec, out_perm, s);
    case 3: return whole_levels<3>(n_cap, W, d_off, ws, out_rec, out_perm, s);
    default: return whole_levels<4>(n_cap, W, d_off, ws, out_rec, out_perm, s);
  }
}

}  // namespace bsort
