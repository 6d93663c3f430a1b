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
//   whole_split_kernel  one level: the output of each pair of runs (runs of
//                       `span` consecutive lengths) cut into units of P
//                       outputs; the merge-path split at every unit's first
//                       output, one warp per unit, all at once
//   whole_merge_kernel  the level's units handed to persistent CTAs: thread 0
//                       stages the next unit's two record ranges and
//                       permutation ranges into one of two shared-memory
//                       buffers with bulk copies (TMA) while the CTA merges
//                       the current one (records compared as big-endian
//                       64-bit words) into a third buffer, written out in
//                       coalesced stores
//   whole_copy_kernel   after an odd number of levels, the answer moves from
//                       the scratch planes back to the caller's outputs
//
// ceil(log2 W) levels: 3 for W = 8, 4 for W = 16, 5 for W = 24 or 32.
#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

constexpr uint32_t kWholeThreads = 256;

// Outputs per unit: the buffers hold a unit's records and permutation entries.
__host__ __device__ constexpr uint32_t whole_part(uint32_t W) { return W <= 16 ? 1024u : 512u; }

// One input buffer: [mbarrier 16 B][record area: P W + 64 B][permutation area:
// 4 P + 64 B].  In each area the first run's range starts at the area's start
// and the second's after the first's bytes; a range is copied from the
// 16-byte boundary at or below its first byte (record shift 0 or 8 bytes,
// permutation shift 0..12 bytes), which the 64 spare bytes per area cover.
__host__ __device__ constexpr size_t whole_rec_area(uint32_t W) {
  return static_cast<size_t>(whole_part(W)) * W + 64;
}
__host__ __device__ constexpr size_t whole_buf_bytes(uint32_t W) {
  return (16 + whole_rec_area(W) + 4 * static_cast<size_t>(whole_part(W)) + 64 + 127) / 128 * 128;
}
// The output buffer: P records, then P permutation entries.
__host__ __device__ constexpr size_t whole_out_bytes(uint32_t W) {
  return (static_cast<size_t>(whole_part(W)) * (W + 4) + 127) / 128 * 128;
}
// Shared memory of a merge CTA, with 128 bytes of alignment slack.
__host__ __device__ constexpr size_t whole_smem_bytes(uint32_t W) {
  return 2 * whole_buf_bytes(W) + whole_out_bytes(W) + 128;
}

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

// The split: the number of elements of run A among the first d outputs of
// the stable merge of A (na records at a) and B (nb records at b), equal
// records taken from A first, found by one warp, 32 candidates a round: the
// predicate "A[i] comes after B[d-1-i]" is false then true along i (every lane
// of the warp calls and gets the split).
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

// A level's units: pair k of runs covers lengths [1 + 2 span k, 1 + 2 span k
// + span) and the next span lengths; its units are numbered after those of
// the earlier pairs (s_upre, thread 0 writes it; np pairs).
__device__ void whole_units(const uint32_t* s_off, uint32_t W, uint32_t span, uint32_t P, uint32_t* s_upre,
                            uint32_t* np) {
  if (threadIdx.x == 0) {
    const uint32_t n = s_off[W + 1];
    uint32_t acc = 0, k = 0;
    for (uint32_t a = 1; a <= W; a += 2 * span, ++k) {
      s_upre[k] = acc;
      const uint32_t p0 = s_off[a], p1 = a + 2 * span <= W ? s_off[a + 2 * span] : n;
      acc += (p1 - p0 + P - 1) / P;
    }
    s_upre[k] = acc;
    *np = k;
  }
}

struct WholePair {
  uint32_t p0, na, nb;  // the pair's first position and its two runs' lengths
  uint32_t d0;          // the unit's first output, relative to p0
};

__device__ __forceinline__ WholePair whole_pair(const uint32_t* s_off, const uint32_t* s_upre, uint32_t W,
                                                uint32_t span, uint32_t P, uint32_t k, uint32_t q) {
  const uint32_t n = s_off[W + 1], a = 1 + 2 * span * k;
  WholePair r;
  r.p0 = s_off[a];
  const uint32_t pm = a + span <= W ? s_off[a + span] : n, p1 = a + 2 * span <= W ? s_off[a + 2 * span] : n;
  r.na = pm - r.p0;
  r.nb = p1 - pm;
  r.d0 = (q - s_upre[k]) * P;
  return r;
}

template <int KW>
__global__ void __launch_bounds__(kWholeThreads)
whole_split_kernel(const uint32_t* __restrict__ d_off, uint32_t W, uint32_t span, const uint8_t* __restrict__ rec,
                   uint32_t* __restrict__ splits) {
  __shared__ uint32_t s_off[kMaxW + 2], s_upre[kMaxW + 2], s_np;
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  const uint32_t P = whole_part(W);
  whole_units(s_off, W, span, P, s_upre, &s_np);
  __syncthreads();
  const uint32_t total = s_upre[s_np];
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); q < total; q += warps) {
    uint32_t k = 0;
    while (s_upre[k + 1] <= q) ++k;  // warp-uniform
    const WholePair pr = whole_pair(s_off, s_upre, W, span, P, k, q);
    const uint32_t sp = pr.d0 == 0 ? 0u : split_global_warp<KW>(rec, pr.p0, pr.na, pr.p0 + pr.na, pr.nb, pr.d0);
    if ((threadIdx.x & 31u) == 0) splits[q] = sp;
  }
}

struct WholeGeo {
  uint32_t ca, cb;
  uint32_t shA, shB, offB;   // record area: byte shift of each range, byte offset of the second
  uint32_t psA, psB, poffB;  // permutation area: the same
  uint64_t out0;             // first output position
};

// Thread 0: the geometry of unit q (pair pr, raw splits s0 and s1) and its
// bulk copies into buf, whose barrier is told the bytes to expect.
__device__ WholeGeo whole_issue(uint8_t* buf, uint32_t W, uint32_t P, const WholePair& pr, uint32_t s0, uint32_t s1,
                                const uint8_t* src_rec, const uint32_t* src_perm) {
  const uint32_t cnt = pr.na + pr.nb, d0 = pr.d0, d1 = min(d0 + P, cnt);
  const uint32_t na = pr.na, nb = pr.nb;
  // clamped as in the bucket merge: keeps every copy inside the runs should
  // an earlier device error have left them unsorted
  const uint32_t i0 = min(max(s0, d0 > nb ? d0 - nb : 0u), min(na, d0));
  const uint32_t i1 = min(max(s1, max(i0, d1 > nb ? d1 - nb : 0u)), min(na, i0 + (d1 - d0)));
  WholeGeo g;
  g.ca = i1 - i0;
  g.cb = (d1 - d0) - g.ca;
  g.out0 = static_cast<uint64_t>(pr.p0) + d0;
  const uint64_t gA = static_cast<uint64_t>(pr.p0) + i0, gB = static_cast<uint64_t>(pr.p0) + na + (d0 - i0);
  const uint8_t* rA = src_rec + gA * W;
  const uint8_t* rB = src_rec + gB * W;
  const uint32_t* qA = src_perm + gA;
  const uint32_t* qB = src_perm + gB;
  g.shA = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(rA) & 15u);
  g.shB = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(rB) & 15u);
  g.psA = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(qA) & 15u);
  g.psB = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(qB) & 15u);
  const uint32_t rbA = g.ca ? ((g.shA + g.ca * W + 15u) & ~15u) : 0u;
  const uint32_t rbB = g.cb ? ((g.shB + g.cb * W + 15u) & ~15u) : 0u;
  const uint32_t pbA = g.ca ? ((g.psA + g.ca * 4 + 15u) & ~15u) : 0u;
  const uint32_t pbB = g.cb ? ((g.psB + g.cb * 4 + 15u) & ~15u) : 0u;
  g.offB = rbA;
  g.poffB = pbA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf);
  uint8_t* ra = buf + 16;
  uint8_t* pa = ra + whole_rec_area(W);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, rbA + rbB + pbA + pbB);
  // each copy starts at the 16-byte boundary at or below its first byte and
  // ends in the 16-byte block of its last one, so it reads no other page
  if (rbA) bulk_g2s(ra, rA - g.shA, rbA, bar);
  if (rbB) bulk_g2s(ra + rbA, rB - g.shB, rbB, bar);
  if (pbA) bulk_g2s(pa, reinterpret_cast<const uint8_t*>(qA) - g.psA, pbA, bar);
  if (pbB) bulk_g2s(pa + pbA, reinterpret_cast<const uint8_t*>(qB) - g.psB, pbB, bar);
  return g;
}

// A staged record as big-endian key words (16-byte loads when W is a multiple
// of 16: every staged record then starts on a 16-byte boundary).
template <int KW>
__device__ __forceinline__ void staged_key(const uint8_t* p, uint64_t (&k)[KW]) {
  if constexpr (KW % 2 == 0) {
#pragma unroll
    for (int j = 0; j < KW; j += 2) {
      const ulonglong2 v = reinterpret_cast<const ulonglong2*>(p)[j / 2];
      k[j] = bswap64(v.x);
      k[j + 1] = bswap64(v.y);
    }
  } else {
#pragma unroll
    for (int j = 0; j < KW; ++j) k[j] = bswap64(reinterpret_cast<const uint64_t*>(p)[j]);
  }
}

// Writes key words k back as a record at p (16-byte stores when KW is even).
template <int KW>
__device__ __forceinline__ void put_record(uint64_t* p, const uint64_t (&k)[KW]) {
  if constexpr (KW % 2 == 0) {
#pragma unroll
    for (int j = 0; j < KW; j += 2) reinterpret_cast<ulonglong2*>(p)[j / 2] = make_ulonglong2(bswap64(k[j]), bswap64(k[j + 1]));
  } else {
#pragma unroll
    for (int j = 0; j < KW; ++j) p[j] = bswap64(k[j]);
  }
}

// Merges a staged unit into `out` (thread t produces outputs [t per, t per +
// per)), equal records from A first, then writes it out in coalesced stores.
template <int KW>
__device__ void whole_merge_staged(const uint8_t* buf, uint8_t* out, const WholeGeo& g, uint32_t P,
                                   uint8_t* dst_rec, uint32_t* dst_perm) {
  constexpr uint32_t W = 8 * KW;
  const uint8_t* ra = buf + 16;
  const uint8_t* pa = ra + whole_rec_area(W);
  const auto recA = [&](uint32_t i) { return ra + g.shA + i * W; };
  const auto recB = [&](uint32_t i) { return ra + g.offB + g.shB + i * W; };
  const auto permA = [&](uint32_t i) { return *reinterpret_cast<const uint32_t*>(pa + g.psA + 4 * i); };
  const auto permB = [&](uint32_t i) { return *reinterpret_cast<const uint32_t*>(pa + g.poffB + g.psB + 4 * i); };
  uint64_t* orec = reinterpret_cast<uint64_t*>(out);
  uint32_t* operm = reinterpret_cast<uint32_t*>(out + static_cast<size_t>(P) * W);
  const uint32_t tot = g.ca + g.cb;
  const uint32_t per = (P + blockDim.x - 1) / blockDim.x;
  const uint32_t o0 = min(tot, threadIdx.x * per), o1 = min(tot, o0 + per);
  // A elements among the first o0 outputs
  uint32_t lo = o0 > g.cb ? o0 - g.cb : 0u, hi = min(o0, g.ca);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    uint64_t ka[KW], kb[KW];
    staged_key<KW>(recA(mid), ka);
    staged_key<KW>(recB(o0 - 1 - mid), kb);
    if (!key_less<KW>(kb, ka)) lo = mid + 1;
    else hi = mid;
  }
  uint32_t ia = lo, ib = o0 - lo;
  uint64_t ka[KW], kb[KW];
  if (ia < g.ca) staged_key<KW>(recA(ia), ka);
  if (ib < g.cb) staged_key<KW>(recB(ib), kb);
  for (uint32_t o = o0; o < o1; ++o) {
    const bool takeA = ib >= g.cb || (ia < g.ca && !key_less<KW>(kb, ka));
    if (takeA) {
      put_record<KW>(orec + o * KW, ka);
      operm[o] = permA(ia);
      if (++ia < g.ca) staged_key<KW>(recA(ia), ka);
    } else {
      put_record<KW>(orec + o * KW, kb);
      operm[o] = permB(ib);
      if (++ib < g.cb) staged_key<KW>(recB(ib), kb);
    }
  }
  __syncthreads();
  uint64_t* drec = reinterpret_cast<uint64_t*>(dst_rec) + g.out0 * KW;
  if constexpr (KW % 2 == 0) {
    // the output records start on 16-byte boundaries: 16-byte stores
    ulonglong2* d2 = reinterpret_cast<ulonglong2*>(drec);
    const ulonglong2* o2 = reinterpret_cast<const ulonglong2*>(orec);
    for (uint32_t q = threadIdx.x; q < tot * KW / 2; q += blockDim.x) d2[q] = o2[q];
  } else {
    for (uint32_t q = threadIdx.x; q < tot * KW; q += blockDim.x) drec[q] = orec[q];
  }
  for (uint32_t e = threadIdx.x; e < tot; e += blockDim.x) dst_perm[g.out0 + e] = operm[e];
}

template <int KW>
__global__ void __launch_bounds__(kWholeThreads, 4)
whole_merge_kernel(const uint32_t* __restrict__ d_off, uint32_t W, uint32_t span,
                   const uint8_t* __restrict__ src_rec, const uint32_t* __restrict__ src_perm,
                   uint8_t* __restrict__ dst_rec, uint32_t* __restrict__ dst_perm,
                   const uint32_t* __restrict__ splits, Ws ws) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint32_t s_off[kMaxW + 2], s_upre[kMaxW + 2], s_np;
  __shared__ WholeGeo s_geo[2];
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  const uint32_t P = whole_part(W);
  whole_units(s_off, W, span, P, s_upre, &s_np);
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t* buf[2] = {smem, smem + whole_buf_bytes(W)};
  uint8_t* out = smem + 2 * whole_buf_bytes(W);
  if (threadIdx.x == 0) {
    mbar_init(reinterpret_cast<uint64_t*>(buf[0]), 1);
    mbar_init(reinterpret_cast<uint64_t*>(buf[1]), 1);
    fence_barrier_init();
  }
  __syncthreads();
  const uint32_t total = s_upre[s_np];
  uint32_t k = 0;  // thread 0's pair, walking forward with its units
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {false, false};  // thread 0: a copy is in flight into buffer x
  const auto issue = [&](uint32_t q, int x) {
    while (s_upre[k + 1] <= q) ++k;
    const WholePair pr = whole_pair(s_off, s_upre, W, span, P, k, q);
    const uint32_t cnt = pr.na + pr.nb, d1 = min(pr.d0 + P, cnt);
    const uint32_t s0 = pr.d0 == 0 ? 0u : splits[q];
    const uint32_t s1 = d1 == cnt ? pr.na : splits[q + 1];
    s_geo[x] = whole_issue(buf[x], W, P, pr, s0, s1, src_rec, src_perm);
    pending[x] = true;
  };
  int b = 0;
  if (threadIdx.x == 0 && blockIdx.x < total) issue(blockIdx.x, 0);
  for (uint32_t q = blockIdx.x; q < total; q += gridDim.x, b ^= 1) {
    const uint32_t qn = q + gridDim.x;
    if (threadIdx.x == 0 && qn < total) issue(qn, b ^ 1);  // buffer b ^ 1 was released last round
    const bool ok = mbar_wait_bounded(reinterpret_cast<uint64_t*>(buf[b]), phase[b], ws.wait_polls);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        set_error(ws.hdr, BSORT_E_TIMEOUT);
        for (int x = 0; x < 2; ++x)  // let the copies in flight land before the CTA exits
          if (pending[x]) mbar_wait_bounded(reinterpret_cast<uint64_t*>(buf[x]), phase[x]);
      }
      return;
    }
    phase[b] ^= 1u;
    pending[b] = false;
    const WholeGeo g = s_geo[b];
    whole_merge_staged<KW>(buf[b], out, g, P, dst_rec, dst_perm);
    __syncthreads();  // buffer b, its geometry and the output buffer are free again
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
  const size_t sm = whole_smem_bytes(W);
  cudaError_t e = ensure_smem(whole_merge_kernel<KW>, sm, &set);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, whole_merge_kernel<KW>, kWholeThreads, sm);
  if (e != cudaSuccess) return e;
  uint8_t* scr_rec = reinterpret_cast<uint8_t*>(ws.keys[0]);  // n W bytes fit K planes of cap words
  uint32_t* scr_perm = ws.idx[0];
  const uint32_t P = whole_part(W);
  const uint32_t units = (n_cap + P - 1) / P + W;  // at most one partial unit per pair
  const uint32_t sms = static_cast<uint32_t>(device_sm_count());
  const uint32_t fit = sms * static_cast<uint32_t>(occ < 1 ? 1 : occ);
  const uint32_t grid = units < fit ? units : fit;
  const uint32_t split_grid = (units + 7) / 8 < sms * 8 ? (units + 7) / 8 : sms * 8;
  bool in_out = true;  // the current answer is in the caller's outputs
  for (uint32_t span = 1; span < W; span *= 2) {
    const uint8_t* sr = in_out ? out_rec : scr_rec;
    const uint32_t* sp = in_out ? out_perm : scr_perm;
    uint8_t* dr = in_out ? scr_rec : out_rec;
    uint32_t* dp = in_out ? scr_perm : out_perm;
    BSORT_LAUNCH("whole_split", whole_split_kernel<KW>, split_grid, kWholeThreads, 0, s, d_off, W, span, sr,
                 ws.splits);
    BSORT_LAUNCH("whole_merge", whole_merge_kernel<KW>, grid, kWholeThreads, sm, s, d_off, W, span, sr, sp, dr, dp,
                 ws.splits, ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    in_out = !in_out;
  }
  if (!in_out) {
    const uint32_t cgrid = sms * 8;
    BSORT_LAUNCH("whole_copy", whole_copy_kernel, cgrid, kWholeThreads, 0, s, d_off, W,
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
