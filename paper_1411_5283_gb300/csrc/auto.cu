// Sample-sort strategy for large inputs (BSORT_AUTO in the one-call paths).
//
// Same answer as the paper's phases 2-3 and the concatenation (§3
// Methodology, "Pre-processing"): every word ordered by (length, bytes, input
// index).  Phase 2's length buckets are refined into key-range segments small
// enough for one CTA's shared memory, so the words cross HBM about twice
// instead of once per merge pass:
//
//   auto_sample_kernel     stratified sample (one position per 32 words, kept
//                          with probability 1/4, 1/2, 1 for 1, 2, >= 3 key
//                          words: about 20 samples per expected segment),
//                          grouped by length bucket (phase 2's sub-arrays)
//   auto_splitter_kernel   one CTA per bucket sorts its samples and picks
//                          g_L - 1 splitters by (keys, index), so a word
//                          repeated many times is split evenly by index;
//                          every segment gets a region of the shared-memory
//                          capacity, three times its expected count
//   auto_partition_kernel  every word finds its segment by binary search over
//                          the splitters (staged in shared memory) and takes a
//                          slot with a warp-aggregated atomic; a slot past the
//                          region's end only counts and raises the overflow flag
//   auto_layout_kernel     output base of every segment (scan of the exact
//                          counts); on overflow, exact regions for a retry
//   auto_partition_kernel  (again) the retry pass, a no-op unless overflow
//   auto_segsort_kernel    one CTA per segment: bulk-copy (TMA) the segment
//                          into shared memory, merge sort it (register sort of
//                          E elements per thread, then merge-path rounds in
//                          padded shared memory), write the final records and
//                          permutation at the segment's output base; a segment
//                          larger than shared memory (only after a retry) is
//                          sorted in chunks and merged in global memory
#include "block_scan.cuh"
#include "common.cuh"
#include "kernels.h"
#include "sort_impl.cuh"

namespace bsort {

namespace {

constexpr uint32_t kPartThreads = 512;
constexpr uint32_t kSplSmem = 110 * 1024;          // splitter table staged up to this size
constexpr uint32_t kSegThreads = 512;
// One cursor per 128-byte line: the partition's atomics then spread over all
// L2 slices instead of piling onto the few lines a packed array would use.
constexpr uint32_t kCursorStride = 32;

// words per lane kept in flight by the partition pass (fewer for wide keys)
template <int KW> struct PartWords { static constexpr uint32_t value = KW <= 2 ? 4 : 2; };

// ---------------------------------------------------------------------------
// Device view of the AUTO area
// ---------------------------------------------------------------------------
struct AutoHdr {
  uint32_t overflow;        // a partition slot fell past its region
  uint32_t retry;           // the retry pass is armed
  uint32_t G;               // segments in total
  uint32_t spl_bytes;       // bytes of the splitter table
  uint32_t samp_cnt[kBins]; // samples drawn per bucket (may exceed capacity)
  uint32_t total[kBins];    // words per length (the histogram of phase 2)
};

struct AutoView {
  AutoHdr* hdr;
  uint64_t* samp64;   // per bucket L: K_L planes of sample keys (scap each)
  uint32_t* samp32;   // per bucket L: sample indices
  uint8_t* spl;       // splitter table: per bucket, K_L key planes then indices
  uint32_t* cursor;   // per segment: slots taken, at cursor[seg * kCursorStride]
  uint32_t* rcap;     // per segment: region capacity (elements)
  uint32_t* outbase;  // per segment: first output rank
  uint32_t* segL;     // per segment: its length bucket
  uint64_t* rbase;    // per segment: first u64 of its K key planes in the key area
  uint64_t* ibase;    // per segment: first u32 of its index plane in the index area
  uint64_t* area64;   // key area (keys A, B, C of the workspace, contiguous)
  uint32_t* area32;   // index area (idx A, B, C, contiguous)
  uint64_t size64, size32;
  uint64_t cap;
};

__host__ __device__ AutoView auto_view(const Ws& ws, uint32_t W) {
  AutoView v{};
  const uint64_t cap = ws.cap;
  const uint32_t KW = W / 8;
  uint8_t* p = ws.autoa;
  v.hdr = reinterpret_cast<AutoHdr*>(p);
  size_t o = 4096;
  size_t s64 = 0, s32 = 0;
  for (uint32_t L = 1; L <= W; ++L) {
    const uint32_t K = (L + 7) / 8;
    s64 += static_cast<size_t>(auto_sample_cap(K, cap)) * K;
    s32 += auto_sample_cap(K, cap);
  }
  v.samp64 = reinterpret_cast<uint64_t*>(p + o);
  o += 8 * s64;
  v.samp32 = reinterpret_cast<uint32_t*>(p + o);
  o += align_up(4 * s32, 16);
  const uint64_t G = auto_max_segments(cap);
  v.spl = p + o;
  o += align_up(G * (8 * KW + 4) + (16 + kAutoDirBytes) * kBins, 16);
  v.rbase = reinterpret_cast<uint64_t*>(p + o);
  o += 8 * G;
  v.ibase = reinterpret_cast<uint64_t*>(p + o);
  o += 8 * G;
  v.cursor = reinterpret_cast<uint32_t*>(p + o);
  o += 4 * G * kCursorStride;
  v.rcap = reinterpret_cast<uint32_t*>(p + o);
  o += 4 * G;
  v.outbase = reinterpret_cast<uint32_t*>(p + o);
  o += 4 * G;
  v.segL = reinterpret_cast<uint32_t*>(p + o);
  v.area64 = ws.keys[0];
  v.area32 = ws.idx[0];
  const uint64_t third = cap >= kAutoMinWords + 64 ? cap + kAutoSlack : 0;
  v.size64 = (2 * cap + third) * KW;
  v.size32 = 2 * cap + third;
  v.cap = cap;
  return v;
}

// Per-bucket plan, a pure function of the bucket counts.
struct BucketPlan {
  uint32_t g;        // segments
  uint32_t cap;      // region capacity of each segment
  uint32_t seg0;     // first global segment id
  uint32_t K;        // key words
  uint64_t r64, r32; // first u64 / u32 of the bucket's regions
  uint32_t s64, s32; // first u64 / u32 of the bucket's sample planes
  uint32_t scap;     // sample capacity of the bucket
  uint32_t spl_off;  // byte offset of the bucket's splitters in the table
};

__host__ __device__ __forceinline__ uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }

__device__ void bucket_geometry(uint32_t cnt, uint32_t K, uint32_t* g, uint32_t* cap) {
  if (cnt == 0) {
    *g = 0;
    *cap = 0;
  } else if (cnt <= auto_seg_cap(K)) {
    *g = 1;
    *cap = round4(cnt);
  } else {
    *g = (cnt + auto_target(K) - 1) / auto_target(K);
    *cap = auto_seg_cap(K);
  }
}

// A bucket's splitter block: a 257-entry directory on the first key byte
// (dir[b] = splitters whose first byte is below b), then K key planes and the
// index plane of its g - 1 splitters.
constexpr uint32_t kDirBytes = kAutoDirBytes;

__device__ __forceinline__ uint32_t spl_bytes_of(uint32_t g, uint32_t K) {
  return g >= 2 ? static_cast<uint32_t>(kDirBytes + align_up((g - 1) * (8 * K + 4), 16)) : 0u;
}

__device__ BucketPlan plan_for(const uint32_t* off, uint32_t L, uint64_t cap_ws) {
  BucketPlan p{};
  for (uint32_t l = 1; l <= L; ++l) {
    const uint32_t K = (l + 7) / 8;
    uint32_t g, c;
    bucket_geometry(off[l + 1] - off[l], K, &g, &c);
    const uint32_t sc = auto_sample_cap(K, cap_ws);
    if (l == L) {
      p.g = g;
      p.cap = c;
      p.K = K;
      p.scap = sc;
      return p;
    }
    p.seg0 += g;
    p.r64 += static_cast<uint64_t>(g) * c * K;
    p.r32 += static_cast<uint64_t>(g) * c;
    p.s64 += sc * K;
    p.s32 += sc;
    p.spl_off += spl_bytes_of(g, K);
  }
  return p;
}

// 64-bit mix for the stratified sample position (SplitMix64 finaliser).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t word_count(uint32_t n_cap, const uint32_t* d_n) {
  return d_n ? min(*d_n, n_cap) : n_cap;
}

__device__ void load_plans(BucketPlan* plans, uint32_t* s_off, const uint32_t* d_off, uint32_t W,
                           uint64_t cap) {
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  if (threadIdx.x >= 1 && threadIdx.x <= W) plans[threadIdx.x] = plan_for(s_off, threadIdx.x, cap);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// 1. sample
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
auto_sample_kernel(const uint8_t* __restrict__ rec, const uint8_t* __restrict__ len,
                   uint32_t n_cap, const uint32_t* __restrict__ d_n, uint32_t W,
                   const uint32_t* __restrict__ d_off, Ws ws) {
  __shared__ BucketPlan plans[kMaxW + 1];
  __shared__ uint32_t s_off[kMaxW + 2];
  const AutoView v = auto_view(ws, W);
  load_plans(plans, s_off, d_off, W, v.cap);
  const uint32_t n = word_count(n_cap, d_n);
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t h = mix64(s + 0x9E3779B97F4A7C15ull);
  const uint64_t i64 = static_cast<uint64_t>(s) * kAutoSampleEvery + (h & (kAutoSampleEvery - 1));
  if (i64 >= n) return;
  const uint32_t i = static_cast<uint32_t>(i64);
  const uint32_t L = len[i];
  if (L == 0 || L > W) return;
  const BucketPlan& p = plans[L];
  if (p.g < 2) return;  // one segment: no splitters needed
  // Acceptance probability: about 20 samples per expected segment (segments
  // expect 2730 / 1365 / 682 words for 1 / 2 / >= 3 keys, positions are one per
  // 32 words), but never more than 90 % of the bucket's sample capacity.  The
  // capacity must not truncate: arrivals come in position order, and the input
  // index is part of the sort key, so a truncated sample would cover only the
  // early copies of a frequent word.
  const uint32_t cnt = s_off[L + 1] - s_off[L];
  const double want = p.K == 1 ? 0.25 : (p.K == 2 ? 0.5 : 1.0);
  const double room = 0.9 * p.scap * static_cast<double>(kAutoSampleEvery) / cnt;
  const double q = want < room ? want : room;
  if (static_cast<double>(h >> 32) >= q * 4294967296.0) return;
  const uint32_t slot = atomicAdd(&v.hdr->samp_cnt[L], 1u);
  if (slot >= p.scap) return;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + static_cast<uint64_t>(i) * W);
  for (uint32_t k = 0; k < p.K; ++k)
    v.samp64[p.s64 + k * p.scap + slot] = bswap64(__ldg(src + k)) & key_mask(L, k);
  v.samp32[p.s32 + slot] = i;
}

// ---------------------------------------------------------------------------
// 2. splitters and region layout (one CTA per bucket)
// ---------------------------------------------------------------------------
template <int K>
__device__ void choose_splitters(uint8_t* smem, const AutoView& v, const BucketPlan& p, uint32_t L) {
  const uint32_t m = min(v.hdr->samp_cnt[L], p.scap);
  SmemTile<K> t;
  uint64_t* kp = reinterpret_cast<uint64_t*>(smem);
#pragma unroll
  for (int j = 0; j < K; ++j) t.k[j] = kp + j * p.scap;
  t.idx = reinterpret_cast<uint32_t*>(kp + K * p.scap);
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    Elem<K> e;
#pragma unroll
    for (int j = 0; j < K; ++j) e.k[j] = v.samp64[p.s64 + j * p.scap + i];
    e.idx = v.samp32[p.s32 + i];
    t.put(i, e);
  }
  __syncthreads();
  bitonic_flip<K>(t, m);
  __syncthreads();
  // splitter s (0 <= s < g-1) = lower bound of segment s+1 = sample of rank
  // floor((s+1) m / g); with no samples every splitter is +inf, so all words
  // land in the first segment (overflow then gives it an exact region)
  const uint32_t ns = p.g - 1;
  uint16_t* dir = reinterpret_cast<uint16_t*>(v.spl + p.spl_off);
  uint64_t* sk = reinterpret_cast<uint64_t*>(v.spl + p.spl_off + kDirBytes);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + static_cast<size_t>(K) * ns);
  auto rank_of = [&](uint32_t s) {
    return static_cast<uint32_t>((static_cast<uint64_t>(s + 1) * m) / p.g);
  };
  for (uint32_t s = threadIdx.x; s < ns; s += blockDim.x) {
    if (m == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) sk[k * ns + s] = ~0ull;
      si[s] = ~0u;
    } else {
      const Elem<K> e = t.get(rank_of(s));
#pragma unroll
      for (int k = 0; k < K; ++k) sk[k * ns + s] = e.k[k];
      si[s] = e.idx;
    }
  }
  // directory: dir[b] = number of splitters whose first byte is below b
  // (splitters are sorted, so their first bytes never decrease)
  for (uint32_t b = threadIdx.x; b <= 256; b += blockDim.x) {
    uint32_t lo = 0, hi = ns;  // first splitter with first byte >= b
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint64_t k0 = m == 0 ? ~0ull : t.k[0][rank_of(mid)];
      if ((k0 >> 56) < b) lo = mid + 1;
      else hi = mid;
    }
    dir[b] = static_cast<uint16_t>(lo);
  }
}

__global__ void __launch_bounds__(1024)
auto_splitter_kernel(const uint32_t* __restrict__ d_off, uint32_t W, Ws ws) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_off[kMaxW + 2];
  __shared__ BucketPlan p;
  const AutoView v = auto_view(ws, W);
  const uint32_t L = blockIdx.x + 1;
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    p = plan_for(s_off, L, v.cap);
    if (L == W) {
      const BucketPlan last = p;
      v.hdr->G = last.seg0 + last.g;
      v.hdr->spl_bytes = last.spl_off + spl_bytes_of(last.g, last.K);
      // the regions must fit the key and index areas
      if (last.r64 + static_cast<uint64_t>(last.g) * last.cap * last.K > v.size64 ||
          last.r32 + static_cast<uint64_t>(last.g) * last.cap > v.size32)
        set_error(ws.hdr, BSORT_E_WORKSPACE);
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < p.g; j += blockDim.x) {
    const uint32_t seg = p.seg0 + j;
    v.cursor[seg * kCursorStride] = 0;
    v.rcap[seg] = p.cap;
    v.segL[seg] = L;
    v.rbase[seg] = p.r64 + static_cast<uint64_t>(j) * p.cap * p.K;
    v.ibase[seg] = p.r32 + static_cast<uint64_t>(j) * p.cap;
  }
  if (p.g < 2) return;
  switch (p.K) {
    case 1: choose_splitters<1>(smem, v, p, L); break;
    case 2: choose_splitters<2>(smem, v, p, L); break;
    case 3: choose_splitters<3>(smem, v, p, L); break;
    default: choose_splitters<4>(smem, v, p, L); break;
  }
}

// ---------------------------------------------------------------------------
// 3. partition
// ---------------------------------------------------------------------------
// Segment of the element (key[0..K), idx) of bucket plan p: the number of
// splitters <= the element (splitters are sorted ascending).
template <int K>
__device__ __forceinline__ uint32_t find_segment(const uint8_t* tab, const BucketPlan& p,
                                                 const uint64_t (&key)[K], uint32_t idx) {
  const uint32_t ns = p.g - 1;
  const uint16_t* dir = reinterpret_cast<const uint16_t*>(tab + p.spl_off);
  const uint64_t* sk = reinterpret_cast<const uint64_t*>(tab + p.spl_off + kDirBytes);
  const uint32_t* si = reinterpret_cast<const uint32_t*>(sk + static_cast<size_t>(K) * ns);
  // splitters below dir[c] have a smaller first byte (all <= the element),
  // those from dir[c+1] on a larger one; search only between
  const uint32_t c = static_cast<uint32_t>(key[0] >> 56);
  uint32_t lo = dir[c], hi = dir[c + 1];  // answer in [lo, hi]
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;  // is splitter mid-1 <= element ?
    const uint32_t s = mid - 1;
    bool le = false, decided = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t a = sk[k * ns + s];
      if (!decided && a != key[k]) {
        le = a < key[k];
        decided = true;
      }
    }
    if (!decided) le = si[s] <= idx;
    if (le) lo = mid;
    else hi = mid - 1;
  }
  return p.seg0 + lo;
}

// Record words raw[0..K) (as loaded) of word i, length L -> big-endian masked
// keys in key[0..K) and the word's segment.
template <int K, int KW>
__device__ __forceinline__ uint32_t classify(uint64_t (&key)[KW], uint32_t i, uint32_t L,
                                             const BucketPlan& p, const uint8_t* tab) {
  uint64_t kk[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    kk[k] = bswap64(key[k]) & key_mask(L, k);
    key[k] = kk[k];
  }
  return p.g > 1 ? find_segment<K>(tab, p, kk, i) : p.seg0;
}

template <int KW>
__global__ void __launch_bounds__(kPartThreads, 2)
auto_partition_kernel(const uint8_t* __restrict__ rec, const uint8_t* __restrict__ len,
                      uint32_t n_cap, const uint32_t* __restrict__ d_n, uint32_t W,
                      const uint32_t* __restrict__ d_off, int retry_pass, Ws ws) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BucketPlan plans[kMaxW + 1];
  __shared__ uint32_t s_off[kMaxW + 2];
  const AutoView v = auto_view(ws, W);
  if (retry_pass && v.hdr->retry == 0) return;
  load_plans(plans, s_off, d_off, W, v.cap);
  // splitter table: staged in shared memory when it fits
  const uint32_t tb = v.hdr->spl_bytes;
  const uint8_t* tab = v.spl;
  if (tb <= kSplSmem) {
    const uint4* src = reinterpret_cast<const uint4*>(v.spl);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (uint32_t i = threadIdx.x; i < tb / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    tab = smem;
  }
  const uint32_t n = word_count(n_cap, d_n);
  const uint32_t lane = lane_id();
  bool overflow = false;
  constexpr uint32_t kPartWords = PartWords<KW>::value;
  const uint32_t warps_total = gridDim.x * (blockDim.x / 32);
  const uint32_t step = 32 * kPartWords;
  for (uint32_t base = (blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * step; base < n;
       base += warps_total * step) {
    uint32_t L[kPartWords], seg[kPartWords];
    uint64_t key[kPartWords][KW];
    // all loads first: kPartWords independent records per lane in flight
#pragma unroll
    for (uint32_t u = 0; u < kPartWords; ++u) {
      const uint32_t i = base + u * 32 + lane;
      const uint32_t l = i < n ? len[i] : 0u;
      L[u] = l > W ? 0u : l;
      const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + static_cast<uint64_t>(i) * W);
#pragma unroll
      for (int k = 0; k < KW; ++k) key[u][k] = L[u] ? __ldg(src + k) : 0ull;
    }
#pragma unroll
    for (uint32_t u = 0; u < kPartWords; ++u) {
      const uint32_t i = base + u * 32 + lane;
      seg[u] = 0xFFFFFFFFu;
      if (L[u]) {
        const BucketPlan& p = plans[L[u]];
        if (KW == 1 || p.K == 1) seg[u] = classify<1, KW>(key[u], i, L[u], p, tab);
        else if (KW == 2 || p.K == 2) seg[u] = classify<(KW >= 2 ? 2 : 1), KW>(key[u], i, L[u], p, tab);
        else if (KW == 3 || p.K == 3) seg[u] = classify<(KW >= 3 ? 3 : 1), KW>(key[u], i, L[u], p, tab);
        else seg[u] = classify<KW, KW>(key[u], i, L[u], p, tab);
      }
    }
    uint32_t peers[kPartWords], first[kPartWords];
#pragma unroll
    for (uint32_t u = 0; u < kPartWords; ++u) {
      peers[u] = __match_any_sync(0xffffffffu, seg[u]);
      first[u] = 0;
      if (seg[u] != 0xFFFFFFFFu && lane == __ffs(peers[u]) - 1)
        first[u] = atomicAdd(&v.cursor[seg[u] * kCursorStride], __popc(peers[u]));
    }
#pragma unroll
    for (uint32_t u = 0; u < kPartWords; ++u) {
      const uint32_t f = __shfl_sync(0xffffffffu, first[u], __ffs(peers[u]) - 1);
      if (seg[u] == 0xFFFFFFFFu) continue;
      const uint32_t pos = f + __popc(peers[u] & lanemask_lt());
      const BucketPlan& p = plans[L[u]];
      uint32_t rc;
      uint64_t rb, ib;
      if (!retry_pass) {
        // optimistic layout: a pure function of the bucket plan
        const uint32_t j = seg[u] - p.seg0;
        rc = p.cap;
        rb = p.r64 + static_cast<uint64_t>(j) * p.cap * p.K;
        ib = p.r32 + static_cast<uint64_t>(j) * p.cap;
      } else {
        rc = v.rcap[seg[u]];
        rb = v.rbase[seg[u]];
        ib = v.ibase[seg[u]];
      }
      if (pos < rc) {
#pragma unroll
        for (int k = 0; k < KW; ++k)
          if (k < static_cast<int>(p.K)) v.area64[rb + static_cast<uint64_t>(k) * rc + pos] = key[u][k];
        v.area32[ib + pos] = base + u * 32 + lane;
      } else {
        overflow = true;
      }
    }
  }
  if (overflow) atomicExch(&v.hdr->overflow, 1u);
}

// ---------------------------------------------------------------------------
// 4. layout: output bases; on overflow, exact regions for the retry pass
// ---------------------------------------------------------------------------
// Exact region (elements) for a segment of x words after a retry: a segment
// too large for shared memory gets a second half as merge scratch.
__device__ __forceinline__ uint32_t exact_region(uint32_t x, uint32_t K) {
  return x > auto_seg_cap(K) ? 2 * round4(x) : round4(x);
}

__global__ void __launch_bounds__(1024)
auto_layout_kernel(uint32_t W, Ws ws) {
  __shared__ uint32_t tmp[1024 / 32 + 1];
  const AutoView v = auto_view(ws, W);
  const uint32_t G = v.hdr->G;
  const bool redo = v.hdr->overflow != 0;
  const uint32_t per = (G + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = min(G, b + per);
  // exclusive scans of counts (output ranks) and, for a retry, of exact
  // regions (index area) and region x K (key area)
  uint32_t c = 0, c4 = 0, ck = 0;
  for (uint32_t j = b; j < e; ++j) {
    const uint32_t x = v.cursor[j * kCursorStride];
    const uint32_t K = keys_for_len(v.segL[j]);
    c += x;
    c4 += exact_region(x, K);
    ck += exact_region(x, K) * K;
  }
  uint32_t tot, tot4, totk;
  uint32_t run = block_exclusive_scan(c, tmp, &tot);
  uint32_t run4 = block_exclusive_scan(c4, tmp, &tot4);
  uint32_t runk = block_exclusive_scan(ck, tmp, &totk);
  const bool fits = tot4 <= v.size32 && totk <= v.size64;
  for (uint32_t j = b; j < e; ++j) {
    const uint32_t x = v.cursor[j * kCursorStride];
    const uint32_t K = keys_for_len(v.segL[j]);
    v.outbase[j] = run;
    run += x;
    if (redo && fits) {
      const uint32_t r = exact_region(x, K);
      v.rcap[j] = r;
      v.ibase[j] = run4;
      v.rbase[j] = runk;
      run4 += r;
      runk += r * K;
      v.cursor[j * kCursorStride] = 0;
    }
  }
  if (threadIdx.x == 0 && redo) {
    if (fits) v.hdr->retry = 1;
    else set_error(ws.hdr, BSORT_E_WORKSPACE);
  }
}

// ---------------------------------------------------------------------------
// 5. segment sort + gather
// ---------------------------------------------------------------------------
// Padded shared-memory position: one spare slot per 16 elements keeps the
// strided accesses of the merge rounds free of bank conflicts.
__device__ __forceinline__ uint32_t pad16(uint32_t i) { return i + (i >> 4); }

// Elements per thread of the one-key (key, index) merge sort.
template <int K> struct SegE { static constexpr int value = 8; };

__host__ __device__ constexpr size_t seg_plane_elems(uint32_t K) {
  // padded capacity: pad16(cap - 1) + 1 rounded up to an even count
  return (static_cast<size_t>(auto_seg_cap(K)) * 17 / 16 + 2) & ~static_cast<size_t>(1);
}

constexpr size_t kSegPlanesBytes = 104576;  // >= max over K of seg_plane_elems(K) x (8K + 4)

// One segment buffer per CTA (two CTAs per SM overlap each other's copies,
// sorts and stores): barrier + planes.
constexpr size_t kSegBufBytes = 16 + kSegPlanesBytes;
__host__ __device__ constexpr size_t segsort_smem_bytes() {
  return 128 + kSegBufBytes;  // alignment slack, buffer
}

template <int K>
__device__ __forceinline__ Elem<K> elem_inf() {
  Elem<K> e;
#pragma unroll
  for (int k = 0; k < K; ++k) e.k[k] = ~0ull;
  e.idx = ~0u;
  return e;
}

template <int K>
__device__ __forceinline__ void cswap(Elem<K>& a, Elem<K>& b) {
  if (elem_less<K>(b, a)) {
    const Elem<K> t = a;
    a = b;
    b = t;
  }
}

// Bitonic network on E registers (E a power of two), ascending.
template <int K, int E>
__device__ __forceinline__ void sort_regs(Elem<K> (&r)[E]) {
#pragma unroll
  for (int k = 2; k <= E; k <<= 1) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int j = i ^ (k - 1);
      if (j > i && (i & (k >> 1)) == 0) cswap<K>(r[i], r[j]);
    }
#pragma unroll
    for (int jj = k >> 2; jj > 0; jj >>= 1) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int j = i ^ jj;
        if (j > i) cswap<K>(r[i], r[j]);
      }
    }
  }
}

template <int K>
__device__ __forceinline__ void write_word(uint32_t W, uint8_t* out_rec, uint32_t* out_perm,
                                           uint32_t r, const Elem<K>& e) {
  const uint32_t KW = W / 8;
  uint64_t* dst = reinterpret_cast<uint64_t*>(out_rec + static_cast<uint64_t>(r) * W);
  if ((W & 15u) == 0) {
    for (uint32_t k = 0; k < KW; k += 2) {
      const uint64_t a = k < static_cast<uint32_t>(K) ? bswap64(e.k[k]) : 0ull;
      const uint64_t b = k + 1 < static_cast<uint32_t>(K) ? bswap64(e.k[k + 1]) : 0ull;
      reinterpret_cast<ulonglong2*>(dst)[k / 2] = make_ulonglong2(a, b);
    }
  } else {
    for (uint32_t k = 0; k < KW; ++k) dst[k] = k < static_cast<uint32_t>(K) ? bswap64(e.k[k]) : 0ull;
  }
  out_perm[r] = e.idx;
}

// Sorts the c elements held unpadded in t (planes of seg_plane_elems(K)) and
// writes them at output ranks ob.. .  Register sort of E elements per thread,
// then merge-path rounds through padded shared memory.  Only the first
// ceil(c / E) threads carry elements; positions at or past c read as +inf, so
// the work follows c, not the capacity.
template <int K, int E>
__device__ void block_merge_sort_out(const SmemTile<K>& t, uint32_t c, uint32_t W, uint32_t ob,
                                     uint8_t* out_rec, uint32_t* out_perm) {
  const uint32_t tid = threadIdx.x;
  const uint32_t active = (c + E - 1) / E;
  const bool act = tid < active;
  Elem<K> r[E];
  // thread tid takes positions tid*E .. tid*E+E-1, so the +inf padding sits
  // at the end of the last active thread's run only
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t i = tid * E + j;
    r[j] = (act && i < c) ? t.get(i) : elem_inf<K>();
  }
  if (act) sort_regs<K, E>(r);
  auto get = [&](uint32_t i) { return i < c ? t.get(pad16(i)) : elem_inf<K>(); };
  for (uint32_t R = E; R < c; R <<= 1) {
    __syncthreads();  // previous readers are done with shared memory
    if (act) {
#pragma unroll
      for (int j = 0; j < E; ++j)
        if (tid * E + j < c) t.put(pad16(tid * E + j), r[j]);
    }
    __syncthreads();
    if (act) {
      const uint32_t my = tid * E, ps = my & ~(2 * R - 1), d = my - ps;
      uint32_t lo = d > R ? d - R : 0u, hi = min(d, R);
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (elem_less<K>(get(ps + mid), get(ps + R + d - 1 - mid))) lo = mid + 1;
        else hi = mid;
      }
      uint32_t ia = ps + lo, ib = ps + R + (d - lo);
      const uint32_t ae = ps + R, be = ps + 2 * R;
      Elem<K> ha = ia < ae ? get(ia) : elem_inf<K>();
      Elem<K> hb = ib < be ? get(ib) : elem_inf<K>();
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const bool ta = elem_less<K>(ha, hb);
        r[j] = ta ? ha : hb;
        if (ta) {
          ++ia;
          ha = ia < ae ? get(ia) : elem_inf<K>();
        } else {
          ++ib;
          hb = ib < be ? get(ib) : elem_inf<K>();
        }
      }
    }
  }
  if (act) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t pos = tid * E + j;
      if (pos < c) write_word<K>(W, out_rec, out_perm, ob + pos, r[j]);
    }
  }
  __syncthreads();  // shared memory is reused by the next segment
}

// A segment larger than shared memory (only after a retry, whose region is
// data + scratch): sort chunks in shared memory, then merge runs pairwise with
// merge-path tiles, ping-ponging between the two halves.
template <int K>
__device__ void segsort_big(uint8_t* smem, const AutoView& v, uint32_t seg, uint32_t c,
                            uint32_t W, uint8_t* out_rec, uint32_t* out_perm) {
  const uint32_t rc = v.rcap[seg], half = rc / 2;
  const uint64_t rb = v.rbase[seg], ib = v.ibase[seg];
  SmemTile<K> a, b, t;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    a.k[k] = v.area64 + rb + static_cast<uint64_t>(k) * rc;
    b.k[k] = a.k[k] + half;
  }
  a.idx = v.area32 + ib;
  b.idx = a.idx + half;
  const uint32_t C = auto_seg_cap(K);
  uint64_t* kp = reinterpret_cast<uint64_t*>(smem);
#pragma unroll
  for (int k = 0; k < K; ++k) t.k[k] = kp + k * C;
  t.idx = reinterpret_cast<uint32_t*>(kp + static_cast<size_t>(K) * C);
  for (uint32_t c0 = 0; c0 < c; c0 += C) {
    const uint32_t m = min(C, c - c0);
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) t.put(i, a.get(c0 + i));
    __syncthreads();
    bitonic_flip<K>(t, m);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) a.put(c0 + i, t.get(i));
    __syncthreads();
  }
  const uint32_t part = K == 1 ? 4096u : K == 2 ? 2048u : 1024u;  // 2 x part elements fit smem
  SmemTile<K> src = a, dst = b;
  for (uint32_t R = C; R < c; R <<= 1) {
    for (uint32_t o0 = 0; o0 < c; o0 += part) merge_tile<K>(smem, part, src, dst, c, R, o0);
    const SmemTile<K> x = src;
    src = dst;
    dst = x;
  }
  const uint32_t ob = v.outbase[seg];
  for (uint32_t r = threadIdx.x; r < c; r += blockDim.x)
    write_word<K>(W, out_rec, out_perm, ob + r, src.get(r));
  __syncthreads();
}

// Issues the bulk copies (TMA) of segment seg (c <= capacity) into buffer buf.
template <int K>
__device__ void prefetch_segment(uint8_t* buf, const AutoView& v, uint32_t seg, uint32_t c) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf);
  uint64_t* kp = reinterpret_cast<uint64_t*>(buf + 16);
  const uint32_t C = static_cast<uint32_t>(seg_plane_elems(K));
  uint32_t* ip = reinterpret_cast<uint32_t*>(kp + static_cast<size_t>(K) * C);
  const uint32_t rc = v.rcap[seg];
  const uint64_t rb = v.rbase[seg], ib = v.ibase[seg];
  // regions start 16-byte aligned (rcap, rbase, ibase are multiples of 4) and
  // hold rcap >= round4(c) elements, so the rounded copies stay inside
  const uint32_t kbytes = (c * 8 + 15) & ~15u, ibytes = (c * 4 + 15) & ~15u;
  mbar_arrive_expect_tx(bar, K * kbytes + ibytes);
#pragma unroll
  for (int k = 0; k < K; ++k)
    bulk_g2s(kp + k * C, v.area64 + rb + static_cast<uint64_t>(k) * rc, kbytes, bar);
  bulk_g2s(ip, v.area32 + ib, ibytes, bar);
}

__device__ __forceinline__ uint32_t seg_count(const AutoView& v, uint32_t seg) {
  return min(v.cursor[seg * kCursorStride], v.rcap[seg]);
}

// Thread 0: start the copy of segment `seg` into `buf` when it will be sorted
// from shared memory; returns whether a copy was issued.
__device__ bool maybe_prefetch(uint8_t* buf, const AutoView& v, uint32_t seg, uint32_t G) {
  if (seg >= G) return false;
  const uint32_t c = seg_count(v, seg);
  const uint32_t K = keys_for_len(v.segL[seg]);
  if (c == 0 || c > auto_seg_cap(K)) return false;
  switch (K) {
    case 1: prefetch_segment<1>(buf, v, seg, c); break;
    case 2: prefetch_segment<2>(buf, v, seg, c); break;
    case 3: prefetch_segment<3>(buf, v, seg, c); break;
    default: prefetch_segment<4>(buf, v, seg, c); break;
  }
  return true;
}

// ---- one-word composite elements -----------------------------------------
// A one-key segment whose keys (without their zero tail bytes) span at most
// kb bits and whose indices fit ib bits, with kb + ib <= 64, sorts as single
// uint64 values ((key >> shift) - kmin) << ib | idx: the integer order of the
// composites is the (key, index) order.

__device__ __forceinline__ void cswap64(uint64_t& a, uint64_t& b) {
  const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}

template <int E>
__device__ __forceinline__ void sort_regs64(uint64_t (&r)[E]) {
#pragma unroll
  for (int k = 2; k <= E; k <<= 1) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int j = i ^ (k - 1);
      if (j > i && (i & (k >> 1)) == 0) cswap64(r[i], r[j]);
    }
#pragma unroll
    for (int jj = k >> 2; jj > 0; jj >>= 1) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int j = i ^ jj;
        if (j > i) cswap64(r[i], r[j]);
      }
    }
  }
}

// Register bitonic sort of N = E * blockDim.x positions, blocked layout:
// thread t holds positions t*E .. t*E+E-1 in r[].  All-ascending form: for
// each block size k the first step pairs i with i ^ (k-1), the next ones pair
// i with i ^ j (j = k/4 .. 1); the lower position keeps the smaller value.
// A partner in the same thread is compared in registers, one in the same warp
// through __shfl_xor_sync, one in another warp through shared memory.  Every
// compare-exchange of a step is independent, so all threads and warps work in
// every step.  Ops supplies the element order, the warp shuffle and the
// shared-memory exchange slots (padded positions).

// Plain uint64 composites; exchange slots in plane[].
struct U64Ops {
  using T = uint64_t;
  uint64_t* plane;
  __device__ static bool less(uint64_t a, uint64_t b) { return a < b; }
  __device__ static uint64_t shfl(uint64_t x, uint32_t m) { return __shfl_xor_sync(0xffffffffu, x, m); }
  __device__ static uint64_t inf() { return ~0ull; }
  __device__ void st(uint32_t i, uint64_t v) const { plane[pad16(i)] = v; }
  __device__ uint64_t ld(uint32_t i) const { return plane[pad16(i)]; }
};

// (key words, index) elements; exchange slots in the tile's planes.
template <int K>
struct ElemOps {
  using T = Elem<K>;
  SmemTile<K> t;
  __device__ static bool less(const Elem<K>& a, const Elem<K>& b) { return elem_less<K>(a, b); }
  __device__ static Elem<K> shfl(const Elem<K>& x, uint32_t m) {
    Elem<K> y;
#pragma unroll
    for (int k = 0; k < K; ++k) y.k[k] = __shfl_xor_sync(0xffffffffu, x.k[k], m);
    y.idx = __shfl_xor_sync(0xffffffffu, x.idx, m);
    return y;
  }
  __device__ static Elem<K> inf() { return elem_inf<K>(); }
  __device__ void st(uint32_t i, const Elem<K>& v) const { t.put(pad16(i), v); }
  __device__ Elem<K> ld(uint32_t i) const { return t.get(pad16(i)); }
};

template <typename Ops, int M, int E>
__device__ __forceinline__ void reg_step(typename Ops::T (&r)[E]) {
  if constexpr (M < E) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      constexpr int m = M;
      const int q = j ^ m;
      if (q > j && Ops::less(r[q], r[j])) {
        const typename Ops::T x = r[j];
        r[j] = r[q];
        r[q] = x;
      }
    }
  }
}

template <typename Ops, int E>
__device__ __forceinline__ void bitonic_step(typename Ops::T (&r)[E], const Ops& ops, uint32_t mask) {
  using T = typename Ops::T;
  constexpr uint32_t LE = E == 2 ? 1 : E == 4 ? 2 : E == 8 ? 3 : 4;
  const uint32_t tid = threadIdx.x;
  const uint32_t lane_mask = mask >> LE;
  if (mask < E) {
    // in registers: masks are the flips 1, 3, 7, 15 or the cleaners 1, 2, 4, 8
    switch (mask) {
      case 1: reg_step<Ops, 1, E>(r); break;
      case 2: reg_step<Ops, 2, E>(r); break;
      case 3: reg_step<Ops, 3, E>(r); break;
      case 4: reg_step<Ops, 4, E>(r); break;
      case 7: reg_step<Ops, 7, E>(r); break;
      case 8: reg_step<Ops, 8, E>(r); break;
      default: reg_step<Ops, 15, E>(r); break;
    }
  } else if (lane_mask < 32) {
    // across lanes of one warp; my position is the upper one of its pair when
    // the highest bit of the lane part of the mask is set in my lane
    const uint32_t top = 1u << (31 - __clz(lane_mask));
    const bool keep_small = (tid & top) == 0;
    if ((mask & (E - 1)) == 0) {
      // cleaner step: the partner holds the same slot j
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const T other = Ops::shfl(r[j], lane_mask);
        if (Ops::less(other, r[j]) == keep_small) r[j] = other;
      }
    } else {
      // flip step (mask = k - 1): slot j pairs with the partner's slot E-1-j.
      // Slots j and E-1-j are exchanged together: sending slot E-1-j delivers
      // the partner's value for my slot j, sending slot j the one for E-1-j.
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        const T for_j = Ops::shfl(r[E - 1 - j], lane_mask);
        const T for_m = Ops::shfl(r[j], lane_mask);
        if (Ops::less(for_j, r[j]) == keep_small) r[j] = for_j;
        if (Ops::less(for_m, r[E - 1 - j]) == keep_small) r[E - 1 - j] = for_m;
      }
    }
  } else {
    // across warps: exchange through shared memory
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) ops.st(tid * E + j, r[j]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t i = tid * E + j, pi = i ^ mask;
      const T other = ops.ld(pi);
      if (Ops::less(other, r[j]) == (i < pi)) r[j] = other;
    }
  }
}

// Sorts the first c values (read by get(i), unpadded) with a register bitonic
// network of E per thread and hands them to sink(pos, value).  Needs
// c <= E * blockDim.x; ops' exchange slots must hold pad16(E*blockDim.x - 1) + 1.
template <typename Ops, int E, typename Get, typename Sink>
__device__ void block_sort(const Ops& ops, uint32_t c, Get get, Sink sink) {
  using T = typename Ops::T;
  const uint32_t tid = threadIdx.x;
  T r[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t i = tid * E + j;
    r[j] = i < c ? get(i) : Ops::inf();
  }
  uint32_t N = 2;
  while (N < c) N <<= 1;
  if (N < E) N = E;
  for (uint32_t k = 2; k <= N; k <<= 1) {
    bitonic_step<Ops, E>(r, ops, k - 1);
    for (uint32_t j = k >> 2; j > 0; j >>= 1) bitonic_step<Ops, E>(r, ops, j);
  }
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (tid * E + j < c) sink(tid * E + j, r[j]);
  __syncthreads();
}

// LSD radix sort of c uint64 values on their low `bits` bits, 8 bits per
// pass, stable: each pass counts digits per warp over warp-contiguous ranges
// (warp w owns positions [w S, (w+1) S)), scans the (digit, warp) counts in
// digit-major order, then every warp writes its values in position order to
// base[digit][warp] + (earlier equal digits in the warp).  A and B hold c
// values each (A the input), hist 16 x 256 counters (one row per warp of a
// 512-thread block).  Returns the array holding the result.
constexpr uint32_t kRadixWarps = kSegThreads / 32;
constexpr uint32_t kRadixMaxC = 5504;  // A, B and hist fit one segment buffer

__device__ uint64_t* block_radix_u64(uint64_t* A, uint64_t* B, uint32_t* hist, uint32_t c,
                                     uint32_t bits) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t S = ((c + kRadixWarps - 1) / kRadixWarps + 31) / 32 * 32;
  const uint32_t w0 = min(c, warp * S), w1 = min(c, w0 + S);
  uint32_t* row = hist + warp * 256;
  uint64_t* src = A;
  uint64_t* dst = B;
  for (uint32_t shift = 0; shift < bits; shift += 8) {
    for (uint32_t i = threadIdx.x; i < kRadixWarps * 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // 1. counts per (warp, digit)
    for (uint32_t b = w0; b < w1; b += 32) {
      const uint32_t pos = b + lane;
      const bool valid = pos < w1;
      const uint32_t d = valid ? static_cast<uint32_t>(src[pos] >> shift) & 255u : 256u + lane;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (valid && lane == __ffs(peers) - 1) row[d] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // 2. exclusive scan in digit-major, warp-minor order (entry d * 16 + w)
    {
      __shared__ uint32_t tmp[kSegThreads / 32 + 1];
      constexpr uint32_t per = kRadixWarps * 256 / kSegThreads;  // 8 entries per thread
      uint32_t v[per], sum = 0;
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) {
        const uint32_t e = threadIdx.x * per + k, d = e / kRadixWarps, w = e % kRadixWarps;
        v[k] = hist[w * 256 + d];
        sum += v[k];
      }
      uint32_t tot;
      uint32_t run = block_exclusive_scan(sum, tmp, &tot);
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) {
        const uint32_t e = threadIdx.x * per + k, d = e / kRadixWarps, w = e % kRadixWarps;
        hist[w * 256 + d] = run;
        run += v[k];
      }
    }
    __syncthreads();
    // 3. stable scatter
    for (uint32_t b = w0; b < w1; b += 32) {
      const uint32_t pos = b + lane;
      const bool valid = pos < w1;
      const uint64_t x = valid ? src[pos] : 0ull;
      const uint32_t d = valid ? static_cast<uint32_t>(x >> shift) & 255u : 256u + lane;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (valid) dst[row[d] + __popc(peers & lanemask_lt())] = x;
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) row[d] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y < x ? y : x;
  }
  return x;
}
__device__ __forceinline__ uint64_t warp_max64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

// Segments of words with two or more key words (longer than 8 letters, a
// small share of typical text): bitonic network in shared memory, which keeps
// no elements in registers.
template <int K>
__device__ void sort_resident(uint8_t* buf, const AutoView& v, uint32_t seg, uint32_t c,
                              uint32_t W, uint8_t* out_rec, uint32_t* out_perm) {
  uint64_t* kp = reinterpret_cast<uint64_t*>(buf + 16);
  const uint32_t C = static_cast<uint32_t>(seg_plane_elems(K));
  SmemTile<K> t;
#pragma unroll
  for (int k = 0; k < K; ++k) t.k[k] = kp + k * C;
  t.idx = reinterpret_cast<uint32_t*>(kp + static_cast<size_t>(K) * C);
  bitonic_flip<K>(t, c);
  __syncthreads();
  const uint32_t ob = v.outbase[seg];
  for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) write_word<K>(W, out_rec, out_perm, ob + r, t.get(r));
  __syncthreads();
}

// One-key segment of length-L words resident in buf: composite sort when the
// key span and index width fit 64 bits, else the (key, index) merge sort.
__device__ void sort_resident_k1(uint8_t* buf, const AutoView& v, uint32_t seg, uint32_t c,
                                 uint32_t L, uint32_t W, uint8_t* out_rec, uint32_t* out_perm) {
  __shared__ uint64_t red[3][kSegThreads / 32];
  __shared__ uint64_t s_kmin;
  __shared__ uint32_t s_kb, s_ib;
  uint64_t* kp = reinterpret_cast<uint64_t*>(buf + 16);
  const uint32_t C = static_cast<uint32_t>(seg_plane_elems(1));
  uint32_t* ip = reinterpret_cast<uint32_t*>(kp + C);
  const uint32_t shift = 64 - 8 * L;  // L <= 8: the low 64-8L key bits are zero
  uint64_t kmin = ~0ull, kmax = 0, imax = 0;
  for (uint32_t i = threadIdx.x; i < c; i += blockDim.x) {
    const uint64_t k = kp[i] >> shift;
    kmin = k < kmin ? k : kmin;
    kmax = k > kmax ? k : kmax;
    imax = ip[i] > imax ? ip[i] : imax;
  }
  kmin = warp_min64(kmin);
  kmax = warp_max64(kmax);
  imax = warp_max64(imax);
  const uint32_t warp = threadIdx.x >> 5;
  if (lane_id() == 0) {
    red[0][warp] = kmin;
    red[1][warp] = kmax;
    red[2][warp] = imax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t a = ~0ull, b = 0, m = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
      a = red[0][w] < a ? red[0][w] : a;
      b = red[1][w] > b ? red[1][w] : b;
      m = red[2][w] > m ? red[2][w] : m;
    }
    s_kmin = a;
    s_kb = b == a ? 0u : 64u - static_cast<uint32_t>(__clzll(b - a));
    s_ib = 32u - static_cast<uint32_t>(__clz(static_cast<uint32_t>(m) | 1u));
  }
  __syncthreads();
  const uint32_t kb = s_kb, ib = s_ib;
  const uint64_t k0 = s_kmin;
  const uint32_t ob = v.outbase[seg];
  if (kb + ib <= 64) {
    for (uint32_t i = threadIdx.x; i < c; i += blockDim.x)
      kp[i] = (((kp[i] >> shift) - k0) << ib) | ip[i];
    __syncthreads();
    const uint64_t imask = (1ull << ib) - 1;
    auto sink = [&](uint32_t pos, uint64_t x) {
      Elem<1> e;
      e.k[0] = ((x >> ib) + k0) << shift;
      e.idx = static_cast<uint32_t>(x & imask);
      write_word<1>(W, out_rec, out_perm, ob + pos, e);
    };
    if (c <= kRadixMaxC) {
      // A = composites over the key plane; B and the counters reuse the (now
      // dead) rest of the buffer
      uint64_t* B = kp + kRadixMaxC;
      uint32_t* hist = reinterpret_cast<uint32_t*>(kp + 2 * kRadixMaxC);
      const uint64_t* res = block_radix_u64(kp, B, hist, c, kb + ib);
      for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) sink(r, res[r]);
      __syncthreads();
      return;
    }
    const U64Ops ops{kp};
    auto get = [&](uint32_t i) { return kp[i]; };
    // reads happen before the first exchange writes (each step syncs first)
    if (c <= 4 * blockDim.x) block_sort<U64Ops, 4>(ops, c, get, sink);
    else if (c <= 8 * blockDim.x) block_sort<U64Ops, 8>(ops, c, get, sink);
    else block_sort<U64Ops, 16>(ops, c, get, sink);
  } else {
    SmemTile<1> t;
    t.k[0] = kp;
    t.idx = ip;
    const ElemOps<1> ops{t};
    auto get = [&](uint32_t i) { return t.get(i); };
    auto sink = [&](uint32_t pos, const Elem<1>& e) { write_word<1>(W, out_rec, out_perm, ob + pos, e); };
    if (c <= 4 * blockDim.x) block_sort<ElemOps<1>, 4>(ops, c, get, sink);
    else if (c <= 8 * blockDim.x) block_sort<ElemOps<1>, 8>(ops, c, get, sink);
    else {
      // rare: a wide-key segment above 4096 words
      bitonic_flip<1>(t, c);
      __syncthreads();
      for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) write_word<1>(W, out_rec, out_perm, ob + r, t.get(r));
      __syncthreads();
    }
  }
}

// Persistent CTAs (two per SM) walk the segments: bulk-copy the segment into
// shared memory, sort, write the output records and permutation.
__global__ void __launch_bounds__(kSegThreads, 2)
auto_segsort_kernel(uint32_t W, Ws ws, uint8_t* __restrict__ out_rec,
                    uint32_t* __restrict__ out_perm) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* buf = align128(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf);
  const AutoView v = auto_view(ws, W);
  const uint32_t G = v.hdr->G;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  for (uint32_t seg = blockIdx.x; seg < G; seg += gridDim.x) {
    const uint32_t c = seg_count(v, seg);
    const uint32_t L = v.segL[seg];
    const uint32_t K = keys_for_len(L);
    if (c == 0) continue;
    if (c > auto_seg_cap(K)) {
      // larger than shared memory (after a retry): chunked sort + merges
      uint8_t* scratch = buf + 16;
      switch (K) {
        case 1: segsort_big<1>(scratch, v, seg, c, W, out_rec, out_perm); break;
        case 2: segsort_big<2>(scratch, v, seg, c, W, out_rec, out_perm); break;
        case 3: segsort_big<3>(scratch, v, seg, c, W, out_rec, out_perm); break;
        default: segsort_big<4>(scratch, v, seg, c, W, out_rec, out_perm); break;
      }
      continue;
    }
    // earlier generic-proxy use of the buffer must be ordered before the bulk
    // copy (async proxy) overwrites it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) maybe_prefetch(buf, v, seg, G);
    const bool ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        set_error(ws.hdr, BSORT_E_TIMEOUT);
        mbar_wait_bounded(bar, phase ^ 1u);  // let the copy in flight land before exiting
      }
      return;
    }
    switch (K) {
      case 1: sort_resident_k1(buf, v, seg, c, L, W, out_rec, out_perm); break;
      case 2: sort_resident<2>(buf, v, seg, c, W, out_rec, out_perm); break;
      case 3: sort_resident<3>(buf, v, seg, c, W, out_rec, out_perm); break;
      default: sort_resident<4>(buf, v, seg, c, W, out_rec, out_perm); break;
    }
  }
}

// ---------------------------------------------------------------------------
// 0. length histogram (totals only) and bucket offsets
// ---------------------------------------------------------------------------
constexpr uint32_t kHistThreads = 256;

// Each thread counts in its own shared-memory column (no contention), then
// the block adds its column sums to the global totals: one atomic per length
// per block.
__global__ void __launch_bounds__(kHistThreads)
auto_hist_kernel(const uint8_t* __restrict__ len, uint32_t n_cap, const uint32_t* __restrict__ d_n,
                 uint32_t W, Ws ws) {
  __shared__ uint32_t cnt[kBins][kHistThreads];
  const AutoView v = auto_view(ws, W);
  for (uint32_t L = 0; L < kBins; ++L) cnt[L][threadIdx.x] = 0;
  const uint32_t n = word_count(n_cap, d_n);
  bool bad_zero = false, bad_long = false;
  const uint32_t stride = gridDim.x * kHistThreads;
  if ((reinterpret_cast<uintptr_t>(len) & 3u) == 0) {
    const uint32_t n4 = n / 4;
    const uchar4* l4 = reinterpret_cast<const uchar4*>(len);
    for (uint32_t q = blockIdx.x * kHistThreads + threadIdx.x; q < n4; q += stride) {
      const uchar4 b = __ldg(l4 + q);
      const uint32_t ls[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t L = ls[k];
        bad_zero |= L == 0;
        bad_long |= L > W;
        if (L >= 1 && L <= W) ++cnt[L][threadIdx.x];
      }
    }
    for (uint32_t i = 4 * n4 + blockIdx.x * kHistThreads + threadIdx.x; i < n; i += stride) {
      const uint32_t L = len[i];
      bad_zero |= L == 0;
      bad_long |= L > W;
      if (L >= 1 && L <= W) ++cnt[L][threadIdx.x];
    }
  } else {
    for (uint32_t i = blockIdx.x * kHistThreads + threadIdx.x; i < n; i += stride) {
      const uint32_t L = len[i];
      bad_zero |= L == 0;
      bad_long |= L > W;
      if (L >= 1 && L <= W) ++cnt[L][threadIdx.x];
    }
  }
  __syncthreads();
  // warp w sums lengths w, w + 8, ...: lanes add 8 columns each, then reduce
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  for (uint32_t L = 1 + warp; L <= W; L += kHistThreads / 32) {
    uint32_t sum = 0;
    for (uint32_t j = lane; j < kHistThreads; j += 32) sum += cnt[L][j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0 && sum) atomicAdd(&v.hdr->total[L], sum);
  }
  if (bad_zero) set_error(ws.hdr, BSORT_E_INVALID);
  if (bad_long) set_error(ws.hdr, BSORT_E_WORD_TOO_LONG);
}

// Bucket offsets off[L] (words shorter than L) from the totals; also resets
// the per-call state of the sample sort.
__global__ void auto_offsets_kernel(uint32_t W, Ws ws, uint32_t* __restrict__ off) {
  __shared__ uint32_t tot[kBins];
  const AutoView v = auto_view(ws, W);
  const uint32_t L = threadIdx.x;
  if (L < kBins) tot[L] = (L >= 1 && L <= W) ? v.hdr->total[L] : 0u;
  __syncthreads();
  if (L <= W + 1) {
    uint32_t s = 0;
    for (uint32_t l = 1; l < L && l <= W; ++l) s += tot[l];
    off[L] = s;
  }
  if (L < kMaxW + 2) ws.hdr->final_buf[L] = 0;
  if (L < kBins) v.hdr->samp_cnt[L] = 0;
  if (L == 0) {
    v.hdr->overflow = 0;
    v.hdr->retry = 0;
  }
}

static_assert(seg_plane_elems(1) * 12 <= kSegPlanesBytes && seg_plane_elems(2) * 20 <= kSegPlanesBytes &&
                  seg_plane_elems(3) * 28 <= kSegPlanesBytes && seg_plane_elems(4) * 36 <= kSegPlanesBytes,
              "segment planes exceed the shared-memory budget");
static_assert(16 * kSegThreads >= 8192, "composite E x threads must cover the segment capacity");
static_assert((2 * kRadixMaxC * 8 + kRadixWarps * 256 * 4) <= kSegPlanesBytes,
              "radix buffers exceed the segment buffer");
static_assert(kRadixMaxC * 8 <= seg_plane_elems(1) * 8,
              "the composite input must lie inside the key plane");
static_assert(2 * (segsort_smem_bytes() + 1024) <= 228 * 1024, "two segsort CTAs must fit an SM");

int g_sm_count = 0;

template <int KW>
cudaError_t launch_partition(const uint8_t* rec, const uint8_t* len, uint32_t n_cap,
                             const uint32_t* d_n, uint32_t W, const uint32_t* d_off, const Ws& ws,
                             int retry, cudaStream_t s) {
  static size_t set = 0;
  cudaError_t e = ensure_smem(auto_partition_kernel<KW>, kSplSmem, &set);
  if (e != cudaSuccess) return e;
  const uint32_t grid = static_cast<uint32_t>(g_sm_count) * 2;
  BSORT_LAUNCH(retry ? "auto_partition_retry" : "auto_partition", auto_partition_kernel<KW>, grid,
               kPartThreads, kSplSmem, s, rec, len, n_cap, d_n, W, d_off, retry, ws);
  return cudaGetLastError();
}

cudaError_t partition(const uint8_t* rec, const uint8_t* len, uint32_t n_cap, const uint32_t* d_n,
                      uint32_t W, const uint32_t* d_off, const Ws& ws, int retry, cudaStream_t s) {
  switch (W / 8) {
    case 1: return launch_partition<1>(rec, len, n_cap, d_n, W, d_off, ws, retry, s);
    case 2: return launch_partition<2>(rec, len, n_cap, d_n, W, d_off, ws, retry, s);
    case 3: return launch_partition<3>(rec, len, n_cap, d_n, W, d_off, ws, retry, s);
    default: return launch_partition<4>(rec, len, n_cap, d_n, W, d_off, ws, retry, s);
  }
}

}  // namespace

bool auto_applies(uint32_t n_cap, const Ws& ws, uint32_t W) {
  (void)W;
  // u32 region offsets in the layout scan stay below 2^32 for n < 2^28
  return n_cap >= kAutoMinWords && n_cap < (1u << 28) &&
         ws.cap >= static_cast<uint64_t>(n_cap) + 64 && ws.cap >= kAutoMinWords + 64;
}

cudaError_t launch_auto(const uint8_t* rec, const uint8_t* len, uint32_t n_cap,
                        const uint32_t* d_n, uint32_t W, uint32_t* d_off, const Ws& ws,
                        uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s) {
  static size_t split_set = 0, seg_set = 0;
  const size_t split_smem = 16384 * 12;  // max over K of auto_sample_max(K) x (8K + 4)
  cudaError_t e = ensure_smem(auto_splitter_kernel, split_smem, &split_set);
  if (e == cudaSuccess) e = ensure_smem(auto_segsort_kernel, segsort_smem_bytes(), &seg_set);
  if (e != cudaSuccess) return e;
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 148;
  }
  const uint32_t samples = n_cap / kAutoSampleEvery + 1;
  // phase 2 counts: totals per length, then bucket offsets
  const AutoView v = auto_view(ws, W);
  e = cudaMemsetAsync(v.hdr->total, 0, sizeof(v.hdr->total), s);
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("auto_hist", auto_hist_kernel, static_cast<uint32_t>(g_sm_count) * 4, kHistThreads,
               0, s, len, n_cap, d_n, W, ws);
  BSORT_LAUNCH("auto_offsets", auto_offsets_kernel, 1, 64, 0, s, W, ws, d_off);
  BSORT_LAUNCH("auto_sample", auto_sample_kernel, (samples + 255) / 256, 256, 0, s, rec, len,
               n_cap, d_n, W, d_off, ws);
  BSORT_LAUNCH("auto_splitters", auto_splitter_kernel, W, 1024, split_smem, s, d_off, W, ws);
  e = partition(rec, len, n_cap, d_n, W, d_off, ws, 0, s);
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("auto_layout", auto_layout_kernel, 1, 1024, 0, s, W, ws);
  e = partition(rec, len, n_cap, d_n, W, d_off, ws, 1, s);
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("auto_segsort", auto_segsort_kernel, static_cast<uint32_t>(g_sm_count) * 2,
               kSegThreads, segsort_smem_bytes(), s, W, ws, out_rec, out_perm);
  return cudaGetLastError();
}

}  // namespace bsort
