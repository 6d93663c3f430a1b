// Sample-sort strategy for large inputs (BSORT_AUTO in the one-call paths).
//
// Same answer as the paper's phases 2-3 and the concatenation (§3
// Methodology, "Pre-processing"): every word ordered by (length, bytes, input
// index).  Phase 2's length buckets are refined into key-range segments small
// enough for one CTA's shared memory, so each word crosses HBM a fixed number
// of times instead of once per merge pass:
//
//   auto_hist_kernel       words per length (phase 2's counts)
//   auto_offsets_kernel    bucket offsets and every bucket's segment plan
//   auto_sample_kernel     stratified sample (one position per 32 words, kept
//                          with probability 1/4, 1/2, 1 for 1, 2, >= 3 key
//                          words: about 20 samples per expected segment),
//                          grouped by length bucket
//   auto_bucket_kernel     phase 2's sub-arrays: every word's key words and
//                          index go to its length's staging planes; the AND
//                          and OR of all bytes inside words bound their range
//   auto_spl_sort_kernel   eight CTAs per bucket sort chunks of its samples
//   auto_spl_select_kernel each sample's rank across the sorted chunks (binary
//                          search) picks the g_L - 1 splitters by (keys,
//                          index), so a word repeated many times is split
//                          evenly by index
//   auto_spl_dir_kernel    per bucket, the splitters' directory (two-byte
//                          codes) and every segment's byte-code record, taken
//                          from its two bounding splitters
//   auto_partition_kernel  tiles of a bucket: every word finds its segment
//                          (directory, then binary search over the splitters
//                          staged in shared memory), counts per segment in the
//                          tile, one reservation per (tile, segment); a slot
//                          past the region's end only counts and raises the
//                          overflow flag
//   auto_layout_kernel     output base of every segment (scan of the exact
//                          counts); on overflow, exact regions for a retry
//   auto_partition_kernel  (again) the retry pass, a no-op unless overflow
//   auto_segsort_kernel    persistent CTAs take segments from a counter:
//                          bulk-copy (TMA) the segment into shared memory,
//                          recode one- and two-key words with the segment's
//                          byte code, sort the (code, index) items by a
//                          counting pass and rank placement within buckets
//                          (overfull buckets split again in shared memory;
//                          LSD radix passes only past the split area), sort
//                          longer keys with a bitonic network, and write the
//                          final records and permutation at the segment's
//                          output base (or, for the packed calls, each word's
//                          bytes and offset in the §3.1 form); a segment larger
//                          than shared memory (only after a retry) is sorted in
//                          chunks and merged in global memory
#include <type_traits>

#include "block_scan.cuh"
#include "common.cuh"
#include "kernels.h"
#include "sort_impl.cuh"

namespace bsort {

namespace {

constexpr uint32_t kSegThreads = 512;
// One cursor per 128-byte line: the partition's atomics then spread over all
// L2 slices instead of piling onto the few lines a packed array would use.
constexpr uint32_t kCursorStride = 32;


// ---------------------------------------------------------------------------
// Device view of the AUTO area
// ---------------------------------------------------------------------------
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

struct AutoHdr {
  uint32_t overflow;        // a partition slot fell past its region
  uint32_t retry;           // the retry pass is armed
  uint32_t G;               // segments in total
  uint32_t spl_bytes;       // bytes of the splitter table
  uint32_t samp_cnt[kBins]; // samples drawn per bucket (may exceed capacity)
  uint32_t total[kBins];    // words per length (the histogram of phase 2)
  uint32_t bcur[kBins];     // staging slots taken per length bucket
  uint32_t next_seg;        // segments handed out to the sorting CTAs
  uint32_t band, bor;       // AND and OR of every byte inside a word: bounds of their range
  uint32_t imax;            // largest word index
  BucketPlan plans[kBins];  // per length bucket, from the offsets
};
static_assert(sizeof(AutoHdr) <= 4096, "the header fits its page of the AUTO area");

struct AutoView {
  AutoHdr* hdr;
  uint64_t* samp64;   // per bucket L: K_L planes of sample keys (scap each)
  uint32_t* samp32;   // per bucket L: sample indices
  uint8_t* spl;       // splitter table: per bucket, K_L key planes then indices
  uint32_t* cursor;   // per segment: slots taken, at cursor[seg * kCursorStride]
  uint32_t* rcap;     // per segment: region capacity (elements)
  uint32_t* outbase;  // per segment: first output rank
  uint32_t* segL;     // per segment: its length bucket
  uint32_t* segf;     // per segment: byte code fields, code width, index width (kSegFWords)
  uint64_t* stage64;  // per bucket L: K_L planes of its words' keys (count_L each)
  uint32_t* stage32;  // per bucket L: its words' indices, at the bucket offset
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
  o += 4 * G;
  v.segf = reinterpret_cast<uint32_t*>(p + o);
  o += 4 * kSegFWords * G;
  // staging planes: per bucket L, K_L key planes then (separately) the indices
  o = align_up(o, 256);
  v.stage64 = reinterpret_cast<uint64_t*>(p + o);
  o += align_up(8 * (cap + 64) * KW, 256);
  v.stage32 = reinterpret_cast<uint32_t*>(p + o);
  v.area64 = ws.keys[0];
  v.area32 = ws.idx[0];
  const uint64_t third = cap >= kAutoMinWords + 64 ? cap + kAutoSlack : 0;
  v.size64 = (2 * cap + third) * KW;
  v.size32 = 2 * cap + third;
  v.cap = cap;
  return v;
}


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
static_assert(kDirBytes >= 2 * (kAutoDir2Max + 1) && kDirBytes >= 2 * 257 && kDirBytes % 16 == 0,
              "the directory area holds either directory, 16-byte aligned");

// Directory code of a first key word.  Bytes fall into r classes: 0 below
// band (a word's zero tail), 1 .. r-1 for band .. bor (and above, only in the
// all-ones splitters of an unsampled bucket).  When r^2 <= kAutoDir2Max the
// code is the class pair of the first two bytes, c0 r + c1, else the first
// byte; either way it never decreases as the key grows, so a bucket's sorted
// splitters have sorted codes, and a splitter whose code differs from an
// element's compares with it as the codes do.
struct DirShape {
  uint32_t band, r;
  bool two;
};
__device__ __forceinline__ DirShape dir_shape(const AutoHdr* h) {
  const uint32_t band = h->band, bor = h->bor;
  const uint32_t r = bor >= band ? bor - band + 2 : 2u;
  return DirShape{band, r, r * r <= kAutoDir2Max};
}
__device__ __forceinline__ uint32_t dir_class(uint32_t b, const DirShape& d) {
  return b < d.band ? 0u : min(b - d.band + 1, d.r - 1);
}
__device__ __forceinline__ uint32_t dir_code(uint64_t k0, const DirShape& d) {
  const uint32_t b0 = static_cast<uint32_t>(k0 >> 56);
  if (!d.two) return b0;
  return dir_class(b0, d) * d.r + dir_class(static_cast<uint32_t>(k0 >> 48) & 255u, d);
}
__device__ __forceinline__ uint32_t dir_entries(const DirShape& d) { return d.two ? d.r * d.r : 256u; }

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
                           const AutoHdr* hdr) {
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  if (threadIdx.x >= 1 && threadIdx.x <= W) plans[threadIdx.x] = hdr->plans[threadIdx.x];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// 1. sample
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
auto_sample_kernel(const uint8_t* __restrict__ rec, const uint8_t* __restrict__ len,
                   uint32_t n_cap, const uint32_t* __restrict__ d_n, uint32_t W,
                   const uint32_t* __restrict__ d_off, Ws ws, AutoView av) {
  __shared__ BucketPlan plans[kMaxW + 1];
  __shared__ uint32_t s_off[kMaxW + 2];
  __shared__ uint32_t thr[kMaxW + 1], bcnt[kMaxW + 1], bbase[kMaxW + 1];
  const AutoView& v = av;
  load_plans(plans, s_off, d_off, W, v.hdr);
  // Acceptance probability per bucket: about 20 samples per expected segment
  // (segments expect 2730 / 1365 / 682 words for 1 / 2 / >= 3 keys, positions
  // are one per 32 words), but never more than 90 % of the bucket's sample
  // capacity.  The capacity must not truncate: the index is part of the sort
  // key, so a truncated sample would miss the later copies of a frequent word.
  // A position is kept when the high word of its hash is below thr[L].
  if (threadIdx.x <= W) {
    const uint32_t L = threadIdx.x;
    const BucketPlan& p = plans[L];
    uint32_t t = 0;
    if (L >= 1 && p.g >= 2) {
      const uint32_t cnt = s_off[L + 1] - s_off[L];
      const double want = p.K == 1 ? 0.25 : (p.K == 2 ? 0.5 : 1.0);
      const double room = 0.9 * p.scap * static_cast<double>(kAutoSampleEvery) / cnt;
      const double q = want < room ? want : room;
      t = q >= 1.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(q * 4294967296.0);
    }
    thr[L] = t;
    bcnt[L] = 0;
  }
  __syncthreads();
  const uint32_t n = word_count(n_cap, d_n);
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t h = mix64(s + 0x9E3779B97F4A7C15ull);
  const uint64_t i64 = static_cast<uint64_t>(s) * kAutoSampleEvery + (h & (kAutoSampleEvery - 1));
  const uint32_t i = static_cast<uint32_t>(i64);
  uint32_t L = i64 < n ? len[i] : 0u;
  if (L > W || static_cast<uint32_t>(h >> 32) >= thr[L]) L = 0;  // thr[0] = 0: never kept
  // slots: counted per bucket in the block, one global reservation per bucket
  const uint32_t local = L ? atomicAdd(&bcnt[L], 1u) : 0u;
  __syncthreads();
  if (threadIdx.x <= W && bcnt[threadIdx.x])
    bbase[threadIdx.x] = atomicAdd(&v.hdr->samp_cnt[threadIdx.x], bcnt[threadIdx.x]);
  __syncthreads();
  if (!L) return;
  const BucketPlan& p = plans[L];
  const uint32_t slot = bbase[L] + local;
  if (slot >= p.scap) return;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + static_cast<uint64_t>(i) * W);
  for (uint32_t k = 0; k < p.K; ++k)
    v.samp64[p.s64 + k * p.scap + slot] = bswap64(__ldg(src + k)) & key_mask(L, k);
  v.samp32[p.s32 + slot] = i;
}

// ---------------------------------------------------------------------------
// 2. splitters and region layout
// ---------------------------------------------------------------------------
// A bucket's m samples are cut into kSplChunks chunks, each sorted by its own
// CTA; a sample's rank among all m is its position in its chunk plus, for
// every other chunk, the number of that chunk's samples below it (samples are
// distinct: the index is part of the element).  Splitter s (0 <= s < g-1) is
// the sample of rank floor((s+1) m / g), the lower bound of segment s+1; with
// no samples every splitter is +inf, so all words land in the first segment
// (overflow then gives it an exact region).
constexpr uint32_t kSplChunks = 8;
__host__ __device__ constexpr uint32_t spl_chunk(uint32_t K) { return auto_sample_max(K) / kSplChunks; }
// the chunk sort's exchange planes (1024 threads), largest over K
__host__ __device__ constexpr size_t chunk_smem(uint32_t K) {
  return static_cast<size_t>(((spl_chunk(K) > 1024 ? spl_chunk(K) : 1024) - 1) * 17 / 16 + 1) * (8 * K + 4);
}
constexpr size_t kSplSortSmem = chunk_smem(4) > chunk_smem(1) ? chunk_smem(4) : chunk_smem(1);
static_assert(chunk_smem(2) <= kSplSortSmem && chunk_smem(3) <= kSplSortSmem, "chunk planes fit");

template <int K>
__device__ SmemTile<K> sample_tile(const AutoView& v, const BucketPlan& p) {
  SmemTile<K> t;
#pragma unroll
  for (int k = 0; k < K; ++k) t.k[k] = v.samp64 + p.s64 + static_cast<size_t>(k) * p.scap;
  t.idx = v.samp32 + p.s32;
  return t;
}

// Elements per thread of a chunk sort (1024 threads) and its exchange planes.
template <int K> struct ChunkE { static constexpr int value = spl_chunk(K) > 1024 ? spl_chunk(K) / 1024 : 1; };

template <int K>
__device__ void sort_sample_chunk(uint8_t* smem, const AutoView& v, const BucketPlan& p, uint32_t m,
                                  uint32_t j) {
  constexpr uint32_t CH = spl_chunk(K);
  constexpr int E = ChunkE<K>::value;
  constexpr uint32_t P = pad16(E * 1024 - 1) + 1;  // exchange slots per plane
  const uint32_t lo = j * CH;
  if (lo >= m) return;
  const uint32_t cnt = min(CH, m - lo);
  const SmemTile<K> g = sample_tile<K>(v, p);
  SmemTile<K> t;
  uint64_t* kp = reinterpret_cast<uint64_t*>(smem);
#pragma unroll
  for (int k = 0; k < K; ++k) t.k[k] = kp + k * P;
  t.idx = reinterpret_cast<uint32_t*>(kp + K * P);
  const ElemOps<K> ops{t};
  auto get = [&](uint32_t i) { return g.get(lo + i); };
  auto sink = [&](uint32_t i, const Elem<K>& e) { g.put(lo + i, e); };
  block_sort<ElemOps<K>, E>(ops, cnt, get, sink);
}

// (a) grid (W, kSplChunks): CTA (L-1, j) sorts chunk j of bucket L's samples;
// CTA (L-1, 0) also lays out the bucket's segment regions.
__global__ void __launch_bounds__(1024)
auto_spl_sort_kernel(const uint32_t* __restrict__ d_off, uint32_t W, Ws ws, AutoView av) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BucketPlan p;
  const AutoView& v = av;
  const uint32_t L = blockIdx.x + 1, j = blockIdx.y;
  if (threadIdx.x == 0) {
    p = v.hdr->plans[L];
    if (L == W && j == 0) {
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
  if (j == 0) {
    for (uint32_t q = threadIdx.x; q < p.g; q += blockDim.x) {
      const uint32_t seg = p.seg0 + q;
      v.cursor[seg * kCursorStride] = 0;
      v.rcap[seg] = p.cap;
      v.segL[seg] = L;
      v.rbase[seg] = p.r64 + static_cast<uint64_t>(q) * p.cap * p.K;
      v.ibase[seg] = p.r32 + static_cast<uint64_t>(q) * p.cap;
    }
  }
  if (p.g < 2) return;
  const uint32_t m = min(v.hdr->samp_cnt[L], p.scap);
  switch (p.K) {
    case 1: sort_sample_chunk<1>(smem, v, p, m, j); break;
    case 2: sort_sample_chunk<2>(smem, v, p, m, j); break;
    case 3: sort_sample_chunk<3>(smem, v, p, m, j); break;
    default: sort_sample_chunk<4>(smem, v, p, m, j); break;
  }
}

// (b) ranks.  The CTA stages the bucket's sorted first key words and indices
// in shared memory (kSplSelectSmem); a tie on the first word with more key
// words reads the rest from the sample planes.
constexpr size_t kSplSelectSmem = static_cast<size_t>(auto_sample_max(1)) * 12;
static_assert(auto_sample_max(2) * 12 <= kSplSelectSmem && auto_sample_max(3) * 12 <= kSplSelectSmem,
              "every bucket's first key words and indices fit the staging area");

template <int K>
__device__ void select_splitters(uint8_t* smem, const AutoView& v, const BucketPlan& p, uint32_t m,
                                 uint32_t j) {
  constexpr uint32_t CH = spl_chunk(K);
  const uint32_t ns = p.g - 1;
  uint64_t* sk = reinterpret_cast<uint64_t*>(v.spl + p.spl_off + kDirBytes);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + static_cast<size_t>(K) * ns);
  if (m == 0) {
    if (j == 0) {
      for (uint32_t s = threadIdx.x; s < ns; s += blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k) sk[k * ns + s] = ~0ull;
        si[s] = ~0u;
      }
    }
    return;
  }
  const uint32_t lo = j * CH;
  if (lo >= m) return;
  const uint32_t cnt = min(CH, m - lo);
  const uint32_t chunks = (m + CH - 1) / CH;
  const SmemTile<K> g = sample_tile<K>(v, p);
  uint64_t* k0s = reinterpret_cast<uint64_t*>(smem);
  uint32_t* ids = reinterpret_cast<uint32_t*>(k0s + m);
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    k0s[i] = g.k[0][i];
    ids[i] = g.idx[i];
  }
  __syncthreads();
  // is sample q (sorted position) below element e (at sorted position x)?
  auto below = [&](uint32_t q, const Elem<K>& e) {
    const uint64_t a = k0s[q];
    if (a != e.k[0]) return a < e.k[0];
    if constexpr (K == 1) return ids[q] < e.idx;
    else return elem_less<K>(g.get(q), e);
  };
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    Elem<K> e;
    e.k[0] = k0s[lo + i];
#pragma unroll
    for (int k = 1; k < K; ++k) e.k[k] = g.k[k][lo + i];
    e.idx = ids[lo + i];
    // binary searches in all other chunks in lockstep (independent loads)
    uint32_t a[kSplChunks], b[kSplChunks];
#pragma unroll
    for (uint32_t q = 0; q < kSplChunks; ++q) {
      a[q] = 0;
      b[q] = (q < chunks && q != j) ? min(CH, m - q * CH) : 0u;
    }
    for (uint32_t w = CH; w > 0; w >>= 1) {  // at most log2(CH) + 1 halvings
#pragma unroll
      for (uint32_t q = 0; q < kSplChunks; ++q) {
        if (a[q] < b[q]) {
          const uint32_t mid = (a[q] + b[q]) >> 1;
          if (below(q * CH + mid, e)) a[q] = mid + 1;
          else b[q] = mid;
        }
      }
    }
    uint32_t r = i;
#pragma unroll
    for (uint32_t q = 0; q < kSplChunks; ++q) r += a[q];
    // splitters s with floor((s+1) m / g) == r: s+1 in [ceil(r g / m), ceil((r+1) g / m))
    const uint64_t s1 = (static_cast<uint64_t>(r) * p.g + m - 1) / m;
    const uint64_t s2 = (static_cast<uint64_t>(r + 1) * p.g + m - 1) / m;
    for (uint64_t t = s1 < 1 ? 1 : s1; t < s2 && t <= ns; ++t) {
      const uint32_t sp = static_cast<uint32_t>(t - 1);
#pragma unroll
      for (int k = 0; k < K; ++k) sk[k * ns + sp] = e.k[k];
      si[sp] = e.idx;
    }
  }
}

// (b) grid (W, kSplChunks): CTA (L-1, j) ranks the samples of chunk j of
// bucket L and writes those that are splitters.
__global__ void __launch_bounds__(1024)
auto_spl_select_kernel(const uint32_t* __restrict__ d_off, uint32_t W, Ws ws, AutoView av) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BucketPlan p;
  const AutoView& v = av;
  const uint32_t L = blockIdx.x + 1, j = blockIdx.y;
  if (threadIdx.x == 0) p = v.hdr->plans[L];
  __syncthreads();
  if (p.g < 2) return;
  const uint32_t m = min(v.hdr->samp_cnt[L], p.scap);
  switch (p.K) {
    case 1: select_splitters<1>(smem, v, p, m, j); break;
    case 2: select_splitters<2>(smem, v, p, m, j); break;
    case 3: select_splitters<3>(smem, v, p, m, j); break;
    default: select_splitters<4>(smem, v, p, m, j); break;
  }
}

// Byte code records of a one- or two-key bucket's segments.  Segment q holds
// the words between splitters q-1 and q (inclusive on the keys), so its keys
// agree with both splitters up to the first byte position p0 where the two
// differ: those positions are constant (width 0), position p0 spans the two
// splitters' bytes, and every later position of the word the range of all
// bytes inside words, [band, bor]; positions past the word are zero.  The
// first segment has no lower splitter (band in every position), the last no
// upper one (bor).  The index width covers the largest word index.  Every key
// of the segment fits the fields, and the code keeps the key order.
__device__ void segment_codes(const AutoView& v, const BucketPlan& p, uint32_t L) {
  const uint32_t band = v.hdr->band, bor = v.hdr->bor;
  const uint32_t wl = bor > band ? 32u - static_cast<uint32_t>(__clz(bor - band)) : 0u;
  const uint32_t ib = 32u - static_cast<uint32_t>(__clz(v.hdr->imax | 1u));
  const uint32_t ns = p.g - 1;
  const uint64_t* sk = reinterpret_cast<const uint64_t*>(v.spl + p.spl_off + kDirBytes);
  const uint64_t lo_all = 0x0101010101010101ull * band, hi_all = 0x0101010101010101ull * bor;
  const uint32_t step = gridDim.y * blockDim.x;
  for (uint32_t q = blockIdx.y * blockDim.x + threadIdx.x; q < p.g; q += step) {
    uint64_t lk[2], uk[2];
#pragma unroll
    for (uint32_t k = 0; k < 2; ++k) {
      lk[k] = k < p.K && q > 0 ? sk[k * ns + q - 1] : lo_all;
      uk[k] = k < p.K && q < ns ? sk[k * ns + q] : hi_all;
    }
    uint32_t fl[16];  // lo | width << 16
    bool split = false;
    uint32_t p0 = 7;  // first position where the bounds differ (7: none)
#pragma unroll
    for (uint32_t pos = 0; pos < 16; ++pos) {
      const uint32_t k = pos >> 3, sh = 56 - 8 * (pos & 7);
      const uint32_t lb = static_cast<uint32_t>(lk[k] >> sh) & 255u;
      const uint32_t ub = static_cast<uint32_t>(uk[k] >> sh) & 255u;
      uint32_t lo = 0, w = 0;
      if (pos < L && k < p.K) {
        if (split) {
          lo = band;
          w = wl;
        } else if (lb == ub) {
          lo = lb;
        } else {
          // lb < ub, but for the all-ones splitters of an unsampled bucket,
          // whose later segments stay empty
          split = true;
          p0 = pos;
          lo = min(lb, ub);
          w = 32u - static_cast<uint32_t>(__clz(max(lb, ub) - lo));
        }
      }
      fl[pos] = lo | (w << 16);
    }
    uint32_t* f = v.segf + static_cast<size_t>(p.seg0 + q) * kSegFWords;
    uint32_t off = 0;
#pragma unroll
    for (int pos = 15; pos >= 0; --pos) {
      const uint32_t w = fl[pos] >> 16;
      f[pos] = (fl[pos] & 255u) | ((off > 63u ? 63u : off) << 8) | (w << 16);
      off += w;
    }
    f[16] = off;
    f[17] = ib;
    if (p.K != 1) continue;
    // one-key shape: packed smallest bytes, p0, its width, the later width
    // and the number of later positions of the word
    uint64_t lo8 = 0;
#pragma unroll
    for (uint32_t pos = 0; pos < 8; ++pos) lo8 |= static_cast<uint64_t>(fl[pos] & 255u) << (56 - 8 * pos);
    const uint32_t w0 = fl[p0 & 7] >> 16, n = split && L > p0 + 1 ? min(L, 8u) - 1 - p0 : 0u;
    f[18] = static_cast<uint32_t>(lo8 >> 32);
    f[19] = static_cast<uint32_t>(lo8);
    f[20] = (p0 & 7) | (w0 << 8) | (wl << 16) | (n << 24);
  }
}

// (c) grid (W, kSplDirCtas): the CTAs of bucket L write its segments' byte
// code records and its directory: dir[c] = number of splitters whose
// directory code is below c (splitters are sorted, so their codes never
// decrease).
constexpr uint32_t kSplDirCtas = 4;
__global__ void __launch_bounds__(288)
auto_spl_dir_kernel(const uint32_t* __restrict__ d_off, uint32_t W, Ws ws, AutoView av) {
  __shared__ BucketPlan p;
  const AutoView& v = av;
  const uint32_t L = blockIdx.x + 1;
  if (threadIdx.x == 0) p = v.hdr->plans[L];
  __syncthreads();
  if (p.K <= 2) segment_codes(v, p, L);
  if (p.g < 2) return;
  const uint32_t ns = p.g - 1;
  const DirShape ds = dir_shape(v.hdr);
  const uint32_t N = dir_entries(ds);
  uint16_t* dir = reinterpret_cast<uint16_t*>(v.spl + p.spl_off);
  const uint64_t* sk0 = reinterpret_cast<const uint64_t*>(v.spl + p.spl_off + kDirBytes);
  for (uint32_t c = blockIdx.y * blockDim.x + threadIdx.x; c <= N; c += gridDim.y * blockDim.x) {
    uint32_t lo = 0, hi = ns;  // first splitter with code >= c
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (dir_code(sk0[mid], ds) < c) lo = mid + 1;
      else hi = mid;
    }
    dir[c] = static_cast<uint16_t>(lo);
  }
}

// ---- one-key segments: byte recoding -----------------------------------
// A one-key segment's keys (big-endian, bytes past the word zero) are recoded
// position by position: byte position p (0 = most significant) maps value b to
// b - lo_p in a field just wide enough for the segment's range at p, and the
// fields are laid out most significant first.  The code orders like the key
// (the byte order is kept within every field and the fields follow the byte
// positions) and decodes back exactly.  A segment's ranges come from its
// bounding splitters: positions before p0 (where the splitters first differ)
// are constant and take no bits, position p0 takes w0 bits, each of the n
// later positions of the word wl bits (the range of all bytes inside words, 5
// for lower-case letters), so codes are narrow and their top bits spread.
// key - lo (lo: every position's smallest byte, packed) has no borrows, so its
// bytes are the field values; packing byte lanes into wl-bit fields, and back,
// takes three halving steps of masked shifts on the two 32-bit halves.
struct ByteCode {
  uint64_t lo;
  uint32_t p0, w0, wl, n;  // n wl <= 56, p0 <= 7
  __device__ __forceinline__ uint64_t encode(uint64_t key) const {
    const uint64_t d = (key - lo) << (8 * p0);  // lane 0 (top byte): position p0
    const uint32_t b0 = static_cast<uint32_t>(d >> 56);
    const uint64_t t = d << 8;  // lanes 0 .. n-1: the later positions, then zeros
    const uint32_t s1 = 8 - wl, s2 = 16 - 2 * wl;
    uint32_t h = static_cast<uint32_t>(t >> 32), l = static_cast<uint32_t>(t);
    h = ((h & 0xFF00FF00u) >> s1) | (h & 0x00FF00FFu);  // 16-bit groups of 2 fields
    l = ((l & 0xFF00FF00u) >> s1) | (l & 0x00FF00FFu);
    h = ((h & 0xFFFF0000u) >> s2) | (h & 0x0000FFFFu);  // halves of 4 fields
    l = ((l & 0xFFFF0000u) >> s2) | (l & 0x0000FFFFu);
    const uint64_t packed = (static_cast<uint64_t>(h) << (4 * wl)) | l;  // lanes 0..7 in 8 wl bits
    const uint64_t tail = n ? packed >> (wl * (8 - n)) : 0ull;
    return (static_cast<uint64_t>(b0) << (n * wl)) | tail;
  }
  __device__ __forceinline__ uint64_t decode(uint64_t code) const {
    const uint32_t nt = n * wl;
    const uint32_t b0 = static_cast<uint32_t>(code >> nt);
    const uint64_t packed = n ? (code & ((1ull << nt) - 1)) << (wl * (8 - n)) : 0ull;
    const uint32_t s1 = 8 - wl, s2 = 16 - 2 * wl;
    const uint32_t m4 = wl == 8 ? 0xFFFFFFFFu : (1u << (4 * wl)) - 1u;
    const uint32_t m2 = (1u << (2 * wl)) - 1u, m1 = ((1u << wl) - 1u) * 0x00010001u;
    uint32_t h = static_cast<uint32_t>(packed >> (4 * wl)), l = static_cast<uint32_t>(packed) & m4;
    h = ((h << s2) & (m2 << 16)) | (h & m2);
    l = ((l << s2) & (m2 << 16)) | (l & m2);
    h = ((h << s1) & (m1 << 8)) | (h & m1);
    l = ((l << s1) & (m1 << 8)) | (l & m1);
    const uint64_t t = (static_cast<uint64_t>(h) << 32) | l;
    const uint64_t d = (static_cast<uint64_t>(b0) << 56) | (t >> 8);
    return (d >> (8 * p0)) + lo;
  }
};

// ---------------------------------------------------------------------------
// 3. partition
// ---------------------------------------------------------------------------
// Per-bucket constants of the partition (shared memory, 32 bytes: two
// vector loads).
struct __align__(16) PartPlan {
  uint32_t g, seg0, spl_off, cap;
  uint64_t r64, r32;
};

// ---- 3a. length buckets -------------------------------------------------
// Tiles of kBucketTile words: each tile counts its words per length in shared
// memory (the count so far is a word's slot within its tile), reserves one
// range per length with a single global atomic, and writes every word's key
// words and index into its bucket's staging planes (bucket L: K_L key planes
// of count_L words at key offset kb_L = sum over l < L of count_l K_l, the
// indices at the bucket offset off[L]).  A tile's words of one length land in
// one contiguous range, so the writes combine in L2.
constexpr uint32_t kBucketThreads = 512;
constexpr uint32_t kBucketPer = 4;
constexpr uint32_t kBucketTile = kBucketThreads * kBucketPer;

// Folds key word w (bytes past the word cleared by mask m) into the AND and
// the OR of the bytes inside words.  Every such byte b has band <= b <= bor
// (band's bits are a subset of b's, b's a subset of bor's); for letters the
// bounds are as tight as the smallest and largest letter's in bit width.
__device__ __forceinline__ void letter_bounds(uint64_t w, uint64_t m, uint64_t& band, uint64_t& bor) {
  band &= w | ~m;  // bytes past the word read as all ones for the AND
  bor |= w;
}

// Key offsets kb[L] (u64 units) of the staging planes, from the offsets.
__device__ __forceinline__ void stage_key_bases(const uint32_t* s_off, uint32_t W, uint32_t* kb) {
  if (threadIdx.x == 0) {
    uint32_t o = 0;
    for (uint32_t L = 0; L <= W + 1; ++L) {
      kb[L] = o;
      if (L >= 1 && L <= W) o += (s_off[L + 1] - s_off[L]) * keys_for_len(L);
    }
  }
}

__global__ void __launch_bounds__(kBucketThreads)
auto_bucket_kernel(const uint8_t* __restrict__ rec, const uint8_t* __restrict__ len,
                   uint32_t n_cap, const uint32_t* __restrict__ d_n, uint32_t W,
                   const uint32_t* __restrict__ d_off, Ws ws, AutoView av) {
  __shared__ uint32_t s_off[kMaxW + 2], kb[kMaxW + 2], cnt[kBins], base[kBins];
  const AutoView& v = av;
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  stage_key_bases(s_off, W, kb);
  const uint32_t n = word_count(n_cap, d_n);
  uint64_t band = ~0ull, bor = 0;  // AND and OR of the bytes inside words
  if (blockIdx.x == 0 && threadIdx.x == 0) v.hdr->imax = n ? n - 1 : 0;
  for (uint32_t t0 = blockIdx.x * kBucketTile; t0 < n; t0 += gridDim.x * kBucketTile) {
    if (threadIdx.x < kBins) cnt[threadIdx.x] = 0;
    __syncthreads();
    uint32_t L[kBucketPer], r[kBucketPer];
    uint64_t k0[kBucketPer];
    // lengths and first key words first, all loads in flight together (the
    // record read does not wait for the length): they overlap the counting
#pragma unroll
    for (uint32_t q = 0; q < kBucketPer; ++q) {
      const uint32_t i = t0 + q * kBucketThreads + threadIdx.x;
      const uint32_t l = i < n ? len[i] : 0u;
      L[q] = (l >= 1 && l <= W) ? l : 0u;  // bad lengths are flagged by the histogram
      k0[q] = i < n ? __ldg(reinterpret_cast<const uint64_t*>(rec + static_cast<uint64_t>(i) * W)) : 0ull;
    }
#pragma unroll
    for (uint32_t q = 0; q < kBucketPer; ++q) r[q] = L[q] ? atomicAdd(&cnt[L[q]], 1u) : 0u;
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x <= W && cnt[threadIdx.x])
      base[threadIdx.x] = atomicAdd(&v.hdr->bcur[threadIdx.x], cnt[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (uint32_t q = 0; q < kBucketPer; ++q) {
      if (!L[q]) continue;
      const uint32_t i = t0 + q * kBucketThreads + threadIdx.x, l = L[q];
      const uint32_t count = s_off[l + 1] - s_off[l], dest = base[l] + r[q];
      const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + static_cast<uint64_t>(i) * W);
      uint64_t* dk = v.stage64 + kb[l] + dest;
      const uint64_t w0 = bswap64(k0[q]) & key_mask(l, 0);
      dk[0] = w0;
      letter_bounds(w0, key_mask(l, 0), band, bor);
      for (uint32_t k = 1; k < keys_for_len(l); ++k) {
        const uint64_t w = bswap64(__ldg(src + k)) & key_mask(l, k);
        dk[static_cast<uint64_t>(k) * count] = w;
        letter_bounds(w, key_mask(l, k), band, bor);
      }
      v.stage32[s_off[l] + dest] = i;
    }
    __syncthreads();
  }
  band &= band >> 32;
  band &= band >> 16;
  band &= band >> 8;
  bor |= bor >> 32;
  bor |= bor >> 16;
  bor |= bor >> 8;
  const uint32_t a = __reduce_and_sync(0xffffffffu, static_cast<uint32_t>(band) & 255u);
  const uint32_t o = __reduce_or_sync(0xffffffffu, static_cast<uint32_t>(bor) & 255u);
  if (lane_id() == 0) {
    if (a != 255u) atomicAnd(&v.hdr->band, a);
    if (o != 0u) atomicOr(&v.hdr->bor, o);
  }
}

// ---- 3b. segments ---------------------------------------------------------
// Bucket-uniform tiles of kPartTile staged elements: every element finds its
// segment, the tile counts its elements per segment in shared memory (the
// count so far is an element's slot within the tile's run), reserves one run
// per segment with a single global atomic on the segment's cursor, and writes
// the elements.  The bucket's splitter table is staged in shared memory when
// it fits.  A slot past the region's end only counts and raises the overflow
// flag (the retry pass then runs on exact regions).
constexpr uint32_t kPartThreads2 = 1024;  // one CTA per SM: tiles of 4,096 elements
constexpr uint32_t kPartPer = 4;
constexpr uint32_t kPartTile = kPartThreads2 * kPartPer;
constexpr uint32_t kPartCounters = 8192;                  // segments per bucket counted in shared memory
constexpr uint32_t kPartSplSmem = 160 * 1024;             // bucket splitter table staged up to this size
constexpr size_t kPartSmem = kPartCounters * 4 + kPartSplSmem;
static_assert(kPartSmem + 4096 <= 227 * 1024, "the partition CTA's shared memory fits an SM");

// Segments (indices within the bucket) of a thread's kPartPer elements (first
// key words k0, input indices i; active[u] false for none), in a bucket whose
// splitter table (directory, key planes, indices) starts at tab and holds g - 1
// splitters: the number of splitters <= the element.  key(u, k) reads key word
// k >= 1 of element u, needed only when first words tie.  The directory
// narrows each search to the splitters with the element's directory code,
// [lo, hi]; the searches step together (one halving step of every element per
// round, their loads independent) for as many rounds as the warp's widest
// range needs, so the loop does not diverge.
template <typename KeyK>
__device__ __forceinline__ void find_segments(const uint8_t* tab, const DirShape& ds, uint32_t g, uint32_t K,
                                              const uint64_t (&k0)[kPartPer], const uint32_t (&i)[kPartPer],
                                              const bool (&active)[kPartPer], KeyK key,
                                              uint32_t (&seg)[kPartPer]) {
  const uint32_t ns = g - 1;
  const uint16_t* dir = reinterpret_cast<const uint16_t*>(tab);
  const uint64_t* sk = reinterpret_cast<const uint64_t*>(tab + kDirBytes);
  const uint32_t* si = reinterpret_cast<const uint32_t*>(sk + static_cast<size_t>(K) * ns);
  // splitters below dir[c] have a smaller code (all <= the element), those
  // from dir[c+1] on a larger one
  uint32_t lo[kPartPer], hi[kPartPer], w = 0;
#pragma unroll
  for (uint32_t u = 0; u < kPartPer; ++u) {
    const uint32_t c = dir_code(k0[u], ds);
    lo[u] = active[u] ? dir[c] : 0u;
    hi[u] = active[u] ? dir[c + 1] : 0u;
    w = max(w, 32u - static_cast<uint32_t>(__clz(hi[u] - lo[u])));
  }
  const uint32_t steps = __reduce_max_sync(0xffffffffu, w);
  for (uint32_t t = 0; t < steps; ++t) {
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
      if (lo[u] < hi[u]) {
        const uint32_t mid = (lo[u] + hi[u] + 1) >> 1, sp = mid - 1;  // is splitter mid-1 <= element ?
        const uint64_t a = sk[sp];
        bool le = a < k0[u];
        if (a == k0[u]) {
          if (K == 1) {
            le = si[sp] <= i[u];
          } else {
            // multi-key tie on the first word (rare): later words, then the index
            uint32_t k = 1;
            uint64_t ak = 0, bk = 0;
            for (; k < K; ++k) {
              ak = sk[k * ns + sp];
              bk = key(u, k);
              if (ak != bk) break;
            }
            le = k < K ? ak < bk : si[sp] <= i[u];
          }
        }
        lo[u] = le ? mid : lo[u];
        hi[u] = le ? hi[u] : mid - 1;
      }
    }
  }
#pragma unroll
  for (uint32_t u = 0; u < kPartPer; ++u) seg[u] = lo[u];
}

__global__ void __launch_bounds__(kPartThreads2, 1)
auto_partition_kernel(uint32_t W, const uint32_t* __restrict__ d_off, int retry_pass, Ws ws,
                      AutoView av) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem);
  uint8_t* tabs = smem + kPartCounters * 4;
  __shared__ PartPlan plans[kMaxW + 1];
  __shared__ uint32_t s_off[kMaxW + 2], kb[kMaxW + 2], tp[kMaxW + 2];
  const AutoView& v = av;
  if (retry_pass && v.hdr->retry == 0) return;
  if (threadIdx.x < W + 2) s_off[threadIdx.x] = d_off[threadIdx.x];
  __syncthreads();
  if (threadIdx.x <= W) {
    const BucketPlan bp = v.hdr->plans[threadIdx.x];
    plans[threadIdx.x] = PartPlan{bp.g, bp.seg0, bp.spl_off, bp.cap, bp.r64, bp.r32};
  }
  stage_key_bases(s_off, W, kb);
  if (threadIdx.x == 0) {  // tile prefix: tiles of buckets below L
    uint32_t o = 0;
    for (uint32_t L = 0; L <= W + 1; ++L) {
      tp[L] = o;
      if (L >= 1 && L <= W) o += (s_off[L + 1] - s_off[L] + kPartTile - 1) / kPartTile;
    }
  }
  __syncthreads();
  const uint32_t tiles = tp[W + 1];
  const DirShape ds = dir_shape(v.hdr);
  // A one-key segment that will be sorted in shared memory and whose item
  // (code 2^ib + index) fits 64 bits gets its elements as that item, the code
  // from the segment's byte-code record (staged in shared memory after the
  // splitter table when it fits): the segment sort then copies 8 instead of
  // 12 bytes per element and skips the encoding.
  const uint32_t item_ib = 32u - static_cast<uint32_t>(__clz(v.hdr->imax | 1u));
  uint32_t staged = 0;  // bucket whose splitter table is in shared memory
  bool overflow = false;
  uint32_t L = 1;  // bucket of tile t (block-uniform; a CTA's tiles increase)
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    while (L < W && tp[L + 1] <= t) ++L;
    const PartPlan p = plans[L];
    const uint32_t K = keys_for_len(L), count = s_off[L + 1] - s_off[L];
    const uint32_t e0 = (t - tp[L]) * kPartTile, m = min(kPartTile, count - e0);
    const uint64_t* k0p = v.stage64 + kb[L];
    const uint32_t* ipp = v.stage32 + s_off[L];
    // the bucket's splitter table
    const uint8_t* tab = v.spl + p.spl_off;
    const uint32_t tb = p.g > 1 ? static_cast<uint32_t>(spl_bytes_of(p.g, K)) : 0u;
    const bool tab_smem = tb <= kPartSplSmem;
    // one-key records: lo (two words), shape, code width per segment
    uint4* recs = reinterpret_cast<uint4*>(tabs + tb);
    const bool rec_smem = K == 1 && tb + p.g * 16 <= kPartSplSmem;
    if (staged != L) {
      // earlier readers of the staged table are done (barrier ending the
      // previous tile)
      if (tab_smem && tb) {
        const uint4* src = reinterpret_cast<const uint4*>(tab);
        uint4* dst = reinterpret_cast<uint4*>(tabs);
        for (uint32_t q = threadIdx.x; q < tb / 16; q += blockDim.x) dst[q] = src[q];
      }
      if (rec_smem) {
        for (uint32_t q = threadIdx.x; q < p.g; q += blockDim.x) {
          const uint32_t* f = v.segf + static_cast<size_t>(p.seg0 + q) * kSegFWords;
          recs[q] = make_uint4(f[18], f[19], f[20], f[16]);
        }
      }
      staged = L;
    }
    if (tab_smem) tab = tabs;
    const auto seg_rec = [&](uint32_t sgm) {
      if (rec_smem) return recs[sgm];
      const uint32_t* f = v.segf + static_cast<size_t>(p.seg0 + sgm) * kSegFWords;
      return make_uint4(f[18], f[19], f[20], f[16]);
    };
    // element e of the tile to its region slot: the item of a one-key segment
    // sorted in shared memory when it fits 64 bits, else key words and index
    const auto put = [&](uint32_t sgm, uint32_t pos, uint32_t rc, uint64_t rb, uint64_t ib, uint64_t key0,
                         uint32_t idx, uint32_t e) {
      if (K == 1 && rc <= auto_seg_cap(1)) {
        const uint4 r = seg_rec(sgm);
        if (r.w + item_ib <= 64) {
          ByteCode bc;
          bc.lo = (static_cast<uint64_t>(r.x) << 32) | r.y;
          bc.p0 = r.z & 255u;
          bc.w0 = (r.z >> 8) & 255u;
          bc.wl = (r.z >> 16) & 255u;
          bc.n = r.z >> 24;
          v.area64[rb + pos] = (bc.encode(key0) << item_ib) | idx;
          return;
        }
      }
      v.area64[rb + pos] = key0;
      for (uint32_t k = 1; k < K; ++k)
        v.area64[rb + static_cast<uint64_t>(k) * rc + pos] = k0p[static_cast<uint64_t>(k) * count + e0 + e];
      v.area32[ib + pos] = idx;
    };
    const bool local = p.g <= kPartCounters;
    if (local)
      for (uint32_t q = threadIdx.x; q < p.g; q += blockDim.x) cnt[q] = 0;
    uint32_t idxs[kPartPer];
    uint64_t key0s[kPartPer];
    bool in[kPartPer];
#pragma unroll
    for (uint32_t q = 0; q < kPartPer; ++q) {
      const uint32_t e = q * kPartThreads2 + threadIdx.x;
      in[q] = e < m;
      key0s[q] = in[q] ? k0p[e0 + e] : 0ull;
      idxs[q] = in[q] ? ipp[e0 + e] : 0u;
    }
    __syncthreads();  // table and zeroed counters visible
    // segment (within the bucket) and slot of every element: s << 16 | slot
    uint32_t sg[kPartPer], sr[kPartPer];
    const auto keyk = [&](uint32_t u, uint32_t k) {
      return k0p[static_cast<uint64_t>(k) * count + e0 + u * kPartThreads2 + threadIdx.x];
    };
    if (p.g > 1) {
      find_segments(tab, ds, p.g, K, key0s, idxs, in, keyk, sg);
    } else {
#pragma unroll
      for (uint32_t q = 0; q < kPartPer; ++q) sg[q] = 0;
    }
#pragma unroll
    for (uint32_t q = 0; q < kPartPer; ++q) {
      const uint32_t e = q * kPartThreads2 + threadIdx.x;
      uint32_t slot = 0;
      if (in[q]) slot = local ? atomicAdd(&cnt[sg[q]], 1u) : atomicAdd(&v.cursor[(p.seg0 + sg[q]) * kCursorStride], 1u);
      sr[q] = (in[q] && local) ? (sg[q] << 16 | slot) : 0xFFFFFFFFu;
      if (!local && in[q]) {
        // no tile counting: the slot came from the segment's cursor directly
        const uint32_t pos = slot;
        uint32_t rc;
        uint64_t rb, ib;
        if (!retry_pass) {
          rc = p.cap;
          rb = p.r64 + static_cast<uint64_t>(sg[q]) * p.cap * K;
          ib = p.r32 + static_cast<uint64_t>(sg[q]) * p.cap;
        } else {
          rc = v.rcap[p.seg0 + sg[q]];
          rb = v.rbase[p.seg0 + sg[q]];
          ib = v.ibase[p.seg0 + sg[q]];
        }
        if (pos < rc) put(sg[q], pos, rc, rb, ib, key0s[q], idxs[q], e);
        else overflow = true;
      }
    }
    if (local) {
      __syncthreads();
      // one run per segment the tile touches; the reservations of a thread
      // are issued back to back
      constexpr uint32_t per = kPartCounters / kPartThreads2;
      const uint32_t rounds = (p.g + kPartThreads2 - 1) / kPartThreads2;  // block-uniform, <= per
      uint32_t got[per];
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) {
        if (k >= rounds) break;
        const uint32_t q = k * kPartThreads2 + threadIdx.x;
        const uint32_t c = q < p.g ? cnt[q] : 0u;
        got[k] = c ? atomicAdd(&v.cursor[(p.seg0 + q) * kCursorStride], c) : 0u;
      }
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) {
        if (k >= rounds) break;
        const uint32_t q = k * kPartThreads2 + threadIdx.x;
        if (q < p.g) cnt[q] = got[k];
      }
      __syncthreads();
      const uint32_t capK = p.cap * K;
#pragma unroll
      for (uint32_t q = 0; q < kPartPer; ++q) {
        if (sr[q] == 0xFFFFFFFFu) continue;
        const uint32_t e = q * kPartThreads2 + threadIdx.x, s = sr[q] >> 16;
        const uint32_t pos = cnt[s] + (sr[q] & 0xFFFFu);
        uint32_t rc;
        uint64_t rb, ib;
        if (!retry_pass) {
          // optimistic layout: a pure function of the bucket plan
          rc = p.cap;
          rb = p.r64 + static_cast<uint64_t>(s) * capK;
          ib = p.r32 + static_cast<uint64_t>(s) * p.cap;
        } else {
          rc = v.rcap[p.seg0 + s];
          rb = v.rbase[p.seg0 + s];
          ib = v.ibase[p.seg0 + s];
        }
        if (pos < rc) put(s, pos, rc, rb, ib, key0s[q], idxs[q], e);
        else overflow = true;
      }
    }
    __syncthreads();  // counters and staged table reused by the next tile
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
auto_layout_kernel(uint32_t W, Ws ws, AutoView av) {
  __shared__ uint32_t tmp[1024 / 32 + 1];
  const AutoView& v = av;
  const uint32_t G = v.hdr->G;
  const bool redo = v.hdr->overflow != 0;
  // thread t owns segments [t per, t per + per); their counts and key word
  // counts are read in batches of kLayoutBatch, every load of a batch in
  // flight together, and kept for the second pass when one batch covers them
  constexpr uint32_t kLayoutBatch = 8;
  const uint32_t per = (G + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = min(G, b + per);
  uint32_t xs[kLayoutBatch], ks[kLayoutBatch];
  const auto load = [&](uint32_t j0) {
#pragma unroll
    for (uint32_t u = 0; u < kLayoutBatch; ++u) {
      const uint32_t j = j0 + u;
      xs[u] = j < e ? v.cursor[j * kCursorStride] : 0u;
      ks[u] = j < e ? keys_for_len(v.segL[j]) : 1u;
    }
  };
  // exclusive scans of counts (output ranks) and, for a retry, of exact
  // regions (index area) and region x K (key area)
  uint32_t c = 0, c4 = 0, ck = 0;
  for (uint32_t j0 = b; j0 < e; j0 += kLayoutBatch) {
    load(j0);
#pragma unroll
    for (uint32_t u = 0; u < kLayoutBatch; ++u) {
      c += xs[u];
      c4 += exact_region(xs[u], ks[u]);
      ck += exact_region(xs[u], ks[u]) * ks[u];
    }
  }
  uint32_t tot, tot4, totk;
  uint32_t run = block_exclusive_scan(c, tmp, &tot);
  uint32_t run4 = block_exclusive_scan(c4, tmp, &tot4);
  uint32_t runk = block_exclusive_scan(ck, tmp, &totk);
  const bool fits = tot4 <= v.size32 && totk <= v.size64;
  for (uint32_t j0 = b; j0 < e; j0 += kLayoutBatch) {
    if (per > kLayoutBatch) load(j0);  // block-uniform
#pragma unroll
    for (uint32_t u = 0; u < kLayoutBatch; ++u) {
      const uint32_t j = j0 + u;
      if (j >= e) break;
      v.outbase[j] = run;
      run += xs[u];
      if (redo && fits) {
        const uint32_t r = exact_region(xs[u], ks[u]);
        v.rcap[j] = r;
        v.ibase[j] = run4;
        v.rbase[j] = runk;
        run4 += r;
        runk += r * ks[u];
        v.cursor[j * kCursorStride] = 0;
      }
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
// Shared-memory planes of a resident segment (capacity elements each); a
// one-key segment's radix counters (one row of 8-bit digit counters per
// warp) and warp totals follow its planes.
constexpr uint32_t kRxWarps = kSegThreads / 32;
constexpr uint32_t kRxDigits = 256;
constexpr size_t kRxHistBytes =
    kRxWarps * kRxDigits * sizeof(uint16_t) + 2 * kRxWarps * sizeof(uint32_t);  // counters, warp sums + maxima

__host__ __device__ constexpr size_t seg_plane_elems(uint32_t K) { return auto_seg_cap(K); }

// >= max over K of the planes (8K + 4 bytes per element), and the one-key
// planes plus the radix counters (checked below)
constexpr size_t kSegPlanesBytes = 106624;

// One segment buffer per CTA (two CTAs per SM overlap each other's copies,
// sorts and stores): barrier + planes.
constexpr size_t kSegBufBytes = 16 + kSegPlanesBytes;
__host__ __device__ constexpr size_t segsort_smem_bytes() { return kSegBufBytes; }

// Where the segment sort puts the word of output rank r: its input index to
// perm[r] and either the zero-padded record at rec[r W] (RecSink) or, in the
// packed form (§3.1), its L bytes at bytes[base + r L] with that start in
// offsets[r] (PackSink; the bytes only when the total fits the buffer).
struct RecSink {
  uint8_t* rec;
  uint32_t* perm;
  uint32_t W;
  template <int K>
  __device__ __forceinline__ void put(uint32_t r, const Elem<K>& e) const {
    const uint32_t KW = W / 8;
    uint64_t* dst = reinterpret_cast<uint64_t*>(rec + static_cast<uint64_t>(r) * W);
    if ((W & 15u) == 0) {
      for (uint32_t k = 0; k < KW; k += 2) {
        const uint64_t a = k < static_cast<uint32_t>(K) ? bswap64(e.k[k]) : 0ull;
        const uint64_t b = k + 1 < static_cast<uint32_t>(K) ? bswap64(e.k[k + 1]) : 0ull;
        reinterpret_cast<ulonglong2*>(dst)[k / 2] = make_ulonglong2(a, b);
      }
    } else {
      for (uint32_t k = 0; k < KW; ++k) dst[k] = k < static_cast<uint32_t>(K) ? bswap64(e.k[k]) : 0ull;
    }
    perm[r] = e.idx;
  }
};

struct PackSink {
  uint8_t* bytes;
  uint32_t* offsets;
  uint32_t* perm;
  uint32_t L, base, fits;
  template <int K>
  __device__ __forceinline__ void put(uint32_t r, const Elem<K>& e) const {
    const uint32_t o = base + r * L;
    offsets[r] = o;
    if (fits) put_word_bytes<K>(bytes + o, L, e.k);
    perm[r] = e.idx;
  }
};

// A segment larger than shared memory (only after a retry, whose region is
// data + scratch): sort chunks in shared memory, then merge runs pairwise with
// merge-path tiles, ping-ponging between the two halves.
template <int K, typename Sink>
__device__ void segsort_big(uint8_t* smem, const AutoView& v, uint32_t seg, uint32_t c,
                            const Sink& o) {
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
  for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) o.template put<K>(ob + r, src.get(r));
  __syncthreads();
}

// Issues the bulk copies (TMA) of segment seg (c <= capacity) into buffer buf.
template <int K>
__device__ void prefetch_segment(uint8_t* buf, const AutoView& v, uint32_t seg, uint32_t c,
                                 bool with_idx = true) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf);
  uint64_t* kp = reinterpret_cast<uint64_t*>(buf + 16);
  const uint32_t C = static_cast<uint32_t>(seg_plane_elems(K));
  uint32_t* ip = reinterpret_cast<uint32_t*>(kp + static_cast<size_t>(K) * C);
  const uint32_t rc = v.rcap[seg];
  const uint64_t rb = v.rbase[seg], ib = v.ibase[seg];
  // regions start 16-byte aligned (rcap, rbase, ibase are multiples of 4) and
  // hold rcap >= round4(c) elements, so the rounded copies stay inside
  const uint32_t kbytes = (c * 8 + 15) & ~15u, ibytes = with_idx ? (c * 4 + 15) & ~15u : 0u;
  mbar_arrive_expect_tx(bar, K * kbytes + ibytes);
#pragma unroll
  for (int k = 0; k < K; ++k)
    bulk_g2s(kp + k * C, v.area64 + rb + static_cast<uint64_t>(k) * rc, kbytes, bar);
  if (with_idx) bulk_g2s(ip, v.area32 + ib, ibytes, bar);
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
    case 1: {
      // the partition wrote this segment as items (code 2^ib + index) when the
      // item fits 64 bits: then the index plane was never written
      const uint32_t* f = v.segf + static_cast<size_t>(seg) * kSegFWords;
      prefetch_segment<1>(buf, v, seg, c, __ldg(f + 16) + __ldg(f + 17) > 64);
      break;
    }
    case 2: prefetch_segment<2>(buf, v, seg, c); break;
    case 3: prefetch_segment<3>(buf, v, seg, c); break;
    default: prefetch_segment<4>(buf, v, seg, c); break;
  }
  return true;
}

// ---- one-key segments: LSD radix sort -----------------------------------
// A one-key segment (words of at most 8 letters) orders its elements by the
// integer (key - kmin) * 2^ib + idx, where key is the word's key without its
// zero tail bytes, kmin the smallest such key in the segment and ib the bit
// width of the largest index: that integer order is the (key, index) order.
// It spans kb + ib bits, kb the width of kmax - kmin.  An item is one uint64
// when kb + ib <= 64 (Item64), else a (key - kmin, idx) pair (Item96).  The
// sort is least-significant-digit first, 8 bits per pass, each pass stable.
struct Item64 {
  uint64_t v;
  __device__ uint32_t digit(uint32_t s, uint32_t) const { return static_cast<uint32_t>(v >> s) & 255u; }
};
struct Item96 {
  uint64_t k;
  uint32_t i;
  // bits [s, s+8) of k * 2^ib + i
  __device__ uint32_t digit(uint32_t s, uint32_t ib) const {
    if (s + 8 <= ib) return (i >> s) & 255u;
    if (s >= ib) return static_cast<uint32_t>(k >> (s - ib)) & 255u;
    return ((i >> s) | static_cast<uint32_t>(k << (ib - s))) & 255u;
  }
};
struct Store64 {
  uint64_t* a;
  __device__ uint64_t* k_or_a() const { return a; }
  __device__ Item64 load(uint32_t p) const { return Item64{a[p]}; }
  __device__ void store(uint32_t p, const Item64& x) const { a[p] = x.v; }
};
struct Store96 {
  uint64_t* k;
  uint32_t* i;
  __device__ uint64_t* k_or_a() const { return k; }
  __device__ Item96 load(uint32_t p) const { return Item96{k[p], i[p]}; }
  __device__ void store(uint32_t p, const Item96& x) const {
    k[p] = x.k;
    i[p] = x.i;
  }
};

// Lanes of the warp holding the same 8-bit digit d (one ballot per bit).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t m = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? m : ~m;
  }
  return peers;
}

// Exclusive prefix sums of the per-warp digit counts hist[w][d] in (digit,
// warp) order, written back in place: afterwards hist[w][d] is the first
// output position of warp w's items with digit d.  Thread t scans the eight
// entries 8t .. 8t+7 of that order (entry e = digit e / warps, warp
// e % warps), so thread order is (digit, warp) order.
__device__ __forceinline__ void scan_digit_counts(uint16_t* hist, uint32_t* warp_tmp) {
  static_assert(kSegThreads * 8 == kRxWarps * kRxDigits, "eight counters per thread");
  static_assert(kRxWarps % 8 == 0, "a thread's eight entries share one digit");
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  uint16_t* h = hist + ((8 * t) % kRxWarps) * kRxDigits + (8 * t) / kRxWarps;  // entry (warp, digit) of 8t
  uint32_t v[8], sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = h[k * kRxDigits];
    sum += v[k];
  }
  const uint32_t inc = warp_inclusive_scan(sum);
  if (lane == 31) warp_tmp[warp] = inc;
  __syncthreads();
  // lane q holds warp q's total: exclusive prefix at my warp
  const uint32_t mine = lane < kRxWarps ? warp_tmp[lane] : 0u;
  const uint32_t upto = warp_inclusive_scan(mine);
  uint32_t run = __shfl_sync(0xffffffffu, upto - mine, warp) + inc - sum;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    h[k * kRxDigits] = static_cast<uint16_t>(run);
    run += v[k];
  }
  __syncthreads();
}

// Bucket pass: the items (distinct integers below 2^bits) are counted by
// their top kMsdBits bits in 2^kMsdBits shared counters and scattered to their
// bucket's range; then every item of a bucket of at most kMsdMaxBucket items
// takes its place in the bucket by counting the smaller items of its bucket.
// A larger bucket (copies of a frequent word share their code bits) is listed
// and split again by the whole block: counted on the kMsd2Bits bits below the
// highest bit in which its items differ, its sub-buckets placed or listed the
// same way, until the list is empty.  Returns false, with the items untouched
// in registers, when a bucket holds more than the planes' scratch capacity:
// then the radix passes run.  cnt holds kMsdBuckets counters, one padding
// word after every kMsdBuckets / kSegThreads of them; aux holds kMsdAuxWords
// words.
constexpr uint32_t kMsdBits = 13;
constexpr uint32_t kMsdBuckets = 1u << kMsdBits;
constexpr uint32_t kMsdMaxBucket = 128;
constexpr uint32_t kMsd2Bits = 10;
constexpr uint32_t kMsd2Buckets = 1u << kMsd2Bits;
// the counter area: the index plane of a one-key segment, key plane 1 of a
// two-key one; a split bucket is copied into the words the sub-counters leave
// free
constexpr uint32_t kMsdAreaWords = 8192;
constexpr uint32_t kMsdScratchWords = kMsdAreaWords - kMsd2Buckets;
// listed buckets are disjoint and larger than kMsdMaxBucket
constexpr uint32_t kMsdList = auto_seg_cap(1) / (kMsdMaxBucket + 1) + 1;
// warp minima and maxima (2 kRxWarps u64, then 2 kRxWarps u32), list, its size
constexpr uint32_t kMsdAuxWords = 6 * kRxWarps + kMsdList + 1;
// The padded counters run up to one word per thread past the counter area
// (into the next plane); the list lives this far into the radix counter area,
// clear of them.
constexpr uint32_t kMsdAuxOffset = 1024;

// Item planes of the bucket pass.  One-word items (Item64): the integer
// itself.  Two-part items (Item96): code k and index i of the integer
// k 2^ib + i, in a u64 and a u32 plane.  bits(v, s) is the low 32 bits of
// v >> s, width(x, y) the bit width of x ^ y.
struct P64 {
  using T = uint64_t;
  uint64_t* a;
  static constexpr uint32_t kScratch = kMsdScratchWords / 2;
  __device__ static T of(const Item64& x) { return x.v; }
  __device__ T ld(uint32_t p) const { return a[p]; }
  __device__ void st(uint32_t p, const T& v) const { a[p] = v; }
  __device__ P64 at(uint32_t p) const { return P64{a + p}; }
  __device__ P64 scratch(uint32_t* area) const { return P64{reinterpret_cast<uint64_t*>(area)}; }
  __device__ static bool lt(const T& x, const T& y) { return x < y; }
  __device__ static T lowest() { return 0ull; }
  __device__ static T highest() { return ~0ull; }
  __device__ static T shfl_xor(const T& x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
  __device__ uint32_t bits(const T& v, uint32_t s) const { return static_cast<uint32_t>(v >> s); }
  __device__ uint32_t width(const T& x, const T& y) const {
    return 64u - static_cast<uint32_t>(__clzll(x ^ y));
  }
};
struct P96 {
  using T = Item96;
  uint64_t* k;
  uint32_t* i;
  uint32_t ib;
  static constexpr uint32_t kScratch = kMsdScratchWords / 3;
  __device__ static T of(const Item96& x) { return x; }
  __device__ T ld(uint32_t p) const { return Item96{k[p], i[p]}; }
  __device__ void st(uint32_t p, const T& v) const {
    k[p] = v.k;
    i[p] = v.i;
  }
  __device__ P96 at(uint32_t p) const { return P96{k + p, i + p, ib}; }
  __device__ P96 scratch(uint32_t* area) const {
    return P96{reinterpret_cast<uint64_t*>(area), area + 2 * kScratch, ib};
  }
  __device__ static bool lt(const T& x, const T& y) { return x.k < y.k || (x.k == y.k && x.i < y.i); }
  __device__ static T lowest() { return Item96{0ull, 0u}; }
  __device__ static T highest() { return Item96{~0ull, ~0u}; }
  __device__ static T shfl_xor(const T& x, int o) {
    return Item96{__shfl_xor_sync(0xffffffffu, x.k, o), __shfl_xor_sync(0xffffffffu, x.i, o)};
  }
  __device__ uint32_t bits(const T& v, uint32_t s) const {
    if (s >= ib) return static_cast<uint32_t>(v.k >> (s - ib));
    return (v.i >> s) | static_cast<uint32_t>(v.k << (ib - s));
  }
  __device__ uint32_t width(const T& x, const T& y) const {
    return x.k != y.k ? ib + 64u - static_cast<uint32_t>(__clzll(x.k ^ y.k))
                      : 32u - static_cast<uint32_t>(__clz(x.i ^ y.i));
  }
};

// Block-wide minimum and maximum of the threads' (lo, hi), through the warp
// slots in aux; every thread gets the result.
template <typename P>
__device__ __forceinline__ void block_min_max(typename P::T& lo, typename P::T& hi, uint32_t* aux) {
  using T = typename P::T;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint64_t* mk = reinterpret_cast<uint64_t*>(aux);  // 2 kRxWarps u64
  uint32_t* mi = aux + 4 * kRxWarps;                // 2 kRxWarps u32
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T p = P::shfl_xor(lo, o), q = P::shfl_xor(hi, o);
    lo = P::lt(p, lo) ? p : lo;
    hi = P::lt(hi, q) ? q : hi;
  }
  if (lane == 0) {
    if constexpr (sizeof(T) == sizeof(uint64_t)) {
      mk[warp] = lo;
      mk[kRxWarps + warp] = hi;
    } else {
      mk[warp] = lo.k;
      mk[kRxWarps + warp] = hi.k;
      mi[warp] = lo.i;
      mi[kRxWarps + warp] = hi.i;
    }
  }
  __syncthreads();
  if constexpr (sizeof(T) == sizeof(uint64_t)) {
    lo = lane < kRxWarps ? mk[lane] : P::highest();
    hi = lane < kRxWarps ? mk[kRxWarps + lane] : P::lowest();
  } else {
    lo = lane < kRxWarps ? Item96{mk[lane], mi[lane]} : P::highest();
    hi = lane < kRxWarps ? Item96{mk[kRxWarps + lane], mi[kRxWarps + lane]} : P::lowest();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T p = P::shfl_xor(lo, o), q = P::shfl_xor(hi, o);
    lo = P::lt(p, lo) ? p : lo;
    hi = P::lt(hi, q) ? q : hi;
  }
}

// Puts every item of a[0..m) at its place within its bucket.  The items lie
// bucket by bucket; bucket d = digit(item) ends at cnt[slot(d)].  Thread t
// takes positions t, t + kSegThreads, ... (a warp: 32 neighbours, mostly of a
// few buckets, whose items it reads as broadcasts), counts the smaller items
// of the bucket and, after a barrier, stores its item at the bucket's start
// plus that count.  A bucket of more than kMsdMaxBucket items stays in place
// and is appended to list as (base0 + start) | size << 16 by the thread
// holding its first item.
template <int E, typename P, typename Digit, typename Slot>
__device__ __forceinline__ void rank_buckets(const P& a, uint32_t m, const uint32_t* cnt, Digit digit,
                                             Slot slot, uint32_t base0, uint32_t* list, uint32_t* n_list) {
  typename P::T v[E];
  uint32_t dst[E];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const uint32_t i = threadIdx.x + k * kSegThreads;
    v[k] = P::lowest();
    dst[k] = ~0u;
    if (i < m) {
      v[k] = a.ld(i);
      const uint32_t d = digit(v[k]);
      const uint32_t lo = d ? cnt[slot(d - 1)] : 0u, hi = cnt[slot(d)];
      if (hi - lo > kMsdMaxBucket) {
        if (i == lo) list[atomicAdd(n_list, 1u)] = (base0 + lo) | ((hi - lo) << 16);
      } else if (hi - lo > 1) {
        uint32_t r = lo;
        for (uint32_t q = lo; q < hi; ++q) r += P::lt(a.ld(q), v[k]) ? 1u : 0u;
        dst[k] = r;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < E; ++k)
    if (dst[k] != ~0u) a.st(dst[k], v[k]);
}

// Splits the listed buckets until none is left (the list is read after a
// barrier).  The counter area holds the copy of the bucket being split
// (P::kScratch items) and its kMsd2Buckets sub-counters.  The items of a
// bucket are distinct: its minimum and maximum differ, the kMsd2Bits window
// ending at their highest differing bit holds at least two digits, and every
// sub-bucket is smaller than its parent, so the splitting ends.
template <typename P>
__device__ __forceinline__ void split_buckets(const P& a, uint32_t* area, uint32_t* aux,
                                              uint32_t* warp_tmp) {
  using T = typename P::T;
  const P scratch = a.scratch(area);
  uint32_t* sub = area + kMsdScratchWords;
  uint32_t* list = aux + 6 * kRxWarps;
  uint32_t* n_list = list + kMsdList;
  constexpr uint32_t per = kMsd2Buckets / kSegThreads;  // sub-counters per thread
  static_assert(per * kSegThreads == kMsd2Buckets, "sub-counters split evenly over the threads");
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  for (;;) {
    const uint32_t t = *n_list;  // block-uniform
    if (t == 0) break;
    const uint32_t e = list[t - 1];
    const uint32_t lo = e & 0xFFFFu, m = e >> 16;
    __syncthreads();  // the entry is read before it is replaced
    if (threadIdx.x == 0) *n_list = t - 1;
    T vmin = P::highest(), vmax = P::lowest();
    for (uint32_t i = threadIdx.x; i < m; i += kSegThreads) {
      const T y = a.ld(lo + i);
      scratch.st(i, y);
      vmin = P::lt(y, vmin) ? y : vmin;
      vmax = P::lt(vmax, y) ? y : vmax;
    }
#pragma unroll
    for (uint32_t k = 0; k < per; ++k) sub[threadIdx.x * per + k] = 0;
    block_min_max<P>(vmin, vmax, aux);
    // distinct items always differ; equal ones (never produced by the
    // encoding) would need no order, and skipping them keeps the loop finite
    if (!P::lt(vmin, vmax)) {
      __syncthreads();  // the copy and the minima are read before reuse
      continue;
    }
    const uint32_t hb = a.width(vmin, vmax);
    const uint32_t sh = hb > kMsd2Bits ? hb - kMsd2Bits : 0u;
    for (uint32_t i = threadIdx.x; i < m; i += kSegThreads)
      atomicAdd(&sub[a.bits(scratch.ld(i), sh) & (kMsd2Buckets - 1)], 1u);
    __syncthreads();
    uint32_t c[per], sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < per; ++k) {
      c[k] = sub[threadIdx.x * per + k];
      sum += c[k];
    }
    const uint32_t inc = warp_inclusive_scan(sum);
    if (lane == 31) warp_tmp[warp] = inc;
    __syncthreads();
    const uint32_t tw = lane < kRxWarps ? warp_tmp[lane] : 0u;
    const uint32_t tupto = warp_inclusive_scan(tw);
    uint32_t run = __shfl_sync(0xffffffffu, tupto - tw, warp) + inc - sum;
#pragma unroll
    for (uint32_t k = 0; k < per; ++k) {
      sub[threadIdx.x * per + k] = run;  // sub-bucket start, then its cursor
      run += c[k];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += kSegThreads) {
      const T y = scratch.ld(i);
      a.st(lo + atomicAdd(&sub[a.bits(y, sh) & (kMsd2Buckets - 1)], 1u), y);
    }
    __syncthreads();
    rank_buckets<(P::kScratch + kSegThreads - 1) / kSegThreads>(
        a.at(lo), m, sub, [a, sh](const T& y) { return a.bits(y, sh) & (kMsd2Buckets - 1); },
        [](uint32_t d) { return d; }, lo, list, n_list);
    __syncthreads();
  }
}

template <int E, typename P, typename It>
__device__ __forceinline__ bool bucket_sort_items(const It (&x)[E], uint32_t nv, uint32_t bits, const P& a,
                                                  uint32_t* cnt, uint32_t* warp_tmp, uint32_t* aux) {
  const uint32_t sh = bits > kMsdBits ? bits - kMsdBits : 0u;
  // items below 2^bits have digits below kMsdBuckets; the clamp keeps every
  // counter access inside the counters whatever the items hold
  const auto digit = [a, sh](const typename P::T& y) { return min(a.bits(y, sh), kMsdBuckets - 1); };
  constexpr uint32_t per = kMsdBuckets / kSegThreads;  // counters per thread
  static_assert(per * kSegThreads == kMsdBuckets && (per & (per - 1)) == 0 && per >= 2,
                "a power-of-two number of counters per thread");
  // thread t's counters (buckets per t .. per t + per - 1) start at word
  // (per + 1) t: the threads of a warp touch 32 different banks when they walk
  // their counters
  const auto slot = [](uint32_t b) { return b + b / per; };
  uint32_t* mine = cnt + threadIdx.x * (per + 1);
#pragma unroll
  for (uint32_t k = 0; k < per; ++k) mine[k] = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (j < nv) atomicAdd(&cnt[slot(digit(P::of(x[j])))], 1u);
  __syncthreads();
  // exclusive scan of the counts (thread t owns counters t*per .. t*per+per-1;
  // read twice rather than held, which keeps registers for the items)
  uint32_t sum = 0, mx = 0;
#pragma unroll
  for (uint32_t k = 0; k < per; ++k) {
    const uint32_t c = mine[k];
    sum += c;
    mx = c > mx ? c : mx;
  }
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t inc = warp_inclusive_scan(sum);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 31) warp_tmp[warp] = inc;
  if (lane == 0) warp_tmp[kRxWarps + warp] = mx;
  __syncthreads();
  const uint32_t tw = lane < kRxWarps ? warp_tmp[lane] : 0u;
  const uint32_t tupto = warp_inclusive_scan(tw);
  uint32_t tm = lane < kRxWarps ? warp_tmp[kRxWarps + lane] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tm = max(tm, __shfl_xor_sync(0xffffffffu, tm, o));
  if (tm > P::kScratch) return false;  // block-uniform
  uint32_t run = __shfl_sync(0xffffffffu, tupto - tw, warp) + inc - sum;
#pragma unroll
  for (uint32_t k = 0; k < per; ++k) {
    const uint32_t c = mine[k];
    mine[k] = run;  // bucket start, then its cursor
    run += c;
  }
  uint32_t* list = aux + 6 * kRxWarps;
  uint32_t* n_list = list + kMsdList;
  if (threadIdx.x == 0) *n_list = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (j < nv) a.st(atomicAdd(&cnt[slot(digit(P::of(x[j])))], 1u), P::of(x[j]));
  __syncthreads();
  // cnt[slot(b)] is now the end of bucket b; bucket b spans [end(b-1), end(b))
  rank_buckets<E>(a, cnt[slot(kMsdBuckets - 1)], cnt, digit, slot, 0u, list, n_list);
  __syncthreads();
  if (tm > kMsdMaxBucket) split_buckets(a, cnt, aux, warp_tmp);  // block-uniform
  return true;
}

// Stable LSD radix sort of c items in the store st: warp w owns positions
// [w S, w S + S) (S = ceil(c / warps) rounded up to 32), lane l holds
// position w S + 32 j + l in x[j].  Each pass ranks the items of a warp in
// position order (running per-warp digit counters hist[w][*] plus the lanes
// below with the same digit), scans the counters, and scatters every item to
// its new position in the store.  The sorted items end in st[0, c).  The
// planes and counters come as shared-memory offsets (a_off: the one-word
// items or the codes, i_off: the indices of two-part items); not inlined, so
// that the bucket pass, which nearly always succeeds, keeps registers of its
// own.
template <typename It, int E>
__device__ __noinline__ void radix_passes(uint32_t a_off, uint32_t i_off, uint32_t hist_off, uint32_t c,
                                          uint32_t bits, uint32_t ib) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  using St = typename std::conditional<sizeof(It) == sizeof(Item64), Store64, Store96>::type;
  St st;
  if constexpr (sizeof(It) == sizeof(Item64)) {
    st = Store64{reinterpret_cast<uint64_t*>(smem_raw + a_off)};
    (void)i_off;
  } else {
    st = Store96{reinterpret_cast<uint64_t*>(smem_raw + a_off), reinterpret_cast<uint32_t*>(smem_raw + i_off)};
  }
  uint16_t* hist = reinterpret_cast<uint16_t*>(smem_raw + hist_off);
  uint32_t* warp_tmp = reinterpret_cast<uint32_t*>(hist + kRxWarps * kRxDigits);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t S = ((c + kRxWarps - 1) / kRxWarps + 31) & ~31u;
  const uint32_t w0 = warp * S, p0 = w0 + lane, lt = lanemask_lt();
  // item j is in the warp's range when j < nr (warp-uniform) and holds a
  // position below c as well when j < nv (<= nr)
  const uint32_t nr = S / 32, nv = min(nr, c > p0 ? (c - p0 + 31) / 32 : 0u);
  uint16_t* row = hist + warp * kRxDigits;
  It x[E];
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (j < nv) x[j] = st.load(p0 + 32 * j);
  __syncthreads();
  uint32_t rk[(E + 1) / 2];  // ranks, two 16-bit fields per word
  for (uint32_t s = 0; s < bits; s += 8) {
    for (uint32_t i = lane; i < kRxDigits; i += 32) row[i] = 0;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (j < nr) {  // warp-uniform
        const bool valid = j < nv;
        const uint32_t vm = __ballot_sync(0xffffffffu, valid);
        const uint32_t d = x[j].digit(s, ib);
        const uint32_t peers = digit_peers(d) & vm;
        const uint32_t leader = (__ffs(peers) - 1) & 31u;
        uint32_t base = 0;
        if (valid && lane == leader) {
          base = row[d];
          row[d] = static_cast<uint16_t>(base + __popc(peers));
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        const uint32_t r = base + __popc(peers & lt);
        if (j & 1) rk[j / 2] |= r << 16;
        else rk[j / 2] = r;
        __syncwarp();
      }
    }
    __syncthreads();
    scan_digit_counts(hist, warp_tmp);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (j < nv) {
        const uint32_t r = (j & 1) ? rk[j / 2] >> 16 : rk[j / 2] & 0xffffu;
        st.store(row[x[j].digit(s, ib)] + r, x[j]);
      }
    }
    __syncthreads();
    if (s + 8 < bits) {
#pragma unroll
      for (int j = 0; j < E; ++j)
        if (j < nv) x[j] = st.load(p0 + 32 * j);
    }
  }
}

// Sorts c items read through get(p): the bucket pass (bucket counters given)
// into bp, else the radix passes into st; returns whether the bucket pass
// did it.  Items are held in registers as in radix_passes.
template <typename It, typename St, int E, typename Get, typename BP>
__device__ __forceinline__ bool radix_sort_items(Get get, uint32_t c, uint32_t bits, uint32_t ib,
                                                 St st, uint16_t* hist, uint32_t* warp_tmp,
                                                 uint32_t* bucket_cnt, const BP& bp) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t S = ((c + kRxWarps - 1) / kRxWarps + 31) & ~31u;
  const uint32_t p0 = warp * S + lane;
  const uint32_t nr = S / 32, nv = min(nr, c > p0 ? (c - p0 + 31) / 32 : 0u);
  It x[E];
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (j < nv) x[j] = get(p0 + 32 * j);
  // every item is read before the first pass scatters into the store
  __syncthreads();
  // byte-recoded keys spread their top bits: the bucket pass is tried first
  if (bucket_cnt && bits > 8 &&
      bucket_sort_items<E>(x, nv, bits, bp, bucket_cnt, warp_tmp,
                           reinterpret_cast<uint32_t*>(hist) + kMsdAuxOffset))
    return true;
  // the items go to the store at their positions, the radix passes take them
  // from there
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (j < nv) st.store(p0 + 32 * j, x[j]);
  __syncthreads();
  const auto off = [](const void* q) {
    return static_cast<uint32_t>(reinterpret_cast<const uint8_t*>(q) - smem_raw);
  };
  uint32_t i_off = 0;
  if constexpr (sizeof(It) != sizeof(Item64)) i_off = off(st.i);
  radix_passes<It, E>(off(st.k_or_a()), i_off, off(hist), c, bits, ib);
  return false;
}

// Sorts the segment's items (converted from the key and index planes, which
// are then reused as the item store); k1_write then writes the output
// records.  The buffer comes as an offset into dynamic shared memory, so that
// every access compiles to a shared-memory instruction.  Not inlined, and
// apart from the writing: the items need the registers, and the writing loop
// keeps its parameters in registers of its own.  Returns the shared-memory
// offset of the plane that holds the sorted indices of two-part items (0 for
// one-word items, whose indices are their low bits).
template <typename It, int E>
__device__ __noinline__ uint32_t k1_radix(uint32_t buf_off, uint32_t c, ByteCode bc, uint32_t kb,
                                          uint32_t ib) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr uint32_t C = auto_seg_cap(1);
  uint64_t* kp = reinterpret_cast<uint64_t*>(smem_raw + buf_off);
  uint32_t* ip = reinterpret_cast<uint32_t*>(kp + C);
  uint16_t* hist = reinterpret_cast<uint16_t*>(ip + C);
  uint32_t* warp_tmp = reinterpret_cast<uint32_t*>(hist + kRxWarps * kRxDigits);
  uint32_t idx_off = 0;
  if constexpr (sizeof(It) == sizeof(Item64)) {
    // the partition wrote these segments as items (code 2^ib + index)
    auto get = [=](uint32_t p) { return Item64{kp[p]}; };
    // the index plane is free: bucket counters
    radix_sort_items<It, Store64, E>(get, c, kb + ib, ib, Store64{kp}, hist, warp_tmp, ip, P64{kp});
  } else {
    auto get = [=](uint32_t p) { return Item96{bc.encode(kp[p]), ip[p]}; };
    // up to half the capacity, the bucket pass keeps the codes in the key
    // plane and the indices in its upper half, the counters in the index plane
    constexpr uint32_t H = C / 2;
    const P96 bp{kp, reinterpret_cast<uint32_t*>(kp + H), ib};
    const bool bucketed = radix_sort_items<It, Store96, E>(get, c, kb + ib, ib, Store96{kp, ip}, hist, warp_tmp,
                                                           c <= H ? ip : nullptr, bp);
    idx_off = buf_off + (bucketed ? H * 8 : C * 8);
  }
  __syncthreads();
  return idx_off;
}

// Output records and permutation of a sorted one-key segment: codes (with the
// index in their low ib bits when idx_off is 0, else in the plane at idx_off)
// in the key plane at buf_off.
template <typename Sink>
__device__ __noinline__ void k1_write(uint32_t buf_off, uint32_t idx_off, uint32_t c, ByteCode bc, uint32_t ib,
                                      uint32_t ob, Sink o) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint64_t* kp = reinterpret_cast<const uint64_t*>(smem_raw + buf_off);
  if (idx_off == 0) {
    const uint64_t imask = (1ull << ib) - 1;
    for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) {
      const uint64_t v = kp[r];
      Elem<1> e;
      e.k[0] = bc.decode(v >> ib);
      e.idx = static_cast<uint32_t>(v & imask);
      o.template put<1>(ob + r, e);
    }
  } else {
    const uint32_t* op = reinterpret_cast<const uint32_t*>(smem_raw + idx_off);
    for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) {
      Elem<1> e;
      e.k[0] = bc.decode(kp[r]);
      e.idx = op[r];
      o.template put<1>(ob + r, e);
    }
  }
  __syncthreads();
}

// Segments of words with two or more key words (longer than 8 letters, a
// small share of typical text) whose code does not fit the item sort: a
// bitonic network in shared memory, which keeps no elements in registers.
// (A register network over (first key word, slot) pairs was measured slower
// for these segments.)
template <int K, typename Sink>
__device__ void sort_resident(uint8_t* buf, const AutoView& v, uint32_t seg, uint32_t c,
                              const Sink& o) {
  uint64_t* kp = reinterpret_cast<uint64_t*>(buf + 16);
  const uint32_t C = static_cast<uint32_t>(seg_plane_elems(K));
  SmemTile<K> t;
#pragma unroll
  for (int k = 0; k < K; ++k) t.k[k] = kp + k * C;
  t.idx = reinterpret_cast<uint32_t*>(kp + static_cast<size_t>(K) * C);
  bitonic_flip<K>(t, c);
  __syncthreads();
  const uint32_t ob = v.outbase[seg];
  for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) o.template put<K>(ob + r, t.get(r));
  __syncthreads();
}

// Two-key segments (words of 9 to 16 letters) whose byte code fits 64 bits:
// the same item sort on the code of all 16 byte positions.  The code table
// (16 fields, as in ByteCode) is read from shared memory at f.  Key planes 0
// and 1 and the index plane hold the segment; plane 0 becomes the item store
// and plane 1 the bucket counters.
__device__ __forceinline__ uint64_t encode16(const uint32_t* f, uint64_t k0, uint64_t k1) {
  uint64_t code = 0;
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const uint64_t k = p < 8 ? k0 : k1;
    const uint32_t b = static_cast<uint32_t>(k >> (56 - 8 * (p & 7))) & 255u;
    code |= static_cast<uint64_t>(b - (f[p] & 255u)) << ((f[p] >> 8) & 63u);
  }
  return code;
}
__device__ __forceinline__ void decode16(const uint32_t* f, uint64_t code, Elem<2>& e) {
  e.k[0] = 0;
  e.k[1] = 0;
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const uint32_t b = static_cast<uint32_t>(code >> ((f[p] >> 8) & 63u)) & ((1u << (f[p] >> 16)) - 1u);
    e.k[p >> 3] |= static_cast<uint64_t>(b + (f[p] & 255u)) << (56 - 8 * (p & 7));
  }
}

template <typename It, int E>
__device__ __noinline__ uint32_t k2_radix(uint32_t buf_off, uint32_t c, const uint32_t* f, uint32_t kb,
                                          uint32_t ib) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr uint32_t C = auto_seg_cap(2);
  static_assert(2 * C >= kMsdBuckets, "plane 1 holds the bucket counters");
  uint64_t* k0p = reinterpret_cast<uint64_t*>(smem_raw + buf_off);
  uint64_t* k1p = k0p + C;
  uint32_t* ip = reinterpret_cast<uint32_t*>(k1p + C);
  uint16_t* hist = reinterpret_cast<uint16_t*>(ip + C);
  uint32_t* warp_tmp = reinterpret_cast<uint32_t*>(hist + kRxWarps * kRxDigits);
  uint32_t idx_off = 0;
  if constexpr (sizeof(It) == sizeof(Item64)) {
    auto get = [=](uint32_t p) { return Item64{(encode16(f, k0p[p], k1p[p]) << ib) | ip[p]}; };
    radix_sort_items<It, Store64, E>(get, c, kb + ib, ib, Store64{k0p}, hist, warp_tmp,
                                     reinterpret_cast<uint32_t*>(k1p), P64{k0p});
  } else {
    auto get = [=](uint32_t p) { return Item96{encode16(f, k0p[p], k1p[p]), ip[p]}; };
    // the bucket pass keeps the codes in plane 0 and the indices in the lower
    // half of plane 1; its counters take the upper half and the index plane
    const P96 bp{k0p, reinterpret_cast<uint32_t*>(k1p), ib};
    const bool bucketed = radix_sort_items<It, Store96, E>(get, c, kb + ib, ib, Store96{k0p, ip}, hist, warp_tmp,
                                                           reinterpret_cast<uint32_t*>(k1p + C / 2), bp);
    idx_off = buf_off + (bucketed ? C * 8 : 2 * C * 8);
  }
  __syncthreads();
  return idx_off;
}

// Output records and permutation of a sorted two-key segment (as k1_write).
template <typename Sink>
__device__ __noinline__ void k2_write(uint32_t buf_off, uint32_t idx_off, uint32_t c, const uint32_t* f,
                                      uint32_t ib, uint32_t ob, Sink o) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint64_t* k0p = reinterpret_cast<const uint64_t*>(smem_raw + buf_off);
  if (idx_off == 0) {
    const uint64_t imask = (1ull << ib) - 1;
    for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) {
      const uint64_t v = k0p[r];
      Elem<2> e;
      decode16(f, v >> ib, e);
      e.idx = static_cast<uint32_t>(v & imask);
      o.template put<2>(ob + r, e);
    }
  } else {
    const uint32_t* op = reinterpret_cast<const uint32_t*>(smem_raw + idx_off);
    for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) {
      Elem<2> e;
      decode16(f, k0p[r], e);
      e.idx = op[r];
      o.template put<2>(ob + r, e);
    }
  }
  __syncthreads();
}

// Two-key segment resident in buf: a code (from the segment's record) of at
// most 64 bits takes the item sort, a wider one the bitonic network.  Returns
// false when the code is too wide.
template <typename Sink>
__device__ bool sort_resident_k2(const uint8_t* smem_base, uint8_t* buf, const AutoView& v,
                                 uint32_t seg, uint32_t c, const Sink& o) {
  __shared__ uint32_t s_f2[16], s_kb2, s_ib2;
  const uint32_t* sf = v.segf + static_cast<size_t>(seg) * kSegFWords;
  if (threadIdx.x < 16) s_f2[threadIdx.x] = __ldg(sf + threadIdx.x);
  else if (threadIdx.x == 16) s_kb2 = __ldg(sf + 16);
  else if (threadIdx.x == 17) s_ib2 = __ldg(sf + 17);
  __syncthreads();
  const uint32_t kb = s_kb2, ib = s_ib2;
  if (kb > 64) return false;  // block-uniform
  const uint32_t ob = v.outbase[seg];
  const uint32_t off = static_cast<uint32_t>(buf + 16 - smem_base);
  uint32_t idx_off;
  if (kb + ib <= 64) {
    if (c <= 4 * kSegThreads) idx_off = k2_radix<Item64, 4>(off, c, s_f2, kb, ib);
    else idx_off = k2_radix<Item64, 8>(off, c, s_f2, kb, ib);
  } else {
    if (c <= 4 * kSegThreads) idx_off = k2_radix<Item96, 4>(off, c, s_f2, kb, ib);
    else idx_off = k2_radix<Item96, 8>(off, c, s_f2, kb, ib);
  }
  k2_write(off, idx_off, c, s_f2, ib, ob, o);
  return true;
}

// One-key segment resident in buf: its byte code (from the segment's record)
// recodes the keys, then the (code, index) items are sorted.
template <typename Sink>
__device__ void sort_resident_k1(const uint8_t* smem_base, uint8_t* buf, const AutoView& v,
                                 uint32_t seg, uint32_t c, const Sink& o) {
  const uint32_t* sf = v.segf + static_cast<size_t>(seg) * kSegFWords;
  ByteCode bc;
  bc.lo = (static_cast<uint64_t>(__ldg(sf + 18)) << 32) | __ldg(sf + 19);
  const uint32_t shape = __ldg(sf + 20);
  bc.p0 = shape & 255u;
  bc.w0 = (shape >> 8) & 255u;
  bc.wl = (shape >> 16) & 255u;
  bc.n = shape >> 24;
  const uint32_t kb = __ldg(sf + 16), ib = __ldg(sf + 17);
  const uint32_t ob = v.outbase[seg];
  const uint32_t off = static_cast<uint32_t>(buf + 16 - smem_base);
  uint32_t idx_off;
  if (kb + ib <= 64) {
    if (c <= 4 * kSegThreads) idx_off = k1_radix<Item64, 4>(off, c, bc, kb, ib);
    else if (c <= 6 * kSegThreads) idx_off = k1_radix<Item64, 6>(off, c, bc, kb, ib);
    else if (c <= 8 * kSegThreads) idx_off = k1_radix<Item64, 8>(off, c, bc, kb, ib);
    else idx_off = k1_radix<Item64, 16>(off, c, bc, kb, ib);
  } else {
    if (c <= 4 * kSegThreads) idx_off = k1_radix<Item96, 4>(off, c, bc, kb, ib);
    else if (c <= 8 * kSegThreads) idx_off = k1_radix<Item96, 8>(off, c, bc, kb, ib);
    else idx_off = k1_radix<Item96, 16>(off, c, bc, kb, ib);
  }
  k1_write(off, idx_off, c, bc, ib, ob, o);
}

// A segment larger than shared memory (after a retry) and a resident one.
template <typename Sink>
__device__ __forceinline__ void sort_big(uint8_t* scratch, const AutoView& v, uint32_t seg, uint32_t c,
                                         uint32_t K, const Sink& o) {
  switch (K) {
    case 1: segsort_big<1>(scratch, v, seg, c, o); break;
    case 2: segsort_big<2>(scratch, v, seg, c, o); break;
    case 3: segsort_big<3>(scratch, v, seg, c, o); break;
    default: segsort_big<4>(scratch, v, seg, c, o); break;
  }
}

template <typename Sink>
__device__ __forceinline__ void sort_resident_any(const uint8_t* smem_base, uint8_t* buf, const AutoView& v,
                                                  uint32_t seg, uint32_t c, uint32_t K, const Sink& o) {
  switch (K) {
    case 1: sort_resident_k1(smem_base, buf, v, seg, c, o); break;
    case 2:
      if (!sort_resident_k2(smem_base, buf, v, seg, c, o)) sort_resident<2>(buf, v, seg, c, o);
      break;
    case 3: sort_resident<3>(buf, v, seg, c, o); break;
    default: sort_resident<4>(buf, v, seg, c, o); break;
  }
}

// Destinations of the segment sort: records (rec) or the packed form (bytes,
// offsets, cap, with the bucket offsets off); the permutation either way.
struct SegOut {
  uint8_t* rec;
  uint32_t* perm;
  uint8_t* bytes;
  uint32_t* offsets;
  uint64_t cap;
  const uint32_t* off;
};

// Persistent CTAs (two per SM) walk the segments: bulk-copy the segment into
// shared memory, sort, write the output records (or packed words) and the
// permutation.
template <bool kPacked>
__global__ void __launch_bounds__(kSegThreads, 2)
auto_segsort_kernel(uint32_t W, Ws ws, AutoView av, SegOut out) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* buf = smem_raw;  // 16-byte aligned: barrier, then the planes
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf);
  const AutoView& v = av;  // kernel parameter: read from the constant bank
  __shared__ uint32_t s_base[kPacked ? kMaxW + 2 : 1];
  __shared__ uint32_t s_fits;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    if constexpr (kPacked) {
      const uint32_t total = packed_bases(out.off, W, s_base);
      s_fits = total <= out.cap;
      if (blockIdx.x == 0) {
        out.offsets[out.off[W + 1]] = s_fits ? total : 0u;
        if (!s_fits) set_error(ws.hdr, BSORT_E_CAPACITY);
      }
    }
  }
  __syncthreads();
  const uint32_t G = v.hdr->G;
  uint32_t phase = 0;
  __shared__ uint32_t s_next;
  for (;;) {
    // segments are handed out one at a time, longest words first (their
    // segments cost the most per word), so the CTAs finish together
    if (threadIdx.x == 0) s_next = atomicAdd(&v.hdr->next_seg, 1u);
    __syncthreads();
    const uint32_t t = s_next;
    __syncthreads();
    if (t >= G) break;
    const uint32_t seg = G - 1 - t;
    const uint32_t c = seg_count(v, seg);
    const uint32_t L = v.segL[seg];
    const uint32_t K = keys_for_len(L);
    if (c == 0) continue;
    if (c > auto_seg_cap(K)) {
      // larger than shared memory (after a retry): chunked sort + merges
      if constexpr (kPacked)
        sort_big(buf + 16, v, seg, c, K, PackSink{out.bytes, out.offsets, out.perm, L, s_base[L], s_fits});
      else
        sort_big(buf + 16, v, seg, c, K, RecSink{out.rec, out.perm, W});
      continue;
    }
    // earlier generic-proxy use of the buffer must be ordered before the bulk
    // copy (async proxy) overwrites it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) maybe_prefetch(buf, v, seg, G);
    const bool ok = mbar_wait_bounded(bar, phase, ws.wait_polls);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        set_error(ws.hdr, BSORT_E_TIMEOUT);
        mbar_wait_bounded(bar, phase ^ 1u);  // let the copy in flight land before exiting
      }
      return;
    }
    if constexpr (kPacked)
      sort_resident_any(smem_raw, buf, v, seg, c, K,
                        PackSink{out.bytes, out.offsets, out.perm, L, s_base[L], s_fits});
    else
      sort_resident_any(smem_raw, buf, v, seg, c, K, RecSink{out.rec, out.perm, W});
  }
}

// ---------------------------------------------------------------------------
// 0. length histogram (totals only) and bucket offsets
// ---------------------------------------------------------------------------
constexpr uint32_t kHistThreads = 256;

// Each thread counts in its own shared-memory column (no contention), then
// the block adds its column sums to the global totals: one atomic per length
// per block.  Lengths are read 16 per load, two loads in flight per thread.
__device__ __forceinline__ void hist_count(uint32_t L, uint32_t W, uint32_t* col, bool& bad_zero,
                                           bool& bad_long) {
  bad_zero |= L == 0;
  bad_long |= L > W;
  if (L >= 1 && L <= W) atomicAdd(&col[L * kHistThreads], 1u);  // reduction: no read-back
}

__global__ void __launch_bounds__(kHistThreads)
auto_hist_kernel(const uint8_t* __restrict__ len, uint32_t n_cap, const uint32_t* __restrict__ d_n,
                 uint32_t W, Ws ws, AutoView av) {
  __shared__ uint32_t cnt[kBins][kHistThreads];
  const AutoView& v = av;
  for (uint32_t L = 0; L < kBins; ++L) cnt[L][threadIdx.x] = 0;
  uint32_t* col = &cnt[0][threadIdx.x];
  const uint32_t n = word_count(n_cap, d_n);
  bool bad_zero = false, bad_long = false;
  const uint32_t gtid = blockIdx.x * kHistThreads + threadIdx.x, stride = gridDim.x * kHistThreads;
  // bytes before the first 16-byte boundary, then 16-byte groups, then the tail
  const uint32_t head = min(n, static_cast<uint32_t>((16u - (reinterpret_cast<uintptr_t>(len) & 15u)) & 15u));
  const uint32_t n16 = (n - head) / 16;
  if (gtid < head) hist_count(len[gtid], W, col, bad_zero, bad_long);
  const uint4* l16 = reinterpret_cast<const uint4*>(len + head);
  for (uint32_t q = gtid; q < n16; q += 2 * stride) {
    const uint4 a = __ldg(l16 + q);
    const bool two = q + stride < n16;
    const uint4 b = two ? __ldg(l16 + q + stride) : make_uint4(0, 0, 0, 0);
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) hist_count((wa[k >> 2] >> (8 * (k & 3))) & 255u, W, col, bad_zero, bad_long);
    if (two) {
#pragma unroll
      for (int k = 0; k < 16; ++k) hist_count((wb[k >> 2] >> (8 * (k & 3))) & 255u, W, col, bad_zero, bad_long);
    }
  }
  for (uint32_t i = head + 16 * n16 + gtid; i < n; i += stride) hist_count(len[i], W, col, bad_zero, bad_long);
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
__global__ void auto_offsets_kernel(uint32_t W, Ws ws, AutoView av, uint32_t* __restrict__ off) {
  __shared__ uint32_t tot[kBins], so[kMaxW + 2];
  const AutoView& v = av;
  const uint32_t L = threadIdx.x;
  if (L < kBins) tot[L] = (L >= 1 && L <= W) ? v.hdr->total[L] : 0u;
  __syncthreads();
  if (L <= W + 1) {
    uint32_t s = 0;
    for (uint32_t l = 1; l < L && l <= W; ++l) s += tot[l];
    off[L] = s;
    so[L] = s;
  }
  __syncthreads();
  // every later kernel reads its buckets' plans from here
  if (L < kBins) v.hdr->plans[L] = (L >= 1 && L <= W) ? plan_for(so, L, v.cap) : BucketPlan{};
  if (L < kMaxW + 2) ws.hdr->final_buf[L] = 0;
  if (L < kBins) {
    v.hdr->samp_cnt[L] = 0;
    v.hdr->bcur[L] = 0;
  }
  if (L == 0) {
    v.hdr->overflow = 0;
    v.hdr->retry = 0;
    v.hdr->next_seg = 0;
    v.hdr->band = 255;
    v.hdr->bor = 0;
  }
}

static_assert(seg_plane_elems(1) * 12 <= kSegPlanesBytes && seg_plane_elems(2) * 20 <= kSegPlanesBytes &&
                  seg_plane_elems(3) * 28 <= kSegPlanesBytes && seg_plane_elems(4) * 36 <= kSegPlanesBytes,
              "segment planes exceed the shared-memory budget");
static_assert(16 * kSegThreads >= auto_seg_cap(1), "16 radix items per thread cover a one-key segment");
static_assert(auto_seg_cap(1) * 12 + kRxHistBytes <= kSegPlanesBytes,
              "one-key planes and radix counters exceed the segment buffer");
static_assert(9 * kRxWarps * 4 <= kRxHistBytes, "reduction scratch fits the radix counters");
static_assert(auto_seg_cap(2) * 20 + kRxHistBytes <= kSegPlanesBytes, "two-key planes and radix counters fit");
static_assert(auto_seg_cap(2) <= 8 * kSegThreads, "eight radix items per thread cover a two-key segment");
static_assert(kMsdBuckets <= auto_seg_cap(1), "bucket counters fit the index plane");
static_assert((kMsdAuxOffset + kMsdAuxWords) * 4 <= kRxWarps * kRxDigits * sizeof(uint16_t),
              "split list fits the radix counters");
// two-part items: one-key segments keep their indices in the upper half of
// the key plane (segments of at most half the capacity), two-key segments in
// the lower half of key plane 1, whose upper half and the index plane hold the
// counters
static_assert(auto_seg_cap(1) / 2 * 12 <= auto_seg_cap(1) * 8 && auto_seg_cap(2) * 4 <= auto_seg_cap(2) / 2 * 8 &&
                  auto_seg_cap(2) / 2 * 8 + auto_seg_cap(2) * 4 >= kMsdBuckets * 4,
              "two-part item planes and counters fit the segment planes");
// one-key segments: counters in the index plane and the first words of the
// radix counters; two-key segments: in key plane 1 and the first words of the
// index plane
static_assert(kMsdBuckets + kSegThreads <= kMsdAreaWords + kMsdAuxOffset && kMsdBuckets <= kMsdAreaWords &&
                  kMsdBuckets + kSegThreads <= kMsdAreaWords + auto_seg_cap(2),
              "padded bucket counters stay clear of the split list");
static_assert(2 * P64::kScratch + kMsd2Buckets <= kMsdAreaWords && 3 * P96::kScratch + kMsd2Buckets <= kMsdAreaWords &&
                  auto_seg_cap(1) < 65536,
              "split copy and sub-counters fit the counter area; list entries pack start and size");
// two CTAs per SM: dynamic + static (at most 256 bytes: the workspace view and
// a few scalars; ptxas -v reports it) + 1 KB reserved each
static_assert(2 * (segsort_smem_bytes() + 256 + 1024) <= 228 * 1024, "two segsort CTAs must fit an SM");

cudaError_t partition(uint32_t W, const uint32_t* d_off, const Ws& ws, const AutoView& v, int retry,
                      cudaStream_t s) {
  static SmemOptIn set;
  cudaError_t e = ensure_smem(auto_partition_kernel, kPartSmem, &set);
  if (e != cudaSuccess) return e;
  const uint32_t grid = static_cast<uint32_t>(device_sm_count());
  BSORT_LAUNCH(retry ? "auto_partition_retry" : "auto_partition", auto_partition_kernel, grid,
               kPartThreads2, kPartSmem, s, W, d_off, retry, ws, v);
  return cudaGetLastError();
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
                        uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s, const PackOut* pk) {
  static SmemOptIn split_set, select_set, seg_set, seg_packed_set;
  cudaError_t e = ensure_smem(auto_spl_sort_kernel, kSplSortSmem, &split_set);
  if (e == cudaSuccess) e = ensure_smem(auto_spl_select_kernel, kSplSelectSmem, &select_set);
  if (e == cudaSuccess && !pk) e = ensure_smem(auto_segsort_kernel<false>, segsort_smem_bytes(), &seg_set);
  if (e == cudaSuccess && pk)
    e = ensure_smem(auto_segsort_kernel<true>, segsort_smem_bytes(), &seg_packed_set);
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const uint32_t samples = n_cap / kAutoSampleEvery + 1;
  // the workspace view, computed once here and passed to every kernel
  const AutoView v = auto_view(ws, W);
  // phase 2 counts: totals per length, then bucket offsets
  e = cudaMemsetAsync(v.hdr->total, 0, sizeof(v.hdr->total), s);
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("auto_hist", auto_hist_kernel, static_cast<uint32_t>(sms) * 4, kHistThreads,
               0, s, len, n_cap, d_n, W, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BSORT_LAUNCH("auto_offsets", auto_offsets_kernel, 1, 64, 0, s, W, ws, v, d_off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // The samples and their sort into splitters need only the bucket plans, so
  // they run on the thread's helper stream while the bucket pass (bound by
  // HBM) stages the words; the splitter directory needs the bucket pass's byte
  // bounds and waits for both.
  SideStream* ss = side_stream();
  cudaStream_t t = s;
  if (ss) {
    if ((e = cudaEventRecord(ss->fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ss->side, ss->fork, 0)) != cudaSuccess) return e;
    t = ss->side;
  }
  BSORT_LAUNCH("auto_sample", auto_sample_kernel, (samples + 255) / 256, 256, 0, t, rec, len,
               n_cap, d_n, W, d_off, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BSORT_LAUNCH("auto_spl_sort", auto_spl_sort_kernel, dim3(W, kSplChunks), 1024, kSplSortSmem, t,
               d_off, W, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BSORT_LAUNCH("auto_spl_select", auto_spl_select_kernel, dim3(W, kSplChunks), 1024, kSplSelectSmem,
               t, d_off, W, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ss && (e = cudaEventRecord(ss->join, ss->side)) != cudaSuccess) return e;
  BSORT_LAUNCH("auto_bucket", auto_bucket_kernel, static_cast<uint32_t>(sms) * 2, kBucketThreads,
               0, s, rec, len, n_cap, d_n, W, d_off, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ss && (e = cudaStreamWaitEvent(s, ss->join, 0)) != cudaSuccess) return e;
  BSORT_LAUNCH("auto_spl_dir", auto_spl_dir_kernel, dim3(W, kSplDirCtas), 288, 0, s, d_off, W, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = partition(W, d_off, ws, v, 0, s);
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("auto_layout", auto_layout_kernel, 1, 1024, 0, s, W, ws, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = partition(W, d_off, ws, v, 1, s);
  if (e != cudaSuccess) return e;
  const SegOut out{out_rec, out_perm, pk ? pk->bytes : nullptr, pk ? pk->offsets : nullptr,
                   pk ? pk->cap : 0, d_off};
  if (pk) {
    BSORT_LAUNCH("auto_segsort_packed", auto_segsort_kernel<true>, static_cast<uint32_t>(sms) * 2,
                 kSegThreads, segsort_smem_bytes(), s, W, ws, v, out);
  } else {
    BSORT_LAUNCH("auto_segsort", auto_segsort_kernel<false>, static_cast<uint32_t>(sms) * 2,
                 kSegThreads, segsort_smem_bytes(), s, W, ws, v, out);
  }
  return cudaGetLastError();
}

}  // namespace bsort
