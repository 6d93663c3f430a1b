// Batched form: many independent word lists sorted by persistent kernels on
// the call's stream, two planning kernels on a helper stream forked from it
// and joined back (capturable as one CUDA graph).
//
// The method of §3 Methodology, "Pre-processing" (phase 1 tokenise, phase 2
// buckets by length, phase 3 sort each bucket, then concatenation) runs for
// every list at once: a bucket is a (list, length) pair, and every kernel
// walks a flat work list (list chunks, (list, length) tiles, merge
// partitions) with a grid-stride loop over a fixed, SM-sized grid.
//
//   many_init_kernel    validate descriptors, reset per-list state
//   many_tok_kernel     text mode: one CTA per list tokenises its text
//                       (ballot word starts, block scan, records in order)
//   many_plan_kernel    chunks of 4096 words per list -> item numbering
//   many_hist_kernel    per-item length histogram
//   many_lscan_kernel   per list: bucket offsets, per-item scatter bases,
//                       (list, length) segment table
//   many_scatter_kernel stable scatter + big-endian key packing
//   many_tplan_kernel   tiles per segment (prefix sums)
//   many_tile_kernel    odd-even or bitonic tile sort (TMA-staged), as in
//                       the single-list path
//   many_pplan_kernel   partitions of every merge pass (segments ordered by
//                       their pass count, one prefix sum)
//   many_merge_kernel   merge-path passes per segment
//   many_gather_kernel  records and permutation (index within the list)
//   many_finish_kernel  per-list status
#include "block_scan.cuh"
#include "common.cuh"
#include "kernels.h"
#include "sort_impl.cuh"
#include "tok_impl.cuh"

namespace bsort {

namespace {

constexpr uint32_t kItemWords = 4096;  // words per chunk item
constexpr uint32_t kThreads = 256;
constexpr uint32_t kWarps = kThreads / 32;

struct ListState {
  uint32_t n;      // words of the list (after tokenising / clamping to capacity)
  uint32_t flags;  // bit c: error code c seen for this list
};

// Passes of a merge sort over at most 2^32 positions from tiles of >= 64.
constexpr uint32_t kMaxPasses = 32;

struct ManyHdr {
  uint32_t items, tiles, flags;
  uint32_t active;                 // segments that take at least one merge pass
  uint32_t pass_parts[kMaxPasses];  // partitions of merge pass p
};
static_assert(sizeof(ManyHdr) <= 256, "the header's WsHeader starts at byte 256");

// Workspace of bsort_sort_many, a pure function of (cap, W, n_lists).
struct ManyLayout {
  size_t header, lists, item_start, segs, seg_cnt, tile_pre, part_pre, seg_ord, table, keys_a,
      keys_b, idx_a, idx_b, trec, tlen, total;
  uint64_t cap, items_max;
};

constexpr ManyLayout many_layout_cap(uint64_t cap, uint32_t W, uint32_t n_lists) {
  ManyLayout l{};
  const uint32_t K = W / 8;
  const uint64_t S = static_cast<uint64_t>(n_lists) * W;
  l.cap = cap;
  l.items_max = cap / kItemWords + n_lists + 1;
  size_t o = 0;
  l.header = o;  // ManyHdr at 0, a WsHeader (device-detected timeouts) at 256
  o += 4096 + 256;
  l.lists = o;
  o += align_up(sizeof(ListState) * n_lists, 256);
  l.item_start = o;
  o += align_up(4 * (n_lists + 1ull), 256);
  l.segs = o;
  o += align_up(4 * S, 256);
  l.seg_cnt = o;
  o += align_up(4 * S, 256);
  l.tile_pre = o;
  o += align_up(4 * (S + 1), 256);
  l.part_pre = o;
  o += align_up(4 * (S + 1), 256);
  l.seg_ord = o;
  o += align_up(4 * S, 256);
  l.table = o;
  o += align_up(4 * l.items_max * (W + 1), 256);
  l.keys_a = o;
  o += align_up(8 * cap * K, 256);
  l.keys_b = o;
  o += align_up(8 * cap * K, 256);
  l.idx_a = o;
  o += align_up(4 * cap, 256);
  l.idx_b = o;
  o += align_up(4 * cap, 256);
  l.trec = o;
  o += align_up(cap * W, 256);
  l.tlen = o;
  o += align_up(cap, 256);
  l.total = o;
  return l;
}

ManyLayout many_layout_bytes(size_t ws_bytes, uint32_t W, uint32_t n_lists) {
  const size_t fixed = many_layout_cap(0, W, n_lists).total;
  if (ws_bytes <= fixed) return many_layout_cap(0, W, n_lists);
  uint64_t lo = 0, hi = (ws_bytes - fixed) / (W + 1 + 8 * W / 4) / 64 + 1;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;
    if (many_layout_cap(mid * 64, W, n_lists).total <= ws_bytes) lo = mid;
    else hi = mid - 1;
  }
  return many_layout_cap(lo * 64, W, n_lists);
}

struct Many {
  ManyHdr* hdr;
  ListState* ls;
  const bsort_list* lists;
  uint32_t n_lists, W, T, part;
  uint32_t* item_start;
  uint32_t* seg_start;
  uint32_t* seg_cnt;
  uint32_t* tile_pre;
  uint32_t* part_pre;  // over seg_ord[0 .. active)
  uint32_t* seg_ord;   // segments that take merge passes, most passes first
  uint32_t* table;
  uint8_t* trec;
  uint8_t* tlen;
  Ws ws;  // keys / idx ping-pong buffers (hdr unused: statuses are per list)
  uint64_t cap;
};

Many many_view(void* base, size_t ws_bytes, uint32_t W, uint32_t n_lists, const bsort_list* lists) {
  const ManyLayout l = many_layout_bytes(ws_bytes, W, n_lists);
  char* b = static_cast<char*>(base);
  Many m{};
  m.hdr = reinterpret_cast<ManyHdr*>(b + l.header);
  m.ls = reinterpret_cast<ListState*>(b + l.lists);
  m.lists = lists;
  m.n_lists = n_lists;
  m.W = W;
  m.item_start = reinterpret_cast<uint32_t*>(b + l.item_start);
  m.seg_start = reinterpret_cast<uint32_t*>(b + l.segs);
  m.seg_cnt = reinterpret_cast<uint32_t*>(b + l.seg_cnt);
  m.tile_pre = reinterpret_cast<uint32_t*>(b + l.tile_pre);
  m.part_pre = reinterpret_cast<uint32_t*>(b + l.part_pre);
  m.seg_ord = reinterpret_cast<uint32_t*>(b + l.seg_ord);
  m.table = reinterpret_cast<uint32_t*>(b + l.table);
  m.trec = reinterpret_cast<uint8_t*>(b + l.trec);
  m.tlen = reinterpret_cast<uint8_t*>(b + l.tlen);
  m.ws.wait_polls = first_wait_polls();
  m.ws.hdr = reinterpret_cast<WsHeader*>(b + l.header + 256);
  m.ws.table = m.table;
  m.ws.autoa = nullptr;
  m.ws.keys[0] = reinterpret_cast<uint64_t*>(b + l.keys_a);
  m.ws.keys[1] = reinterpret_cast<uint64_t*>(b + l.keys_b);
  m.ws.idx[0] = reinterpret_cast<uint32_t*>(b + l.idx_a);
  m.ws.idx[1] = reinterpret_cast<uint32_t*>(b + l.idx_b);
  m.ws.cap = l.cap;
  m.ws.K = W / 8;
  m.cap = l.cap;
  return m;
}

__device__ __forceinline__ void list_error(const Many& m, uint32_t i, int code) {
  atomicOr(&m.ls[i].flags, 1u << code);
}

// Largest i in [0, n) with a[i] <= x (a ascending, a[0] <= x).
__device__ __forceinline__ uint32_t upper_index(const uint32_t* a, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (a[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}


__device__ __forceinline__ const uint8_t* len_of(const Many& m, const uint8_t* len, int text) {
  return text ? m.tlen : len;
}
__device__ __forceinline__ const uint8_t* rec_of(const Many& m, const uint8_t* rec, int text) {
  return text ? m.trec : rec;
}

// ---------------------------------------------------------------------------
__global__ void many_init_kernel(Many m, int text) {
  for (uint32_t i = threadIdx.x; i < m.n_lists; i += blockDim.x) {
    const bsort_list d = m.lists[i];
    uint32_t flags = 0, n = 0;
    if (d.word_off + d.max_words + 64 > m.cap) {
      flags |= 1u << BSORT_E_WORKSPACE;
    } else if (!text) {
      n = d.n_words;
      if (n > d.max_words) {
        flags |= 1u << BSORT_E_CAPACITY;
        n = d.max_words;
      }
    } else if (d.text_bytes > 0xFFFF0000ull) {
      flags |= 1u << BSORT_E_INVALID;
    }
    m.ls[i].n = n;
    m.ls[i].flags = flags;
  }
  if (threadIdx.x == 0) {
    m.hdr->items = m.hdr->tiles = m.hdr->active = 0;
    for (uint32_t p = 0; p < kMaxPasses; ++p) m.hdr->pass_parts[p] = 0;
    m.hdr->flags = 0;
    m.ws.hdr->status_flags = 0;
  }
}

// One CTA per list (grid-stride over lists): the list's text is scanned in
// 4096-byte chunks; words are numbered in order with a block scan per chunk.
__global__ void __launch_bounds__(kTokThreads)
many_tok_kernel(const uint8_t* __restrict__ text, Many m) {
  __shared__ uint32_t tmp[kTokWarps + 1];
  const uint32_t W = m.W, warp = threadIdx.x >> 5, lane = lane_id();
  for (uint32_t i = blockIdx.x; i < m.n_lists; i += gridDim.x) {
    const bsort_list d = m.lists[i];
    if (m.ls[i].flags & ((1u << BSORT_E_WORKSPACE) | (1u << BSORT_E_INVALID))) continue;
    const uint8_t* t = text + d.text_off;
    const uint32_t nb = static_cast<uint32_t>(d.text_bytes);
    uint32_t base = 0;
    bool too_long = false;
    for (uint32_t c = 0; c < nb; c += kChunkBytes) {
      const uint32_t p = c + warp * kWarpBytes;
      uint32_t starts[kSteps];
      const uint32_t cnt = warp_starts(t, 0u, nb, nb, p, starts);
      uint32_t total;
      uint32_t id = base + block_exclusive_scan(lane == 0 ? cnt : 0u, tmp, &total);
      id = __shfl_sync(0xffffffffu, id, 0);
#pragma unroll 1
      for (uint32_t st = 0; st < kSteps; ++st) {
        const uint32_t mk = starts[st];
        if ((mk >> lane) & 1u) {
          const uint32_t wid = id + __popc(mk & lanemask_lt());
          if (wid < d.max_words) {
            const uint64_t g = d.word_off + wid;
            const uint32_t L = write_word_record(t, nb, p + 32 * st + lane, W, m.trec + g * W);
            if (L > W) too_long = true;
            m.tlen[g] = static_cast<uint8_t>(L > 255 ? 255 : L);
          }
        }
        id += __popc(mk);
      }
      base += total;
    }
    if (too_long) list_error(m, i, BSORT_E_WORD_TOO_LONG);
    if (threadIdx.x == 0) {
      if (base > d.max_words) list_error(m, i, BSORT_E_CAPACITY);
      m.ls[i].n = min(base, d.max_words);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) many_plan_kernel(Many m, uint32_t max_list_words) {
  // a list longer than max_list_words would need more merge passes than
  // were launched: report it and keep its first max_list_words words
  for (uint32_t i = threadIdx.x; i < m.n_lists; i += blockDim.x) {
    if (m.ls[i].n > max_list_words) {
      list_error(m, i, BSORT_E_CAPACITY);
      m.ls[i].n = max_list_words;
    }
  }
  __syncthreads();
  const uint32_t tot = block_scan_into(
      m.n_lists, [&](uint32_t i) { return (m.ls[i].n + kItemWords - 1) / kItemWords; },
      m.item_start, m.item_start + m.n_lists);
  if (threadIdx.x == 0) m.hdr->items = tot;
}

__global__ void __launch_bounds__(kThreads)
many_hist_kernel(const uint8_t* __restrict__ len_in, int text, Many m) {
  __shared__ uint32_t cnt[kWarps][kBins];
  const uint8_t* len = len_of(m, len_in, text);
  const uint32_t W = m.W, warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t items = m.hdr->items;
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    for (uint32_t k = threadIdx.x; k < kWarps * kBins; k += kThreads) (&cnt[0][0])[k] = 0;
    __syncthreads();
    const uint32_t i = upper_index(m.item_start, m.n_lists + 1, it);
    const uint64_t off = m.lists[i].word_off;
    const uint32_t n = m.ls[i].n;
    const uint32_t j0 = (it - m.item_start[i]) * kItemWords, j1 = min(n, j0 + kItemWords);
    bool bad_zero = false, bad_long = false;
    // all of a thread's lengths of the item are loaded before any is counted,
    // so their loads are in flight together
    constexpr uint32_t kPer = kItemWords / kThreads;
    uint32_t Ls[kPer];
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint32_t j = j0 + k * kThreads + threadIdx.x;
      Ls[k] = j < j1 ? len[off + j] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      uint32_t L = Ls[k];
      if (L != 0xFFFFFFFFu) {
        bad_zero |= L == 0;
        bad_long |= L > W;
      }
      if (L > W) L = 0;
      const uint32_t peers = __match_any_sync(0xffffffffu, L);
      if (L != 0 && lane == __ffs(peers) - 1) cnt[warp][L] += __popc(peers);
    }
    __syncthreads();
    for (uint32_t L = threadIdx.x; L <= W; L += kThreads) {
      uint32_t s = 0;
#pragma unroll
      for (uint32_t w = 0; w < kWarps; ++w) s += cnt[w][L];
      m.table[static_cast<uint64_t>(it) * (W + 1) + L] = s;
    }
    if (bad_zero) list_error(m, i, BSORT_E_INVALID);
    if (bad_long) list_error(m, i, BSORT_E_WORD_TOO_LONG);
    __syncthreads();
  }
}

// Per list, one warp: L-major exclusive scan over (length, item) counts ->
// scatter bases (global positions), bucket offsets, segment table.  A list's
// items are scanned 32 at a time with shuffles, so no block barrier is needed.
__global__ void __launch_bounds__(kThreads)
many_lscan_kernel(Many m, uint32_t* __restrict__ out_off) {
  const uint32_t W = m.W, lane = lane_id();
  const uint32_t warps = gridDim.x * kWarps;
  for (uint32_t i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < m.n_lists; i += warps) {
    const uint32_t it0 = m.item_start[i], ni = m.item_start[i + 1] - it0;
    const uint64_t woff = m.lists[i].word_off;
    uint32_t carry = 0;
    for (uint32_t L = 0; L <= W; ++L) {
      const uint32_t first = carry;
      for (uint32_t c0 = 0; c0 < ni; c0 += 32) {
        const uint32_t c = c0 + lane;
        const uint64_t e = static_cast<uint64_t>(it0 + c) * (W + 1) + L;
        const uint32_t v = c < ni ? m.table[e] : 0u;
        const uint32_t inc = warp_inclusive_scan(v);
        if (c < ni) m.table[e] = static_cast<uint32_t>(woff) + carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) {
        if (out_off) out_off[static_cast<uint64_t>(i) * (W + 2) + L] = first;
        if (L >= 1) {
          const uint32_t sg = i * W + (L - 1);
          m.seg_start[sg] = static_cast<uint32_t>(woff) + first;
          m.seg_cnt[sg] = carry - first;
        }
      }
    }
    if (lane == 0 && out_off) out_off[static_cast<uint64_t>(i) * (W + 2) + W + 1] = carry;
  }
}

// Stable scatter of one item's words to their bucket positions with key packing.
template <int KW>
__global__ void __launch_bounds__(kThreads)
many_scatter_kernel(const uint8_t* __restrict__ rec_in, const uint8_t* __restrict__ len_in,
                    int text, Many m) {
  // KW = W / 8 key words at most per word (a template argument, so that a
  // thread holds only the words its record width can have)
  constexpr uint32_t kItems = 4;
  __shared__ uint32_t cursor[kBins];
  __shared__ uint32_t wcnt[kWarps][kBins];
  const uint8_t* len = len_of(m, len_in, text);
  const uint8_t* rec = rec_of(m, rec_in, text);
  const uint32_t W = m.W, warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t items = m.hdr->items;
  const Ws& ws = m.ws;
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    const uint32_t i = upper_index(m.item_start, m.n_lists + 1, it);
    const uint64_t off = m.lists[i].word_off;
    const uint32_t n = m.ls[i].n;
    const uint32_t j0 = (it - m.item_start[i]) * kItemWords, j1 = min(n, j0 + kItemWords);
    if (threadIdx.x <= W) cursor[threadIdx.x] = m.table[static_cast<uint64_t>(it) * (W + 1) + threadIdx.x];
    __syncthreads();
    for (uint32_t c = j0; c < j1; c += kThreads * kItems) {
      for (uint32_t k = lane; k < kBins; k += 32) wcnt[warp][k] = 0;
      __syncwarp();
      uint32_t Ls[kItems], rank[kItems];
      // lengths, then the record words of the chunk: all loads in flight
      // together, ahead of the ranking
      uint64_t words[kItems][KW];
#pragma unroll
      for (uint32_t u = 0; u < kItems; ++u) {
        const uint32_t j = c + warp * 32 * kItems + u * 32 + lane;
        uint32_t L = j < j1 ? len[off + j] : 0u;
        Ls[u] = L > W ? 0u : L;
      }
#pragma unroll
      for (uint32_t u = 0; u < kItems; ++u) {
        const uint32_t j = c + warp * 32 * kItems + u * 32 + lane;
        const uint64_t* src = reinterpret_cast<const uint64_t*>(rec + (off + j) * W);
        const uint32_t K = Ls[u] ? keys_for_len(Ls[u]) : 0u;
#pragma unroll
        for (uint32_t k = 0; k < KW; ++k) words[u][k] = k < K ? __ldg(src + k) : 0ull;
      }
#pragma unroll
      for (uint32_t u = 0; u < kItems; ++u) {
        const uint32_t L = Ls[u];
        const uint32_t peers = __match_any_sync(0xffffffffu, L);
        rank[u] = wcnt[warp][L] + __popc(peers & lanemask_lt());
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
      for (uint32_t u = 0; u < kItems; ++u) {
        const uint32_t L = Ls[u];
        if (L == 0) continue;
        const uint32_t j = c + warp * 32 * kItems + u * 32 + lane;
        const uint32_t pos = wcnt[warp][L] + rank[u];
        const uint32_t K = keys_for_len(L);
#pragma unroll
        for (uint32_t k = 0; k < KW; ++k)
          if (k < K) ws.keys[0][k * ws.cap + pos] = bswap64(words[u][k]) & key_mask(L, k);
        ws.idx[0][pos] = j;
      }
      __syncthreads();
    }
  }
}

// (list, length) buckets of at most kWarpSortMax words are sorted by one warp
// each (many_small_kernel); the tile kernel takes the larger ones.
constexpr uint32_t kWarpSortMax = 64;

__global__ void __launch_bounds__(1024) many_tplan_kernel(Many m) {
  const uint32_t S = m.n_lists * m.W, T = m.T;
  const uint32_t tot = block_scan_into(
      S,
      [&](uint32_t s) {
        const uint32_t c = m.seg_cnt[s];
        return c <= kWarpSortMax ? 0u : (c + T - 1) / T;
      },
      m.tile_pre, m.tile_pre + S);
  if (threadIdx.x == 0) m.hdr->tiles = tot;
}

// One warp sorts one small bucket in registers, two positions per lane
// (positions 2l and 2l + 1 in lane l), with no block barrier: by odd-even
// transposition (the even phase compares a lane's own pair, the odd phase
// its second position with the next lane's first; two quiet phases in a row
// end it) when the bucket has at most `cross` words, else by a bitonic
// network over shuffles.  Many warps of a CTA sort different buckets at once.
template <int K>
__device__ void warp_sort_small(Many& m, uint32_t start, uint32_t cnt, uint32_t cross) {
  const uint32_t lane = lane_id();
  Elem<K> r[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t p = 2 * lane + j;
    r[j] = p < cnt ? load_elem<K>(m.ws, 0, start + p) : elem_inf<K>();
  }
  if (cnt <= cross) {
    bool prev_quiet = false;
    for (uint32_t ph = 0; ph < cnt; ++ph) {
      bool swapped = false;
      if ((ph & 1u) == 0) {
        if (elem_less<K>(r[1], r[0])) {
          const Elem<K> x = r[0];
          r[0] = r[1];
          r[1] = x;
          swapped = true;
        }
      } else {
        // r[1] of lane l against r[0] of lane l + 1 (the last lane's r[1] has no partner)
        Elem<K> up, down;
        up.idx = __shfl_down_sync(0xffffffffu, r[0].idx, 1);
        down.idx = __shfl_up_sync(0xffffffffu, r[1].idx, 1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          up.k[k] = __shfl_down_sync(0xffffffffu, r[0].k[k], 1);
          down.k[k] = __shfl_up_sync(0xffffffffu, r[1].k[k], 1);
        }
        if (lane < 31 && elem_less<K>(up, r[1])) {
          r[1] = up;
          swapped = true;
        }
        if (lane > 0 && elem_less<K>(r[0], down)) r[0] = down;
      }
      const bool quiet = !__any_sync(0xffffffffu, swapped);
      if (quiet && prev_quiet) break;
      prev_quiet = quiet;
    }
  } else {
    SmemTile<K> none{};  // the network below never leaves the warp
    const ElemOps<K> ops{none};
    for (uint32_t k = 2; k <= 64; k <<= 1) {  // 64 positions: two per lane
      bitonic_step<ElemOps<K>, 2>(r, ops, k - 1);
      for (uint32_t j = k >> 2; j > 0; j >>= 1) bitonic_step<ElemOps<K>, 2>(r, ops, j);
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t p = 2 * lane + j;
    if (p < cnt) store_elem<K>(m.ws, 0, start + p, r[j]);
  }
}

__global__ void __launch_bounds__(256) many_small_kernel(Many m, uint32_t cross) {
  const uint32_t S = m.n_lists * m.W;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); s < S; s += warps) {
    const uint32_t cnt = m.seg_cnt[s];  // warp-uniform
    if (cnt < 2 || cnt > kWarpSortMax) continue;
    const uint32_t start = m.seg_start[s];
    switch (keys_for_len(s % m.W + 1)) {
      case 1: warp_sort_small<1>(m, start, cnt, cross); break;
      case 2: warp_sort_small<2>(m, start, cnt, cross); break;
      case 3: warp_sort_small<3>(m, start, cnt, cross); break;
      default: warp_sort_small<4>(m, start, cnt, cross); break;
    }
  }
}

// A (list, length) bucket of at most `cross` words is sorted whole by
// odd-even transposition; a larger one by bitonic tiles (merged afterwards).
__global__ void __launch_bounds__(1024) many_tile_kernel(Many m, uint32_t cross) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sm = align128(smem);
  const uint32_t S = m.n_lists * m.W, T = m.T;
  const uint32_t tiles = m.hdr->tiles;
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t s = upper_index(m.tile_pre, S + 1, t);
    TileRef tr;
    tr.L = s % m.W + 1;
    tr.start = m.seg_start[s] + (t - m.tile_pre[s]) * T;
    tr.len = min(T, m.seg_start[s] + m.seg_cnt[s] - tr.start);
    tr.valid = true;
    const bool odd_even = m.seg_cnt[s] <= cross;
    switch (keys_for_len(tr.L)) {
      case 1: sort_one_tile<1>(sm, T, tr, odd_even, m.ws); break;
      case 2: sort_one_tile<2>(sm, T, tr, odd_even, m.ws); break;
      case 3: sort_one_tile<3>(sm, T, tr, odd_even, m.ws); break;
      default: sort_one_tile<4>(sm, T, tr, odd_even, m.ws); break;
    }
    __syncthreads();
  }
}

// The partitions of every merge pass at once.  A segment of c > T words takes
// merge_passes(c, T) passes; ordering the segments by that count, most first
// (seg_ord), makes the segments still merging at pass p a prefix of the
// order, so one prefix sum of their partition counts (part_pre) serves every
// pass: pass p has pass_parts[p] partitions, the first ones of the order.
__global__ void __launch_bounds__(1024) many_pplan_kernel(Many m) {
  __shared__ uint32_t hist[kMaxPasses + 1], cursor[kMaxPasses + 1];
  const uint32_t S = m.n_lists * m.W, T = m.T, lane = lane_id();
  if (threadIdx.x <= kMaxPasses) hist[threadIdx.x] = 0;
  __syncthreads();
  const auto passes = [&](uint32_t s) { return s < S ? min(merge_passes(m.seg_cnt[s], T), kMaxPasses) : 0u; };
  for (uint32_t b = 0; b < S; b += blockDim.x) {
    const uint32_t c = passes(b + threadIdx.x);
    const uint32_t peers = __match_any_sync(0xffffffffu, c);
    if (c != 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[c], __popc(peers));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t c = kMaxPasses; c >= 1; --c) {
      cursor[c] = run;
      run += hist[c];
    }
    m.hdr->active = run;
  }
  __syncthreads();
  for (uint32_t b = 0; b < S; b += blockDim.x) {
    const uint32_t s = b + threadIdx.x, c = passes(s);
    const uint32_t peers = __match_any_sync(0xffffffffu, c);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (c != 0 && lane == leader) base = atomicAdd(&cursor[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (c != 0) m.seg_ord[base + __popc(peers & lanemask_lt())] = s;
  }
  __syncthreads();
  const uint32_t active = m.hdr->active;
  block_scan_into(
      active,
      [&](uint32_t j) {
        const uint32_t sg = m.seg_ord[j], P = merge_part_for(m.part, keys_for_len(sg % m.W + 1));
        return (m.seg_cnt[sg] + P - 1) / P;
      },
      m.part_pre, m.part_pre + active);
  __syncthreads();
  if (threadIdx.x < kMaxPasses) {
    // segments with more than p passes: the first sum(hist[c], c > p)
    uint32_t k = 0;
    for (uint32_t c = threadIdx.x + 1; c <= kMaxPasses; ++c) k += hist[c];
    m.hdr->pass_parts[threadIdx.x] = m.part_pre[k];
  }
}

// One merge pass over the partitions of every segment longer than R, in
// contiguous chunks per persistent CTA (merge_pass_ws: a producer warp finds
// the splits, short searches over runs of at most one list's segment, and
// stages the inputs by bulk copies; the consumer warps merge).
__global__ void __launch_bounds__(kMergeThreads) many_merge_kernel(Many m, uint32_t pass, uint32_t R, int src) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t active = m.hdr->active;
  const auto part_of = [&](uint32_t p, uint32_t* K, uint32_t* P, uint32_t* bstart, uint32_t* cnt, uint32_t* o0) {
    const uint32_t j = upper_index(m.part_pre, active + 1, p), s = m.seg_ord[j];
    *K = keys_for_len(s % m.W + 1);
    *P = merge_part_for(m.part, *K);
    *o0 = (p - m.part_pre[j]) * *P;
    *bstart = m.seg_start[s];
    *cnt = m.seg_cnt[s];
  };
  merge_pass_ws(align128(smem), m.part, m.hdr->pass_parts[pass], R, src, m.ws, nullptr, part_of);
}

template <int KW>
__global__ void __launch_bounds__(kThreads)
many_gather_kernel(Many m, const uint32_t* __restrict__ out_off, uint8_t* __restrict__ out_rec,
                   uint32_t* __restrict__ out_perm) {
  // KW = W / 8 (a template argument, so that a thread holds only the key
  // words its record width can have)
  __shared__ uint32_t s_off[kMaxW + 2], s_buf[kMaxW + 2];
  const uint32_t W = m.W, T = m.T;
  const uint32_t items = m.hdr->items;
  const Ws& ws = m.ws;
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    const uint32_t i = upper_index(m.item_start, m.n_lists + 1, it);
    const uint64_t off = m.lists[i].word_off;
    if (threadIdx.x < W + 2) s_off[threadIdx.x] = out_off[static_cast<uint64_t>(i) * (W + 2) + threadIdx.x];
    __syncthreads();
    // the buffer each length's sorted segment ends in
    if (threadIdx.x >= 1 && threadIdx.x <= W)
      s_buf[threadIdx.x] = merge_passes(s_off[threadIdx.x + 1] - s_off[threadIdx.x], T) & 1u;
    __syncthreads();
    const uint32_t n = s_off[W + 1];
    const uint32_t j0 = (it - m.item_start[i]) * kItemWords, j1 = min(n, j0 + kItemWords);
    // four positions per thread at a time: all their loads in flight before
    // the stores
    constexpr uint32_t kG = 4;
    for (uint32_t r0 = j0 + threadIdx.x; r0 < j1; r0 += kG * kThreads) {
      uint64_t w[kG][KW];
      uint32_t pm[kG], Ks[kG];
#pragma unroll
      for (uint32_t u = 0; u < kG; ++u) {
        const uint32_t r = r0 + u * kThreads;
        Ks[u] = 0;
        pm[u] = 0;
        if (r < j1) {
          uint32_t lo = 1, hi = W;  // the length L with s_off[L] <= r < s_off[L + 1]
          while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= r) lo = mid;
            else hi = mid - 1;
          }
          Ks[u] = keys_for_len(lo);
          const uint64_t g = off + r;
          const uint64_t* kb = s_buf[lo] ? ws.keys[1] : ws.keys[0];
          const uint32_t* ib = s_buf[lo] ? ws.idx[1] : ws.idx[0];
#pragma unroll
          for (uint32_t k = 0; k < KW; ++k) w[u][k] = k < Ks[u] ? __ldg(kb + k * ws.cap + g) : 0ull;
          pm[u] = __ldg(ib + g);
        }
      }
#pragma unroll
      for (uint32_t u = 0; u < kG; ++u) {
        const uint32_t r = r0 + u * kThreads;
        if (r >= j1) continue;
        const uint64_t g = off + r;
        uint64_t* dst = reinterpret_cast<uint64_t*>(out_rec + g * W);
#pragma unroll
        for (uint32_t k = 0; k < KW; ++k) dst[k] = k < Ks[u] ? bswap64(w[u][k]) : 0ull;
        out_perm[g] = pm[u];
      }
    }
    __syncthreads();
  }
}

// The gather with as many CTAs as fit the SMs (its register count falls with
// the record width).
template <int KW>
cudaError_t launch_gather(int sms, const Many& m, uint32_t* out_off, uint8_t* out_rec, uint32_t* out_perm,
                          cudaStream_t s) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, many_gather_kernel<KW>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const uint32_t g = static_cast<uint32_t>(sms) * (occ < 1 ? 1u : occ > 8 ? 8u : static_cast<uint32_t>(occ));
  BSORT_LAUNCH("many_gather", many_gather_kernel<KW>, g, kThreads, 0, s, m, out_off, out_rec, out_perm);
  return cudaGetLastError();
}

__global__ void many_finish_kernel(Many m, int32_t* __restrict__ status) {
  for (uint32_t i = threadIdx.x + blockIdx.x * blockDim.x; i < m.n_lists; i += blockDim.x * gridDim.x) {
    const uint32_t f = m.ls[i].flags | m.hdr->flags | m.ws.hdr->status_flags;
    int32_t c = 0;
    for (int k = 1; k < 32; ++k)
      if (f & (1u << k)) {
        c = k;
        break;
      }
    status[i] = c;
  }
}


}  // namespace

size_t many_workspace_size(uint64_t total_words, uint32_t n_lists, uint32_t W) {
  return many_layout_cap(align_up(total_words + 64, 64), W, n_lists).total;
}

uint64_t many_capacity(size_t ws_bytes, uint32_t W, uint32_t n_lists) {
  const uint64_t c = many_layout_bytes(ws_bytes, W, n_lists).cap;
  return c > 64 ? c - 64 : 0;
}

cudaError_t launch_many(const uint8_t* text_or_rec, const uint8_t* len, const bsort_list* lists,
                        uint32_t n_lists, uint32_t W, int text, uint32_t max_list_words,
                        const SortParams& p, uint32_t* out_off, uint8_t* out_rec,
                        uint32_t* out_perm, int32_t* list_status, void* d_ws, size_t ws_bytes,
                        cudaStream_t s) {
  const int sms = device_sm_count();
  Many m = many_view(d_ws, ws_bytes, W, n_lists, lists);
  m.T = p.tile;
  m.part = p.part;
  const uint32_t KW = W / 8;
  const size_t tsm = tile_smem_bytes(KW, p.tile);
  const size_t msm = merge_staged_smem_bytes(p.part) + 128;
  static SmemOptIn tile_set, merge_set;
  cudaError_t e = ensure_smem(many_tile_kernel, tsm, &tile_set);
  if (e == cudaSuccess) e = ensure_smem(many_merge_kernel, msm, &merge_set);
  if (e != cudaSuccess) return e;
  const uint32_t grid = static_cast<uint32_t>(sms) * 4;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, many_merge_kernel, kMergeThreads, msm);
  if (e != cudaSuccess) return e;
  // persistent merge CTAs: as many as fit the SMs
  const uint32_t mgrid = static_cast<uint32_t>(sms) * (occ < 1 ? 1u : occ > 8 ? 8u : static_cast<uint32_t>(occ));
  BSORT_LAUNCH("many_init", many_init_kernel, 1, 1024, 0, s, m, text);
  if (text) BSORT_LAUNCH("many_tokenize", many_tok_kernel, grid, kTokThreads, 0, s, text_or_rec, m);
  BSORT_LAUNCH("many_plan", many_plan_kernel, 1, 1024, 0, s, m, max_list_words);
  // the histogram is latency-bound at few registers: twice the CTAs per SM
  BSORT_LAUNCH("many_hist", many_hist_kernel, grid * 2, kThreads, 0, s, len, text, m);
  BSORT_LAUNCH("many_lscan", many_lscan_kernel, grid, kThreads, 0, s, m, out_off);
  // The tile and merge plans (one block each) need only the segment table, so
  // they run on the thread's helper stream while the scatter moves the words;
  // the sorts wait for both.
  SideStream* ss = side_stream();
  cudaStream_t t = s;
  cudaError_t e2;
  if (ss) {
    if ((e2 = cudaEventRecord(ss->fork, s)) != cudaSuccess) return e2;
    if ((e2 = cudaStreamWaitEvent(ss->side, ss->fork, 0)) != cudaSuccess) return e2;
    t = ss->side;
  }
  BSORT_LAUNCH("many_tplan", many_tplan_kernel, 1, 1024, 0, t, m);
  if (p.tile < max_list_words) BSORT_LAUNCH("many_pplan", many_pplan_kernel, 1, 1024, 0, t, m);
  if (ss && (e2 = cudaEventRecord(ss->join, ss->side)) != cudaSuccess) return e2;
  switch (KW) {
    case 1: BSORT_LAUNCH("many_scatter", many_scatter_kernel<1>, grid, kThreads, 0, s, text_or_rec, len, text, m); break;
    case 2: BSORT_LAUNCH("many_scatter", many_scatter_kernel<2>, grid, kThreads, 0, s, text_or_rec, len, text, m); break;
    case 3: BSORT_LAUNCH("many_scatter", many_scatter_kernel<3>, grid, kThreads, 0, s, text_or_rec, len, text, m); break;
    default: BSORT_LAUNCH("many_scatter", many_scatter_kernel<4>, grid, kThreads, 0, s, text_or_rec, len, text, m); break;
  }
  if (ss && (e2 = cudaStreamWaitEvent(s, ss->join, 0)) != cudaSuccess) return e2;
  BSORT_LAUNCH("many_small", many_small_kernel, grid, 256, 0, s, m, p.cross);
  BSORT_LAUNCH(p.alg == BSORT_ODD_EVEN ? "many_tile_odd_even" : "many_tile_bitonic", many_tile_kernel,
               grid, p.threads, tsm, s, m, p.cross);
  int src = 0;
  uint32_t pass = 0;
  for (uint64_t R = p.tile; R < max_list_words && pass < kMaxPasses; R <<= 1, ++pass) {
    BSORT_LAUNCH("many_merge", many_merge_kernel, mgrid, kMergeThreads, msm, s, m, pass, static_cast<uint32_t>(R),
                 src);
    src ^= 1;
  }
  switch (KW) {
    case 1: e = launch_gather<1>(sms, m, out_off, out_rec, out_perm, s); break;
    case 2: e = launch_gather<2>(sms, m, out_off, out_rec, out_perm, s); break;
    case 3: e = launch_gather<3>(sms, m, out_off, out_rec, out_perm, s); break;
    default: e = launch_gather<4>(sms, m, out_off, out_rec, out_perm, s); break;
  }
  if (e != cudaSuccess) return e;
  BSORT_LAUNCH("many_finish", many_finish_kernel, 16, 256, 0, s, m, list_status);
  return cudaGetLastError();
}

}  // namespace bsort
