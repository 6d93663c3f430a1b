// Device building blocks of phase 3 (§3 Methodology, "Pre-processing", third
// phase; §2 bubble sort; §4-§5 merge of sorted chunks), shared by the single-list
// and the batched pipelines: tile sorts staged by the bulk-copy engine (odd-even
// transposition in shared memory; bitonic networks in registers, one-key words
// packed with their tile position into single 64-bit values), and merge-path
// merge passes (a producer warp finding or reading the splits and staging the
// inputs by bulk copies, consumer warps merging).
#pragma once

#include "common.cuh"

namespace bsort {

// Which tile of which bucket a CTA owns.
struct TileRef {
  uint32_t L, start, len;
  bool valid;
};

__device__ __forceinline__ uint32_t merge_passes(uint32_t cnt, uint32_t T) {
  uint32_t p = 0;
  for (uint64_t R = T; cnt > R; R <<= 1) ++p;
  return p;
}

template <int K>
__device__ void bitonic_tile(const SmemTile<K>& t, uint32_t len) {
  uint32_t Tp = 2;
  while (Tp < len) Tp <<= 1;
  Elem<K> inf;
#pragma unroll
  for (int j = 0; j < K; ++j) inf.k[j] = ~0ull;
  inf.idx = ~0u;
  for (uint32_t i = len + threadIdx.x; i < Tp; i += blockDim.x) t.put(i, inf);
  __syncthreads();
  for (uint32_t k = 2; k <= Tp; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t p = threadIdx.x; p < Tp / 2; p += blockDim.x) {
        const uint32_t lo = 2 * j * (p / j) + (p % j);
        const uint32_t hi = lo + j;
        const bool up = (lo & k) == 0;
        const Elem<K> a = t.get(lo), b = t.get(hi);
        if (elem_less(b, a) == up) {
          t.put(lo, b);
          t.put(hi, a);
        }
      }
      __syncthreads();
    }
  }
}

// Bitonic sort in the all-ascending form: for each block size k the first
// step compares element r of a k-block with its mirror k-1-r, the following
// steps compare i with i + j (j = k/4 .. 1).  Positions at or past n act as
// +infinity and are never touched, so no padding is written.  Works on shared
// or global memory (the tile only holds pointers); all threads of the CTA call.
template <int K>
__device__ void bitonic_flip(const SmemTile<K>& t, uint32_t n) {
  if (n < 2) return;
  uint32_t N = 2, lgN = 1;
  while (N < n) {
    N <<= 1;
    ++lgN;
  }
  const uint32_t half = N >> 1;
  for (uint32_t lk = 1; lk <= lgN; ++lk) {
    const uint32_t k = 1u << lk, lhk = lk - 1, hk = k >> 1;
    for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
      const uint32_t blk = p >> lhk, r = p & (hk - 1);
      const uint32_t lo = (blk << lk) + r, hi = (blk << lk) + (k - 1 - r);
      if (hi < n) {
        const Elem<K> a = t.get(lo), b = t.get(hi);
        if (elem_less(b, a)) {
          t.put(lo, b);
          t.put(hi, a);
        }
      }
    }
    __syncthreads();
    for (uint32_t lj = lhk; lj-- > 0;) {
      const uint32_t j = 1u << lj;
      for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
        const uint32_t lo = ((p >> lj) << (lj + 1)) + (p & (j - 1)), hi = lo + j;
        if (hi < n) {
          const Elem<K> a = t.get(lo), b = t.get(hi);
          if (elem_less(b, a)) {
            t.put(lo, b);
            t.put(hi, a);
          }
        }
      }
      __syncthreads();
    }
  }
}

// Odd-even transposition sort: phase ph compares pairs (2p + ph%2, 2p + ph%2 + 1)
// and exchanges those out of order; after an even and an odd phase in a row
// without exchange every neighbour pair is ordered.  At most len phases.
template <int K>
__device__ void odd_even_tile(const SmemTile<K>& t, uint32_t len) {
  bool prev_quiet = false;
  for (uint32_t ph = 0; ph < len; ++ph) {
    const uint32_t s = ph & 1u;
    int swapped = 0;
    for (uint32_t p = threadIdx.x; 2 * p + s + 1 < len; p += blockDim.x) {
      const uint32_t lo = 2 * p + s;
      const Elem<K> a = t.get(lo), b = t.get(lo + 1);
      if (elem_less(b, a)) {
        t.put(lo, b);
        t.put(lo + 1, a);
        swapped = 1;
      }
    }
    const bool quiet = __syncthreads_or(swapped) == 0;
    if (quiet && prev_quiet) break;
    prev_quiet = quiet;
  }
}

// ---------------------------------------------------------------------------
// Register bitonic network (tile sorts of the merge path, the sample sort's
// splitter chunks)
// ---------------------------------------------------------------------------
// Sorts N = E * blockDim.x positions held in registers, blocked layout:
// thread t holds positions t*E .. t*E+E-1 in r[].  All-ascending form: for
// each block size k the first step pairs i with i ^ (k-1), the next ones pair
// i with i ^ j (j = k/4 .. 1); the lower position keeps the smaller value.
// A partner in the same thread is compared in registers, one in the same warp
// through __shfl_xor_sync, one in another warp through shared memory, so only
// those steps need block barriers.

// Padded exchange position: one spare slot per 16 keeps the strided exchange
// accesses free of bank conflicts.
__host__ __device__ constexpr uint32_t pad16(uint32_t i) { return i + (i >> 4); }

template <int K>
__device__ __forceinline__ Elem<K> elem_inf() {
  Elem<K> e;
#pragma unroll
  for (int k = 0; k < K; ++k) e.k[k] = ~0ull;
  e.idx = ~0u;
  return e;
}

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

// Single 64-bit values (a packed key and tile position); exchange slots in
// one plane.
struct U64Ops {
  using T = uint64_t;
  uint64_t* x;
  __device__ static bool less(uint64_t a, uint64_t b) { return a < b; }
  __device__ static uint64_t shfl(uint64_t v, uint32_t m) { return __shfl_xor_sync(0xffffffffu, v, m); }
  __device__ static uint64_t inf() { return ~0ull; }
  __device__ void st(uint32_t i, uint64_t v) const { x[pad16(i)] = v; }
  __device__ uint64_t ld(uint32_t i) const { return x[pad16(i)]; }
};

template <typename Ops, int M, int E>
__device__ __forceinline__ void reg_step(typename Ops::T (&r)[E], const Ops& ops) {
  if constexpr (M < E) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      constexpr int m = M;
      const int q = j ^ m;
      if (q > j && ops.less(r[q], r[j])) {
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
  constexpr uint32_t LE = E == 1 ? 0 : E == 2 ? 1 : E == 4 ? 2 : E == 8 ? 3 : 4;
  const uint32_t tid = threadIdx.x;
  const uint32_t lane_mask = mask >> LE;
  if (mask < E) {
    // in registers: masks are the flips 1, 3, 7, 15 or the cleaners 1, 2, 4, 8
    switch (mask) {
      case 1: reg_step<Ops, 1, E>(r, ops); break;
      case 2: reg_step<Ops, 2, E>(r, ops); break;
      case 3: reg_step<Ops, 3, E>(r, ops); break;
      case 4: reg_step<Ops, 4, E>(r, ops); break;
      case 7: reg_step<Ops, 7, E>(r, ops); break;
      case 8: reg_step<Ops, 8, E>(r, ops); break;
      default: reg_step<Ops, 15, E>(r, ops); break;
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
        if (ops.less(other, r[j]) == keep_small) r[j] = other;
      }
    } else {
      // flip step (mask = k - 1): slot j pairs with the partner's slot E-1-j.
      // Slots j and E-1-j are exchanged together: sending slot E-1-j delivers
      // the partner's value for my slot j, sending slot j the one for E-1-j.
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        const T for_j = Ops::shfl(r[E - 1 - j], lane_mask);
        const T for_m = Ops::shfl(r[j], lane_mask);
        if (ops.less(for_j, r[j]) == keep_small) r[j] = for_j;
        if (ops.less(for_m, r[E - 1 - j]) == keep_small) r[E - 1 - j] = for_m;
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
      if (ops.less(other, r[j]) == (i < pi)) r[j] = other;
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

// One level of the network (block size 2^LK: the flip step, then the
// cleaners 2^(LK-2) .. 1) with every step's partner pattern known at compile
// time, so no step pays for choosing its exchange form.
template <typename Ops, int E, int LK>
__device__ __forceinline__ void bitonic_level(typename Ops::T (&r)[E], const Ops& ops) {
  bitonic_step<Ops, E>(r, ops, (1u << LK) - 1);
#pragma unroll
  for (int lj = LK - 2; lj >= 0; --lj) bitonic_step<Ops, E>(r, ops, 1u << lj);
}

// block_sort with the network's levels unrolled (a level chosen once per
// block size instead of once per step); c <= 4,096.
template <typename Ops, int E, typename Get, typename Sink>
__device__ void block_sort_unrolled(const Ops& ops, uint32_t c, Get get, Sink sink) {
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
  for (uint32_t lk = 1; (1u << lk) <= N; ++lk) {
    switch (lk) {
      case 1: bitonic_level<Ops, E, 1>(r, ops); break;
      case 2: bitonic_level<Ops, E, 2>(r, ops); break;
      case 3: bitonic_level<Ops, E, 3>(r, ops); break;
      case 4: bitonic_level<Ops, E, 4>(r, ops); break;
      case 5: bitonic_level<Ops, E, 5>(r, ops); break;
      case 6: bitonic_level<Ops, E, 6>(r, ops); break;
      case 7: bitonic_level<Ops, E, 7>(r, ops); break;
      case 8: bitonic_level<Ops, E, 8>(r, ops); break;
      case 9: bitonic_level<Ops, E, 9>(r, ops); break;
      case 10: bitonic_level<Ops, E, 10>(r, ops); break;
      case 11: bitonic_level<Ops, E, 11>(r, ops); break;
      default: bitonic_level<Ops, E, 12>(r, ops); break;
    }
  }
#pragma unroll
  for (int j = 0; j < E; ++j)
    if (tid * E + j < c) sink(tid * E + j, r[j]);
  __syncthreads();
}

// Exchange slots of the register network over T positions (padded by pad16).
__host__ __device__ constexpr uint32_t tile_xslots(uint32_t T) { return T + T / 16; }

// Words of at most kPackMaxLen bytes leave the low 16 bits of their one key
// word zero: the tile sort packs the tile position there (T <= 65,536).
// Letter-only words of up to 8 bytes do the same with 6-bit letter codes.
constexpr uint32_t kPackMaxLen = 6;

// A one-key word of L <= 8 bytes (big-endian in w) made only of ASCII
// letters?
__device__ __forceinline__ bool all_letters(uint64_t w, uint32_t L) {
  bool ok = true;
  for (uint32_t i = 0; i < L; ++i) {
    const uint32_t b = static_cast<uint32_t>(w >> (56 - 8 * i)) & 0xFFu;
    ok &= ((b | 0x20u) - 0x61u) < 26u;
  }
  return ok;
}

// Its letters as 6-bit codes in byte order (A..Z -> 0..25, a..z -> 26..51,
// the order of the bytes themselves), first letter highest, the codes ending
// at bit 16: equal-length letter words compare as their codes do, and the
// low 16 bits are free.
__device__ __forceinline__ uint64_t letter_code(uint64_t w, uint32_t L) {
  uint64_t v = 0;
  for (uint32_t i = 0; i < L; ++i) {
    const uint32_t b = static_cast<uint32_t>(w >> (56 - 8 * i)) & 0xFFu;
    v = (v << 6) | (b >= 0x61u ? b - 0x61u + 26u : b - 0x41u);
  }
  return v << (64 - 6 * L);
}

// Byte offset (from the planes' start) of the packed network's exchange
// plane: after a one-key tile's key and index planes.
__host__ __device__ constexpr size_t tile_packed_xoff(uint32_t T) {
  return ((static_cast<size_t>(T) + 2) * 8 + (static_cast<size_t>(T) + 4) * 4 + 15) / 16 * 16;
}

// Shared memory of a tile-sort CTA: [mbarrier 16 B][KW key planes of T+2][idx T+4],
// plus 128 bytes of slack to align the start.  The register network (one or
// two key words) reuses the same area for its exchange planes once the tile
// is in registers; the packed network of a one-key tile keeps the index plane
// and puts its one exchange plane after it.  The area is the largest of these.
__host__ __device__ inline size_t tile_smem_bytes(uint32_t KW, uint32_t T) {
  const size_t planes = static_cast<size_t>(KW) * (T + 2) * 8 + static_cast<size_t>(T + 4) * 4;
  const size_t xch = static_cast<size_t>(tile_xslots(T)) * (8 * (KW < 2 ? KW : 2) + 4);
  const size_t packed = tile_packed_xoff(T) + static_cast<size_t>(tile_xslots(T)) * 8;
  const size_t a = planes > xch ? planes : xch;
  return 128 + 16 + (a > packed ? a : packed);
}

__device__ __forceinline__ uint8_t* align128(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}

template <int K>
__device__ void sort_one_tile(uint8_t* smem, uint32_t T, const TileRef& tr, bool odd_even,
                              const Ws& ws) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  uint64_t* kplane = reinterpret_cast<uint64_t*>(smem + 16);
  uint32_t* iplane = reinterpret_cast<uint32_t*>(smem + 16 + static_cast<size_t>(K) * (T + 2) * 8);
  // 16-byte aligned source ranges covering [start, start + len)
  const uint32_t ks = tr.start & ~1u, is = tr.start & ~3u;
  const uint32_t kbytes = ((tr.start + tr.len - ks) * 8 + 15) & ~15u;
  const uint32_t ibytes = ((tr.start + tr.len - is) * 4 + 15) & ~15u;
  // a persistent caller reuses this shared memory: order its earlier generic
  // accesses before the bulk copy (async proxy) and start a fresh barrier
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, K * kbytes + ibytes);
#pragma unroll
    for (int j = 0; j < K; ++j)
      bulk_g2s(kplane + j * (T + 2), ws.keys[0] + j * ws.cap + ks, kbytes, bar);
    bulk_g2s(iplane, ws.idx[0] + is, ibytes, bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0, ws.wait_polls);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) {
      set_error(ws.hdr, BSORT_E_TIMEOUT);
      mbar_wait_bounded(bar, 0);  // let copies in flight land before the CTA exits
    }
    return;
  }
  // every thread has passed the wait: retire the barrier
  if (threadIdx.x == 0) mbar_inval(bar);
  SmemTile<K> t;
#pragma unroll
  for (int j = 0; j < K; ++j) t.k[j] = kplane + j * (T + 2) + (tr.start - ks);
  t.idx = iplane + (tr.start - is);
  const uint32_t E = T / blockDim.x;
  // one-key words sorted as single 64-bit values (see below): words of at
  // most kPackMaxLen bytes always, those of 7 or 8 bytes when every word of
  // the tile is letters only (block-uniform test)
  bool packed = false, coded = false;
  if (K == 1 && !odd_even && T % blockDim.x == 0 && (E == 2 || E == 4)) {
    if (tr.L <= kPackMaxLen) {
      packed = true;
    } else {
      bool ok = true;
      for (uint32_t i = threadIdx.x; i < tr.len; i += blockDim.x) ok &= all_letters(t.k[0][i], tr.L);
      coded = packed = __syncthreads_and(ok) != 0;
    }
  }
  if (odd_even) {
    odd_even_tile<K>(t, tr.len);
  } else if (packed) {
    // one 64-bit value per position: the key (or its 6-bit letter codes) with
    // the tile position in the zero low 16 bits: distinct values, ordered as
    // (key, position), and the position order is the index order inside a
    // bucket.  Key and index come back through the position from the
    // untouched key and index planes.
    const U64Ops ops{reinterpret_cast<uint64_t*>(smem + 16 + tile_packed_xoff(T))};
    const uint64_t* kp = t.k[0];
    const uint32_t* ip = t.idx;
    const uint32_t L = tr.L;
    auto get = [&](uint32_t i) { return (coded ? letter_code(kp[i], L) : kp[i]) | i; };
    auto sink = [&](uint32_t i, uint64_t v) {
      const uint64_t g = static_cast<uint64_t>(tr.start) + i;
      const uint32_t pos = static_cast<uint32_t>(v & 0xFFFFu);
      ws.keys[0][g] = kp[pos];
      ws.idx[0][g] = ip[pos];
    };
    if (E == 2) block_sort_unrolled<U64Ops, 2>(ops, tr.len, get, sink);
    else block_sort_unrolled<U64Ops, 4>(ops, tr.len, get, sink);
    return;
  } else if (K <= 2 && T % blockDim.x == 0 && (E == 2 || E == 4 || (E == 8 && K == 1))) {
    // bitonic network over registers, E positions per thread; only the
    // cross-warp steps go through shared memory (one barrier pair each),
    // through exchange planes laid over the tile (read into registers before
    // the first exchange), and the sorted positions go straight to the
    // workspace from registers
    uint8_t* xb = smem + 16;
    const uint32_t X = tile_xslots(T);
    SmemTile<K> xt;
#pragma unroll
    for (int j = 0; j < K; ++j) xt.k[j] = reinterpret_cast<uint64_t*>(xb) + j * X;
    xt.idx = reinterpret_cast<uint32_t*>(xb + static_cast<size_t>(K) * X * 8);
    const ElemOps<K> ops{xt};
    auto get = [&](uint32_t i) { return t.get(i); };
    auto sink = [&](uint32_t i, const Elem<K>& e) { store_elem<K>(ws, 0, tr.start + i, e); };
    if constexpr (K <= 2) {
      if (E == 2) block_sort<ElemOps<K>, 2>(ops, tr.len, get, sink);
      else if (E == 4) block_sort<ElemOps<K>, 4>(ops, tr.len, get, sink);
      else if constexpr (K == 1) block_sort<ElemOps<K>, 8>(ops, tr.len, get, sink);
    }
    return;  // block_sort ends with a barrier; the shared memory is free again
  } else {
    bitonic_tile<K>(t, tr.len);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < tr.len; i += blockDim.x)
    store_elem<K>(ws, 0, tr.start + i, t.get(i));
}

// ---------------------------------------------------------------------------
// Merge path
// ---------------------------------------------------------------------------

// Number of elements of A among the first `diag` outputs of merge(A, B).
template <int K, typename GetA, typename GetB>
__device__ uint32_t merge_path(GetA A, uint32_t na, GetB B, uint32_t nb, uint32_t diag) {
  uint32_t lo = diag > nb ? diag - nb : 0u;
  uint32_t hi = min(diag, na);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (elem_less<K>(A(mid), B(diag - 1 - mid)))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The same split found by one warp: each round the 32 lanes test 32 evenly
// spaced candidates of the remaining range at once (their loads are
// independent) and the ballot keeps the sub-range where the predicate turns,
// so a range of r candidates takes about log32(r) rounds of memory latency
// instead of log2(r).  The predicate "A[i] sorts after B[diag-1-i]" is false
// then true along i (a strict total order has no ties).  All lanes return the
// split; every lane of the warp must call.
template <int K, typename GetA, typename GetB>
__device__ uint32_t merge_path_warp(GetA A, uint32_t na, GetB B, uint32_t nb, uint32_t diag) {
  // the split is the first i in [lo, hi] whose predicate holds (i = hi holds
  // by definition)
  uint32_t lo = diag > nb ? diag - nb : 0u;
  uint32_t hi = min(diag, na);
  const uint32_t lane = threadIdx.x & 31u;
  while (lo < hi) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + lane * step;
    const bool holds = p >= hi || !elem_less<K>(A(p), B(diag - 1 - p));
    const uint32_t m = __ballot_sync(0xffffffffu, holds);
    if (m == 0) {  // every candidate fails: the split lies past the last one
      lo += 31 * step + 1;
      continue;
    }
    const uint32_t f = __ffs(m) - 1;  // candidate f holds, candidate f-1 fails
    hi = min(lo + f * step, hi);
    lo = f ? lo + (f - 1) * step + 1 : lo;
  }
  return lo;
}

// Elements per merge partition for elements of K key words when one-key
// partitions hold `part`: wider elements take smaller partitions, so that a
// merge CTA's shared memory (merge_staged_smem_bytes(part)) fits every K and is
// sized for the common one-key words rather than the widest (2 K + 1 words
// per element against 3: halved for two keys, quartered for three or four).
__host__ __device__ constexpr uint32_t merge_part_for(uint32_t part, uint32_t K) {
  return K <= 1 ? part : K == 2 ? part / 2 : part / 4;
}

// Merges output range [o0, min(o0 + part, cnt)) of one merge pass: runs of
// length R at src (planes of a bucket or segment, cnt elements) are merged in
// pairs into dst.  part must divide 2R.  smem holds 2 x part elements.
template <int K>
__device__ void merge_tile(uint8_t* smem, uint32_t part, const SmemTile<K>& src,
                           const SmemTile<K>& dst, uint32_t cnt, uint32_t R, uint32_t o0) {
  __shared__ uint32_t s_split[2];
  const uint32_t o1 = min(o0 + part, cnt);
  const uint32_t ps = o0 / (2 * R) * (2 * R);
  const uint32_t na = min(R, cnt - ps);
  const uint32_t nb = min(R, cnt - ps - na);
  const uint32_t a0 = ps, b0 = ps + na;
  auto gA = [&](uint32_t i) { return src.get(a0 + i); };
  auto gB = [&](uint32_t i) { return src.get(b0 + i); };
  if (threadIdx.x < 64) {  // warps 0 and 1 find the two splits, 32 candidates a round
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t d = (w == 0 ? o0 : o1) - ps;
    const uint32_t sp = merge_path_warp<K>(gA, na, gB, nb, d);
    if ((threadIdx.x & 31u) == 0) s_split[w] = sp;
  }
  __syncthreads();
  // Sorted runs give i0 <= i1 <= i0 + (o1 - o0).  After a device error (a tile
  // left unsorted) the splits may disagree; clamping i1 into that range keeps
  // every access below inside the two runs and the shared tiles (the output
  // is then undefined, as the error status says).
  const uint32_t i0 = s_split[0];
  const uint32_t e1 = o1 - ps, lo1 = e1 > nb ? e1 - nb : 0u;
  const uint32_t i1 = min(max(s_split[1], max(i0, lo1)), min(i0 + (o1 - o0), na));
  const uint32_t j0 = (o0 - ps) - i0, j1 = (o1 - ps) - i1;
  const uint32_t ca = i1 - i0, cb = j1 - j0, tot = ca + cb;
  // smem: input tile (A part then B part), output tile
  SmemTile<K> in, out;
  uint64_t* kp = reinterpret_cast<uint64_t*>(smem);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    in.k[j] = kp + j * part;
    out.k[j] = kp + (K + j) * part;
  }
  in.idx = reinterpret_cast<uint32_t*>(kp + 2 * K * part);
  out.idx = in.idx + part;
  for (uint32_t i = threadIdx.x; i < tot; i += blockDim.x)
    in.put(i, i < ca ? gA(i0 + i) : gB(j0 + i - ca));
  __syncthreads();
  const uint32_t per = (part + blockDim.x - 1) / blockDim.x;
  const uint32_t d0 = min(tot, threadIdx.x * per), d1 = min(tot, d0 + per);
  auto sA = [&](uint32_t i) { return in.get(i); };
  auto sB = [&](uint32_t i) { return in.get(ca + i); };
  uint32_t ia = merge_path<K>(sA, ca, sB, cb, d0);
  uint32_t ib = d0 - ia;
  for (uint32_t d = d0; d < d1; ++d) {
    bool takeA;
    if (ia >= ca) takeA = false;
    else if (ib >= cb) takeA = true;
    else takeA = elem_less<K>(in.get(ia), in.get(ca + ib));
    out.put(d, takeA ? in.get(ia++) : in.get(ca + ib++));
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < tot; i += blockDim.x) dst.put(o0 + i, out.get(i));
  __syncthreads();  // smem and s_split are reused by the caller's next tile
}

// Planes of buffer `buf` of the workspace starting at position `start`.
template <int K>
__device__ __forceinline__ SmemTile<K> ws_planes(const Ws& ws, int buf, uint64_t start) {
  SmemTile<K> t;
#pragma unroll
  for (int j = 0; j < K; ++j) t.k[j] = ws.keys[buf] + j * ws.cap + start;
  t.idx = ws.idx[buf] + start;
  return t;
}

// ---------------------------------------------------------------------------
// Merge pass: a producer warp, consumer warps, two staged input buffers
// ---------------------------------------------------------------------------
// A persistent CTA takes a contiguous chunk of one merge pass's partitions.
// Its last warp (the producer) finds each partition's split (merge path, 32
// candidates a round over global memory; consecutive partitions of a run
// pair share a boundary, so one search per partition), or reads it when a
// separate launch found them all at once (long runs, whose searches take
// more rounds than one warp can hide behind the merges), and stages the
// partition's two input ranges into one of two shared-memory buffers with
// bulk copies (TMA), one per key plane and index plane of each run.  The other
// warps (the consumers) merge a staged partition into a third buffer, release
// its input buffer and write the result out in coalesced stores, while the
// producer already searches and stages the next ones.
//
// Input buffer layout for elements of K key words and partitions of P
// elements: [full mbarrier 16 B][K key planes of P + 32 slots][index plane of
// P + 32 slots].  In each plane the first run's range starts at the plane's
// start and the second's at the next 16-byte boundary after it; a range is
// copied from the 16-byte boundary at or below its first element (up to 1 key
// or 3 indices of slack), so element i of a range sits at (shift + i).
struct MergeGeo {
  uint32_t K, P, ca, cb;
  uint64_t out0;              // first output position (bucket start + o0)
  uint32_t aA, aB, aAi, aBi;  // element shifts of the two ranges in the key / index planes
  uint32_t bB, bBi;           // byte offset of the second range in a key / index plane
};

// One input buffer (a multiple of 128 bytes): the layout above for the
// largest K x P product (one key word and `part` elements; wider elements
// take smaller partitions, merge_part_for).
__host__ __device__ constexpr size_t merge_buf_bytes(uint32_t part) {
  return (16 + static_cast<size_t>(part + 32) * 12 + 512 + 127) / 128 * 128;
}

// The output buffer: K key planes and an index plane of P elements.
__host__ __device__ constexpr size_t merge_out_bytes(uint32_t part) {
  return (static_cast<size_t>(part) * 12 + 127) / 128 * 128;
}

// Shared memory of a merge CTA (without the 128 bytes of alignment slack).
__host__ __device__ constexpr size_t merge_staged_smem_bytes(uint32_t part) {
  return 2 * merge_buf_bytes(part) + merge_out_bytes(part);
}

// On tables of at least kPresplitMinWords words, merge passes over runs of at
// least kPresplitMinRun find their splits in a separate launch (all
// partitions at once): those searches run over data in HBM and take more
// rounds than one producer warp hides behind the merges.  Shorter runs, and
// smaller tables (mostly in L2), search in the merge kernel.
constexpr uint64_t kPresplitMinRun = 4096;
constexpr uint64_t kPresplitMinWords = 1u << 20;

// Consumer threads of a merge CTA; the CTA has one more warp, the producer.
constexpr uint32_t kMergeConsumers = 256;
constexpr uint32_t kMergeThreads = kMergeConsumers + 32;

__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

// Barrier of the consumer warps only (named barrier 1).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kMergeConsumers) : "memory");
}

// AND of p over the consumer warps (named barrier 1).
__device__ __forceinline__ bool consumers_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.and.pred b, 1, %2, a;\n"
      " selp.u32 %0, 1, 0, b;\n}\n"
      : "=r"(r)
      : "r"(p ? 1u : 0u), "r"(kMergeConsumers)
      : "memory");
  return r != 0;
}

// Producer lane 0: the geometry of partition [o0, o0 + P) of a pass over runs
// of R of a bucket (cnt elements at bstart of buffer src) whose raw splits are
// s0 and s1, written to *gp; then the bytes to expect on buf's barrier and the
// partition's bulk copies into buf.
__device__ inline void merge_issue(uint8_t* buf, MergeGeo* gp, uint32_t K, uint32_t P, uint32_t bstart,
                                   uint32_t cnt, uint32_t o0, uint32_t R, int src, const Ws& ws, uint32_t s0,
                                   uint32_t s1) {
  MergeGeo g;
  g.K = K;
  g.P = P;
  const uint32_t o1 = min(o0 + P, cnt);
  const uint32_t ps = o0 / (2 * R) * (2 * R);
  const uint32_t na = min(R, cnt - ps), nb = min(R, cnt - ps - na);
  const uint32_t d0 = o0 - ps, d1 = o1 - ps;
  // Sorted runs give max(0, d0 - nb) <= i0 <= min(na, d0) and
  // max(i0, d1 - nb) <= i1 <= min(na, i0 + d1 - d0).  Clamping the splits into
  // those ranges keeps every copy inside the two runs and the buffer when a
  // device error left a run unsorted (the output is then undefined, as the
  // error status says).
  const uint32_t i0 = min(max(s0, d0 > nb ? d0 - nb : 0u), min(na, d0));
  const uint32_t i1 = min(max(s1, max(i0, d1 > nb ? d1 - nb : 0u)), min(na, i0 + (d1 - d0)));
  const uint32_t j0 = d0 - i0;
  g.ca = i1 - i0;
  g.cb = (d1 - d0) - g.ca;
  g.out0 = static_cast<uint64_t>(bstart) + o0;
  const uint64_t gA = static_cast<uint64_t>(bstart) + ps + i0, gB = static_cast<uint64_t>(bstart) + ps + na + j0;
  g.aA = static_cast<uint32_t>(gA & 1u);
  g.aB = static_cast<uint32_t>(gB & 1u);
  g.aAi = static_cast<uint32_t>(gA & 3u);
  g.aBi = static_cast<uint32_t>(gB & 3u);
  // plane capacities cover the rounding: (a + c) 8 rounded up stays within
  // (P + 32) 8 for both ranges together, and likewise for the indices; the
  // planes hold cap >= n + 64 elements, so no copy reads past one
  const uint32_t kbA = g.ca ? round16((g.aA + g.ca) * 8) : 0u, kbB = g.cb ? round16((g.aB + g.cb) * 8) : 0u;
  const uint32_t ibA = g.ca ? round16((g.aAi + g.ca) * 4) : 0u, ibB = g.cb ? round16((g.aBi + g.cb) * 4) : 0u;
  g.bB = kbA;
  g.bBi = ibA;
  *gp = g;  // published to the consumers by the barrier's release below
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf);
  const uint32_t ks = (P + 32) * 8;
  uint8_t* ib = buf + 16 + K * ks;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, K * (kbA + kbB) + ibA + ibB);
  for (uint32_t k = 0; k < K; ++k) {
    const uint64_t* plane = ws.keys[src] + static_cast<uint64_t>(k) * ws.cap;
    uint8_t* kb = buf + 16 + k * ks;
    if (kbA) bulk_g2s(kb, plane + (gA - g.aA), kbA, bar);
    if (kbB) bulk_g2s(kb + kbA, plane + (gB - g.aB), kbB, bar);
  }
  if (ibA) bulk_g2s(ib, ws.idx[src] + (gA - g.aAi), ibA, bar);
  if (ibB) bulk_g2s(ib + ibA, ws.idx[src] + (gB - g.aBi), ibB, bar);
}

// Producer warp: the split at output o of a bucket's pass (cnt elements at
// bstart of buffer src): how many of the first o - ps outputs of o's run pair
// come from its first run.  Every lane returns it.
template <int K>
__device__ uint32_t merge_split_at(uint32_t bstart, uint32_t cnt, uint32_t R, uint32_t o, int src, const Ws& ws) {
  const SmemTile<K> t = ws_planes<K>(ws, src, bstart);
  const uint32_t ps = o / (2 * R) * (2 * R);
  const uint32_t na = min(R, cnt - ps), nb = min(R, cnt - ps - na);
  auto gA = [&](uint32_t i) { return t.get(ps + i); };
  auto gB = [&](uint32_t i) { return t.get(ps + na + i); };
  return merge_path_warp<K>(gA, na, gB, nb, o - ps);
}

// One warp: the split at partition q's first output o0 into out (0 at a run
// pair's start), for merge_pass_ws's precomputed form.
template <int K>
__device__ void merge_split_warp(uint32_t bstart, uint32_t cnt, uint32_t R, uint32_t o0, int src, const Ws& ws,
                                 uint32_t* out) {
  const uint32_t ps = o0 / (2 * R) * (2 * R);
  const uint32_t s0 = o0 == ps ? 0u : merge_split_at<K>(bstart, cnt, R, o0, src, ws);
  if ((threadIdx.x & 31u) == 0) *out = s0;
}

__device__ __forceinline__ uint32_t merge_split_any(uint32_t K, uint32_t bstart, uint32_t cnt, uint32_t R, uint32_t o,
                                                    int src, const Ws& ws) {
  switch (K) {
    case 1: return merge_split_at<1>(bstart, cnt, R, o, src, ws);
    case 2: return merge_split_at<2>(bstart, cnt, R, o, src, ws);
    case 3: return merge_split_at<3>(bstart, cnt, R, o, src, ws);
    default: return merge_split_at<4>(bstart, cnt, R, o, src, ws);
  }
}

// Consumers: merge a staged partition into `out` (thread t produces outputs
// [t per, t per + per)), release the input buffer (rel), write the result to
// buffer src ^ 1 in coalesced stores.
template <int K>
__device__ void merge_staged(const uint8_t* buf, uint8_t* out, const MergeGeo& g, int src, const Ws& ws,
                             uint64_t* rel) {
  const uint32_t ks = (g.P + 32) * 8;
  const uint8_t* ibase = buf + 16 + K * ks;
  const auto A = [&](uint32_t i) {
    Elem<K> e;
#pragma unroll
    for (int k = 0; k < K; ++k) e.k[k] = reinterpret_cast<const uint64_t*>(buf + 16 + k * ks)[g.aA + i];
    e.idx = reinterpret_cast<const uint32_t*>(ibase)[g.aAi + i];
    return e;
  };
  const auto B = [&](uint32_t i) {
    Elem<K> e;
#pragma unroll
    for (int k = 0; k < K; ++k) e.k[k] = reinterpret_cast<const uint64_t*>(buf + 16 + k * ks + g.bB)[g.aB + i];
    e.idx = reinterpret_cast<const uint32_t*>(ibase + g.bBi)[g.aBi + i];
    return e;
  };
  SmemTile<K> o;
#pragma unroll
  for (int k = 0; k < K; ++k) o.k[k] = reinterpret_cast<uint64_t*>(out) + k * g.P;
  o.idx = reinterpret_cast<uint32_t*>(reinterpret_cast<uint64_t*>(out) + K * g.P);
  const uint32_t tot = g.ca + g.cb;
  const uint32_t per = (g.P + kMergeConsumers - 1) / kMergeConsumers;
  const uint32_t d0 = min(tot, threadIdx.x * per), d1 = min(tot, d0 + per);
  uint32_t ia = merge_path<K>(A, g.ca, B, g.cb, d0), ib = d0 - ia;
  // the two heads stay in registers; only the side taken is read again
  Elem<K> a = ia < g.ca ? A(ia) : elem_inf<K>(), b = ib < g.cb ? B(ib) : elem_inf<K>();
  for (uint32_t d = d0; d < d1; ++d) {
    const bool takeA = ib >= g.cb || (ia < g.ca && elem_less<K>(a, b));
    o.put(d, takeA ? a : b);
    if (takeA) {
      if (++ia < g.ca) a = A(ia);
    } else {
      if (++ib < g.cb) b = B(ib);
    }
  }
  consumers_sync();
  if (threadIdx.x == 0) mbar_arrive(rel);  // the input buffer is free for the producer
  for (uint32_t i = threadIdx.x; i < tot; i += kMergeConsumers) store_elem<K>(ws, src ^ 1, g.out0 + i, o.get(i));
}

// One merge pass over `total` partitions with kMergeThreads threads per CTA;
// part_of(q, &K, &P, &bstart, &cnt, &o0) describes partition q (partitions of
// one bucket numbered consecutively, in output order).  With `pre`, the
// splits were found beforehand (pre[q] at partition q's first output, by
// merge_split_warp, all partitions at once), else the producer searches.
// smem (128-byte aligned) holds merge_staged_smem_bytes(part).  A wait that
// gives up sets BSORT_E_TIMEOUT and makes the CTA stop once the copies in
// flight landed.
template <typename PartOf>
__device__ void merge_pass_ws(uint8_t* smem, uint32_t part, uint32_t total, uint32_t R, int src,
                              const Ws& ws, const uint32_t* pre, PartOf part_of) {
  __shared__ MergeGeo s_geo[2];
  __shared__ __align__(8) uint64_t s_empty[2];
  __shared__ volatile uint32_t s_abort;
  uint8_t* buf[2] = {smem, smem + merge_buf_bytes(part)};
  uint8_t* out = smem + 2 * merge_buf_bytes(part);
  if (threadIdx.x == 0) {
    mbar_init(reinterpret_cast<uint64_t*>(buf[0]), 1);
    mbar_init(reinterpret_cast<uint64_t*>(buf[1]), 1);
    mbar_init(&s_empty[0], 1);
    mbar_init(&s_empty[1], 1);
    s_abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  // this CTA's partitions: a contiguous chunk when the producer searches
  // (neighbours share a split), else q = blockIdx.x + k gridDim.x (CTAs working
  // on neighbouring partitions at the same time)
  const uint32_t q0 = static_cast<uint32_t>(static_cast<uint64_t>(total) * blockIdx.x / gridDim.x);
  const uint32_t q1 = static_cast<uint32_t>(static_cast<uint64_t>(total) * (blockIdx.x + 1) / gridDim.x);
  const uint32_t count = pre ? (blockIdx.x < total ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0u) : q1 - q0;
  const auto part_at = [&](uint32_t it) { return pre ? blockIdx.x + it * gridDim.x : q0 + it; };
  if (threadIdx.x >= kMergeConsumers) {
    // the producer warp
    const bool lead = (threadIdx.x & 31u) == 0;
    uint32_t carry = 0;  // split at the previous partition's end
    bool issued[2] = {false, false};
    uint32_t last_par[2] = {0u, 0u};  // parity of the last phase issued into each buffer
    for (uint32_t it = 0; it < count; ++it) {
      const uint32_t q = part_at(it);
      const int b = static_cast<int>(it & 1u);
      if (__any_sync(0xffffffffu, s_abort != 0)) break;
      if (it >= 2) {  // wait until the consumers released buffer b
        const uint32_t par = ((it >> 1) - 1) & 1u;
        bool ok = false;
        for (uint32_t poll = 0; poll < ws.wait_polls && !ok && !s_abort; ++poll) ok = mbar_try_wait(&s_empty[b], par);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lead) {
            set_error(ws.hdr, BSORT_E_TIMEOUT);
            s_abort = 1;
          }
          break;
        }
      }
      uint32_t K, P, bstart, cnt, o0;
      part_of(q, &K, &P, &bstart, &cnt, &o0);
      const uint32_t o1 = min(o0 + P, cnt), ps = o0 / (2 * R) * (2 * R);
      const uint32_t pair = min(2 * R, cnt - ps);
      uint32_t s0 = 0;
      if (o0 != ps) s0 = pre ? pre[q] : q == q0 ? merge_split_any(K, bstart, cnt, R, o0, src, ws) : carry;
      const uint32_t s1 = o1 - ps == pair ? min(R, cnt - ps)  // the pair's end: the whole first run
                          : pre           ? pre[q + 1]
                                          : merge_split_any(K, bstart, cnt, R, o1, src, ws);
      carry = s1;
      if (lead) merge_issue(buf[b], &s_geo[b], K, P, bstart, cnt, o0, R, src, ws, s0, s1);
      issued[b] = true;
      last_par[b] = (it >> 1) & 1u;
      __syncwarp();
    }
    if (lead && s_abort) {
      // let this CTA's copies in flight land before it exits
      for (int x = 0; x < 2; ++x)
        if (issued[x]) mbar_wait_bounded(reinterpret_cast<uint64_t*>(buf[x]), last_par[x]);
    }
    return;
  }
  // the consumer warps
  for (uint32_t it = 0; it < count; ++it) {
    const int b = static_cast<int>(it & 1u);
    const uint32_t par = (it >> 1) & 1u;
    bool ok = false;
    for (uint32_t poll = 0; poll < ws.wait_polls && !ok && !s_abort; ++poll)
      ok = mbar_try_wait(reinterpret_cast<uint64_t*>(buf[b]), par);
    if (!consumers_and(ok)) {
      if (threadIdx.x == 0) {
        set_error(ws.hdr, BSORT_E_TIMEOUT);
        s_abort = 1;
      }
      return;
    }
    const MergeGeo g = s_geo[b];
    switch (g.K) {
      case 1: merge_staged<1>(buf[b], out, g, src, ws, &s_empty[b]); break;
      case 2: merge_staged<2>(buf[b], out, g, src, ws, &s_empty[b]); break;
      case 3: merge_staged<3>(buf[b], out, g, src, ws, &s_empty[b]); break;
      default: merge_staged<4>(buf[b], out, g, src, ws, &s_empty[b]); break;
    }
    consumers_sync();  // the output buffer is free again
  }
}

}  // namespace bsort
