// Phase 1 of the method (§3 Methodology, "Pre-processing", first phase):
// non-letter bytes are removed / ignored, i.e. act as word separators.
//
// Three launches over a fixed grid of at most kTextBlocksMax blocks, block b
// owning the contiguous byte range [b*per, (b+1)*per):
//   tok_count_kernel  word starts per block
//   scan_kernel       exclusive scan of the per-block counts -> first word id
//   tok_write_kernel  every word start writes its zero-padded record, length
//                     and source offset at its global id
// Each warp classifies 32 consecutive bytes per step, one byte per lane, and
// turns them into a 32-bit letter mask with __ballot_sync; a word starts where
// a letter follows a non-letter, so starts = mask & ~(mask << 1 | carry), the
// carry being the letter bit of the byte before.  A word that straddles a
// block boundary belongs to the block holding its first letter.
#include "block_scan.cuh"
#include "common.cuh"
#include "kernels.h"
#include "tok_impl.cuh"

namespace bsort {

namespace {

__global__ void __launch_bounds__(kTokThreads)
tok_count_kernel(const uint8_t* __restrict__ text, uint32_t n, uint32_t per,
                 uint32_t* __restrict__ blk_cnt) {
  __shared__ uint32_t tmp[kTokWarps + 1];
  const uint32_t b0 = blockIdx.x * per;
  const uint32_t b1 = min(n, b0 + per);
  const uint32_t warp = threadIdx.x >> 5;
  uint32_t cnt = 0;
  for (uint32_t c = b0; c < b1; c += kChunkBytes) {
    uint32_t starts[kSteps];
    cnt += warp_starts(text, 0u, n, b1, c + warp * kWarpBytes, starts);
  }
  uint32_t total;
  block_exclusive_scan(lane_id() == 0 ? cnt : 0u, tmp, &total);
  if (threadIdx.x == 0) blk_cnt[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kTokThreads)
tok_write_kernel(const uint8_t* __restrict__ text, uint32_t n, uint32_t per, uint32_t W,
                 uint32_t max_words, const uint32_t* __restrict__ blk_base,
                 uint8_t* __restrict__ rec, uint8_t* __restrict__ len,
                 uint32_t* __restrict__ src_off, WsHeader* hdr) {
  __shared__ uint32_t tmp[kTokWarps + 1];
  const uint32_t b0 = blockIdx.x * per;
  const uint32_t b1 = min(n, b0 + per);
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  uint32_t base = blk_base[blockIdx.x];
  bool too_long = false;
  for (uint32_t c = b0; c < b1; c += kChunkBytes) {
    const uint32_t p = c + warp * kWarpBytes;
    uint32_t starts[kSteps];
    const uint32_t cnt = warp_starts(text, 0u, n, b1, p, starts);
    uint32_t total;
    uint32_t id = base + block_exclusive_scan(lane == 0 ? cnt : 0u, tmp, &total);
    id = __shfl_sync(0xffffffffu, id, 0);
#pragma unroll 1
    for (uint32_t st = 0; st < kSteps; ++st) {
      const uint32_t m = starts[st];
      if ((m >> lane) & 1u) {
        const uint32_t wid = id + __popc(m & lanemask_lt());
        const uint32_t s = p + 32 * st + lane;
        // word length: letters from s, reading at most W + 1 bytes
        uint32_t L = 0;
        while (L <= W && s + L < n && is_letter(__ldg(text + s + L))) ++L;
        if (L > W) too_long = true;
        if (wid < max_words) {
          const uint32_t Lc = min(L, W);
          uint64_t* dst = reinterpret_cast<uint64_t*>(rec + static_cast<uint64_t>(wid) * W);
          for (uint32_t k = 0; k < W / 8; ++k) {
            uint64_t v = 0;
#pragma unroll
            for (uint32_t q = 0; q < 8; ++q) {
              const uint32_t o = 8 * k + q;
              if (o < Lc) v |= static_cast<uint64_t>(__ldg(text + s + o)) << (8 * q);
            }
            dst[k] = v;
          }
          len[wid] = static_cast<uint8_t>(L > 255 ? 255 : L);
          src_off[wid] = s;
        }
      }
      id += __popc(m);
    }
    base += total;
  }
  if (too_long) set_error(hdr, BSORT_E_WORD_TOO_LONG);
}

// Turns the word total into the device word count and the capacity error.
__global__ void tok_finish_kernel(const uint32_t* __restrict__ total, uint32_t max_words,
                                  uint32_t* __restrict__ d_n_words, WsHeader* hdr) {
  uint32_t t = *total;
  if (t > max_words) {
    set_error(hdr, BSORT_E_CAPACITY);
    t = max_words;
  }
  hdr->n_words = t;
  if (d_n_words) *d_n_words = t;
}

}  // namespace

cudaError_t launch_tokenize(const uint8_t* text, uint32_t n_bytes, uint32_t W, uint32_t max_words,
                            uint8_t* rec, uint8_t* len, uint32_t* src_off, uint32_t* d_n_words,
                            const Ws& ws, cudaStream_t s) {
  uint32_t G = n_bytes == 0 ? 1 : (n_bytes + kChunkBytes - 1) / kChunkBytes;
  if (G > kTextBlocksMax) G = kTextBlocksMax;
  uint32_t per = n_bytes == 0 ? kChunkBytes : (n_bytes + G - 1) / G;
  per = (per + kChunkBytes - 1) / kChunkBytes * kChunkBytes;
  G = n_bytes == 0 ? 1 : (n_bytes + per - 1) / per;
  uint32_t* cnt = ws.table;  // G counts, scanned in place
  uint32_t* total = ws.table + kTextBlocksMax;
  BSORT_LAUNCH("tok_count", tok_count_kernel, G, kTokThreads, 0, s, text, n_bytes, per, cnt);
  launch_scan(cnt, G, total, s);
  BSORT_LAUNCH("tok_finish", tok_finish_kernel, 1, 1, 0, s, total, max_words, d_n_words, ws.hdr);
  BSORT_LAUNCH("tok_write", tok_write_kernel, G, kTokThreads, 0, s, text, n_bytes, per, W,
               max_words, cnt, rec, len, src_off, ws.hdr);
  return cudaGetLastError();
}

}  // namespace bsort
