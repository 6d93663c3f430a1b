// Word-boundary detection shared by the single-text and the batched
// tokenisers (phase 1 of §3 Methodology, "Pre-processing": non-letter bytes
// separate words).  Each warp classifies 32 consecutive bytes per step, one
// byte per lane, into a letter mask with __ballot_sync; a word starts where a
// letter follows a non-letter: starts = mask & ~(mask << 1 | carry).
#pragma once

#include "common.cuh"

namespace bsort {

constexpr uint32_t kTokThreads = 256;
constexpr uint32_t kTokWarps = kTokThreads / 32;
constexpr uint32_t kSteps = 16;                       // 32-byte steps per warp per chunk
constexpr uint32_t kWarpBytes = 32 * kSteps;          // 512
constexpr uint32_t kChunkBytes = kTokWarps * kWarpBytes;  // 4096 per block iteration

__device__ __forceinline__ bool letter_at(const uint8_t* __restrict__ text, uint32_t end,
                                          uint32_t q) {
  return q < end && is_letter(__ldg(text + q));
}

// Word-start masks of the warp's kSteps x 32 bytes starting at p, inside a
// text that begins at byte `begin` (the byte before it is a separator) and
// ends at n; bytes at or past `end` count as separators.  Returns the number
// of starts.
__device__ __forceinline__ uint32_t warp_starts(const uint8_t* __restrict__ text, uint32_t begin,
                                                uint32_t n, uint32_t end, uint32_t p,
                                                uint32_t (&starts)[kSteps]) {
  const uint32_t lane = lane_id();
  uint32_t carry = (p > begin && p - 1 < n && is_letter(__ldg(text + p - 1))) ? 1u : 0u;
  uint32_t cnt = 0;
#pragma unroll
  for (uint32_t st = 0; st < kSteps; ++st) {
    const uint32_t letters = __ballot_sync(0xffffffffu, letter_at(text, end, p + 32 * st + lane));
    starts[st] = letters & ~((letters << 1) | carry);
    carry = letters >> 31;
    cnt += __popc(starts[st]);
  }
  return cnt;
}

// Writes the word starting at text[s] (letters up to `end`, at most W + 1 read)
// as a zero-padded W-byte record; returns its length (W + 1 if longer than W).
__device__ __forceinline__ uint32_t write_word_record(const uint8_t* __restrict__ text, uint32_t end,
                                                      uint32_t s, uint32_t W, uint8_t* __restrict__ dst_rec) {
  uint32_t L = 0;
  while (L <= W && s + L < end && is_letter(__ldg(text + s + L))) ++L;
  const uint32_t Lc = min(L, W);
  uint64_t* dst = reinterpret_cast<uint64_t*>(dst_rec);
  for (uint32_t k = 0; k < W / 8; ++k) {
    uint64_t v = 0;
#pragma unroll
    for (uint32_t q = 0; q < 8; ++q) {
      const uint32_t o = 8 * k + q;
      if (o < Lc) v |= static_cast<uint64_t>(__ldg(text + s + o)) << (8 * q);
    }
    dst[k] = v;
  }
  return L;
}

}  // namespace bsort
