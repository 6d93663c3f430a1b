// Host-side launchers of the bsort kernels (one translation unit each).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace bsort {

// Per-kernel event timing (profile.cu); no-ops unless bsort_profile_enable(1).
bool profiling();
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);

// Launches `kernel<<<grid, block, smem, s>>>(args...)` bracketed by profile events.
#define BSORT_LAUNCH(name, kernel, grid, block, smem, s, ...) \
  do {                                                        \
    ::bsort::prof_begin(name, s);                             \
    kernel<<<grid, block, smem, s>>>(__VA_ARGS__);            \
    ::bsort::prof_end(s);                                     \
  } while (0)

// The calling host thread's helper stream on the current device, with the
// two events that fork work onto it from a call's stream and join it back
// (created on first use, kept for the thread's life); null when they cannot
// be created, and the caller then runs everything on its own stream.
struct SideStream {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream* side_stream();

// Geometry of the histogram / scatter grid: block b owns words [b*wpb, (b+1)*wpb).
struct HistGeom {
  uint32_t wpb, G;
};
HistGeom hist_geom(uint32_t n_cap);

// In-place exclusive scan of data[0..n) on one block; *total receives the sum.
void launch_scan(uint32_t* data, uint32_t n, uint32_t* total, cudaStream_t s);

cudaError_t launch_tokenize(const uint8_t* text, uint32_t n_bytes, uint32_t W, uint32_t max_words,
                            uint8_t* rec, uint8_t* len, uint32_t* src_off, uint32_t* d_n_words,
                            const Ws& ws, cudaStream_t s);

// Phase 2: histogram, scan, stable scatter + key packing into keys/idx A.
// d_n (nullable) holds the word count on the device; n_cap bounds it.
cudaError_t launch_bucket(const uint8_t* rec, const uint8_t* len, uint32_t n_cap,
                          const uint32_t* d_n, uint32_t W, uint32_t* d_off, const Ws& ws,
                          cudaStream_t s);

// Phase 2 counts only: histogram, scan, bucket offsets (no scatter).
cudaError_t launch_hist(const uint8_t* len, uint32_t n_cap, const uint32_t* d_n, uint32_t W,
                        uint32_t* d_off, const Ws& ws, cudaStream_t s);

// Packed destination of a bucketed call's final write (§3.1): the words back
// to back in bytes[cap], offsets[n + 1].  A total above cap records
// BSORT_E_CAPACITY, writes no bytes (the offsets still are) and sets
// offsets[n] = 0.  The caller guarantees n W < 2^32.
struct PackOut {
  uint8_t* bytes;
  uint32_t* offsets;
  uint64_t cap;
};

// Sample-sort strategy (auto.cu): length totals and bucket offsets (d_off),
// then the sort; writes the final records and permutation, or with pk the
// packed words and the permutation (out_rec unused).  auto_applies() says
// whether the sizes and the workspace suit it.
bool auto_applies(uint32_t n_cap, const Ws& ws, uint32_t W);
cudaError_t launch_auto(const uint8_t* rec, const uint8_t* len, uint32_t n_cap,
                        const uint32_t* d_n, uint32_t W, uint32_t* d_off, const Ws& ws,
                        uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s,
                        const PackOut* pk = nullptr);

struct SortParams {
  int alg;             // bsort_alg (resolved: ODD_EVEN or MERGE)
  uint32_t tile;       // elements per tile
  uint32_t threads;    // threads per tile-sort CTA
  uint32_t part;       // elements per merge-path partition
  uint32_t cross;      // buckets of at most this many words take the odd-even tile
};

// Default odd-even / merge crossover of the MERGE path (words per bucket).
constexpr uint32_t kDefaultCross = 64;

// Resolves the algorithm and tuning knobs of a call on records of width W
// (tune may be null); returns false on an invalid knob.
bool resolve_params(bsort_alg alg, const bsort_tune* tune, uint32_t W, SortParams* p);

// Phase 3: tile sort of every bucket, then merge passes until each bucket is
// one run.  n_cap bounds the word count (sizes the grids).
cudaError_t launch_sort(uint32_t n_cap, uint32_t W, const SortParams& p, const uint32_t* d_off,
                        const Ws& ws, cudaStream_t s);

// Concatenation: sorted records (from the keys) and the permutation, or with
// pk the packed words and the permutation (out_rec unused).
cudaError_t launch_gather(uint32_t n_cap, const uint32_t* d_n, uint32_t W, const uint32_t* d_off,
                          const Ws& ws, uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s,
                          const PackOut* pk = nullptr);

// Unbucketed order (whole.cu): merges the length buckets of a bucketed answer
// in out_rec / out_perm (offsets d_off) into one run ordered by bytes, a
// proper prefix first, then input index.  Uses the workspace's key and index
// planes as scratch.
cudaError_t launch_whole(uint32_t n_cap, uint32_t W, const uint32_t* d_off, const Ws& ws,
                         uint8_t* out_rec, uint32_t* out_perm, cudaStream_t s);

// Packed output (pack.cu): the sorted records rec[n][W] back to back without
// padding, offsets[n + 1].  Lengths from the bucket offsets d_off (bucketed
// order) or, when d_off is null, len[perm[r]].  Needs n_cap <= pack_max_words()
// and n_cap W < 2^32; a total above cap records BSORT_E_CAPACITY.
uint32_t pack_max_words();
cudaError_t launch_pack(uint32_t n_cap, uint32_t W, const uint8_t* rec, const uint32_t* d_off,
                        const uint32_t* perm, const uint8_t* len, uint8_t* bytes, uint64_t cap,
                        uint32_t* offsets, const Ws& ws, cudaStream_t s);

// Batched sort (sort_many.cu).
size_t many_workspace_size(uint64_t total_words, uint32_t n_lists, uint32_t W);
uint64_t many_capacity(size_t ws_bytes, uint32_t W, uint32_t n_lists);
cudaError_t launch_many(const uint8_t* text_or_rec, const uint8_t* len, const bsort_list* lists,
                        uint32_t n_lists, uint32_t W, int text, uint32_t max_list_words,
                        const SortParams& p, uint32_t* out_off, uint8_t* out_rec,
                        uint32_t* out_perm, int32_t* list_status, void* d_ws, size_t ws_bytes,
                        cudaStream_t s);

cudaError_t launch_export(uint32_t n, uint32_t W, const uint32_t* d_off, const Ws& ws,
                          uint64_t* keys, uint32_t* idx, cudaStream_t s);

}  // namespace bsort
