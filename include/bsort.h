/*
 * bsort.h -- C ABI of the GB300 (sm_103a) length-bucketed word sort.
 *
 * The method (Alyasseri et al., arXiv 1411.5283, §3 Methodology,
 * "Pre-processing"): strip the special characters from a text (phase 1), put
 * the words into sub-arrays by character count with shorter lengths first
 * (phase 2; the abstract sizes each sub-array by the number of words of that
 * length), and sort every sub-array alphabetically (phase 3) with bubble sort
 * (§2, §3.2) or merge sort (§4 "MPI Implementation", §5: chunks sorted
 * separately, then merged).  The result is every word ordered by
 * (length, bytes), equal words in input order.
 *
 * Conventions shared by every call
 *  - All pointers named d_* are device pointers owned by the caller.  The
 *    library allocates nothing on these paths; scratch lives in a caller-owned
 *    workspace of bsort_workspace_size() bytes (256-byte aligned).  Prepare a
 *    new workspace once with bsort_workspace_init().  Where things live inside
 *    the workspace depends only on (ws_bytes, W), so pass the same ws_bytes
 *    and W to every call that shares a workspace.
 *  - Record arrays (d_rec, d_out_rec) must be 16-byte aligned.
 *  - All calls are asynchronous on stream s and return synchronously only
 *    argument errors (BSORT_E_INVALID, BSORT_E_WORKSPACE, BSORT_E_CAPACITY
 *    for host-visible sizes) or a launch failure (BSORT_E_CUDA).  The AUTO
 *    algorithm runs its splitter selection on a helper stream that the
 *    library keeps per host thread and device, forked from s and joined back
 *    into s by events within the call, so the call stays ordered with the
 *    rest of s.
 *  - Errors found by the kernels (a word longer than W, more words than the
 *    capacity, a zero length) are recorded in a sticky status word inside the
 *    workspace; read it with bsort_get_status(), clear it with
 *    bsort_reset_status().  When several errors occur, the smallest code is
 *    reported.  Kernels never trap; after an error the outputs are undefined
 *    but every access stays inside the buffers described here.
 *  - W is the record width in bytes: 8, 16, 24 or 32.  A word is at most W
 *    letters.  Word lengths L run 1..W.
 *  - Records are W bytes, the word's letters first, zero padded.  Bytes after
 *    the word's length are ignored on input and written as zero on output.
 *  - Indices are uint32: at most 2^32 - 2 words per call.
 *  - Buckets: off[] has W + 2 entries; off[L] is the number of words shorter
 *    than L (off[0] = off[1] = 0, off[W+1] = n).  Bucket L occupies output
 *    ranks off[L] .. off[L+1]-1.
 */
#ifndef BSORT_H_
#define BSORT_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSORT_OK = 0,
  BSORT_E_INVALID = 1,        /* bad argument, or a record of length 0       */
  BSORT_E_WORD_TOO_LONG = 2,  /* a word has more than W letters              */
  BSORT_E_CAPACITY = 3,       /* more words than max_words / list capacity   */
  BSORT_E_WORKSPACE = 4,      /* workspace missing, misaligned or too small  */
  BSORT_E_CUDA = 5,           /* a CUDA launch or copy failed                */
  BSORT_E_TIMEOUT = 6,        /* a bounded device-side wait gave up          */
  BSORT_E_NOMEM = 7           /* serving admission: not enough device memory */
} bsort_status;

/* Per-bucket sort algorithm (third phase of §3 "Pre-processing").
 *  BSORT_ODD_EVEN: odd-even transposition sort of shared-memory tiles (the
 *    data-parallel form of the paper's bubble sort, §2), then merge-path
 *    merging of the sorted tiles (the paper's merge of sorted chunks, §4).
 *  BSORT_MERGE:    bitonic-network sort of shared-memory tiles, then
 *    merge-path merging.
 *  BSORT_AUTO:     the fastest available strategy for the sizes at hand.
 * Every algorithm gives byte-identical output. */
typedef enum { BSORT_ODD_EVEN = 0, BSORT_MERGE = 1, BSORT_AUTO = 2 } bsort_alg;

/* Tuning knobs; a field of 0 takes the library default.  Results never
 * depend on them.
 *  tile               elements per bitonic tile (power of two, 256..4096)
 *  oddeven_max        elements per odd-even tile (power of two, 64..2048)
 *  threads_per_bucket threads per tile-sort CTA (a multiple of 32, 64..1024;
 *                     default 256 for odd-even tiles, tile / 4 for bitonic
 *                     tiles, which then hold 2, 4 or (one key word) 8
 *                     positions per thread in registers)
 *  merge_fanin        elements per merge-path partition of one-key words (power
 *                     of two, 256..4096, default 2048); two-key words take
 *                     half as many, three- and four-key words a quarter
 *  oddeven_cross      BSORT_MERGE (and AUTO where it takes the merge path):
 *                     the crossover between the paper's two sorts.  A length
 *                     bucket of at most this many words (1..tile) is sorted
 *                     whole by odd-even transposition in one shared-memory
 *                     tile (bubble sort's data-parallel form, §2); a larger
 *                     one by bitonic tiles and merge-path merges (§4-§5).
 *                     1 = never odd-even (a one-word bucket is sorted);
 *                     0 = the library default (64). */
typedef struct {
  uint32_t tile, oddeven_max, threads_per_bucket, merge_fanin, oddeven_cross;
} bsort_tune;

/* One list of a batched call (bsort_sort_many).
 *  text_off, text_bytes  byte range of the list's text (text mode only)
 *  word_off              first record of the list in the concatenated word
 *                        arrays (input records in record mode; output records,
 *                        output permutation in both modes)
 *  n_words               number of words (record mode; ignored in text mode)
 *  max_words             capacity of the list's output slots (text mode: the
 *                        most words the text may hold; record mode: >= n_words) */
typedef struct {
  uint64_t text_off, text_bytes;
  uint64_t word_off;
  uint32_t n_words, max_words;
} bsort_list;

/* Bytes of workspace for up to max_words words of width W with algorithm alg
 * (every call below that takes d_ws needs this many bytes; 0 if the arguments
 * are invalid). */
size_t bsort_workspace_size(uint64_t max_words, uint32_t W, bsort_alg alg);

/* Number of words a workspace of ws_bytes bytes holds for width W (the
 * inverse of bsort_workspace_size; 0 if W is invalid). */
uint64_t bsort_workspace_capacity(size_t ws_bytes, uint32_t W);

/* Zeroes the workspace header (status word and counters).  Call once on a new
 * workspace before first use. */
bsort_status bsort_workspace_init(void* d_ws, size_t ws_bytes, cudaStream_t s);

/* Phase 1 (§3 "Pre-processing", first phase): splits text into words.
 * A letter is an ASCII byte 'A'..'Z' or 'a'..'z'; every other byte separates
 * words (so "don't" is "don", "t").  Words are numbered in order of
 * appearance.  Writes, for word i < max_words: d_rec[i*W .. i*W+W-1] (zero
 * padded), d_len[i] and d_src_off[i] (offset of its first byte in the text).
 * *d_n_words receives min(words found, max_words).  n_bytes must be below
 * 2^32.  Device errors: BSORT_E_WORD_TOO_LONG, BSORT_E_CAPACITY.
 * Workspace: bsort_workspace_size(max_words, W, alg) for any alg. */
bsort_status bsort_tokenize(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                            uint32_t max_words, uint8_t* d_rec, uint8_t* d_len,
                            uint32_t* d_src_off, uint32_t* d_n_words, void* d_ws,
                            size_t ws_bytes, cudaStream_t s);

/* Phase 2 (§3 "Pre-processing", second phase; abstract): groups the n words
 * d_rec[n*W], d_len[n] into buckets by length, shorter first, each bucket in
 * input order (a stable scatter), and packs each word into ceil(L/8)
 * big-endian uint64 keys inside the workspace, so that comparing keys as
 * integers compares the words byte by byte.  Writes d_off[W+2].
 * Device errors: BSORT_E_INVALID (a length of 0), BSORT_E_WORD_TOO_LONG
 * (a length above W); such words are left out of every bucket. */
bsort_status bsort_bucket_by_length(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                    uint32_t W, uint32_t* d_off, void* d_ws, size_t ws_bytes,
                                    cudaStream_t s);

/* Phase 3 (§3 "Pre-processing", third phase; §2; §4-§5): sorts every bucket
 * left in the workspace by bsort_bucket_by_length, by the words' bytes and
 * then by input index, with algorithm alg (tune may be NULL).  n, W and d_off
 * must be those given to / written by bsort_bucket_by_length. */
bsort_status bsort_sort_buckets(uint32_t n, uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                const uint32_t* d_off, void* d_ws, size_t ws_bytes,
                                cudaStream_t s);

/* Concatenation in ascending length (§3, second phase "shorter before
 * longer"): writes the sorted words d_out_rec[n*W] (zero padded, rebuilt from
 * the packed keys) and d_out_perm[n] (input index of each output word). */
bsort_status bsort_gather(uint32_t n, uint32_t W, const uint32_t* d_off, const void* d_ws,
                          size_t ws_bytes, uint8_t* d_out_rec, uint32_t* d_out_perm,
                          cudaStream_t s);

/* Phases 2-3 and the concatenation in one call on a word table (the same
 * result as bucket_by_length + sort_buckets + gather).  Resets the status
 * word first. */
bsort_status bsort_sort_records(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                uint8_t* d_out_rec, uint32_t* d_out_perm, uint32_t* d_off,
                                void* d_ws, size_t ws_bytes, cudaStream_t s);

/* Phases 1-3 and the concatenation in one call on raw text.  The word count
 * stays on the device (*d_n_words); nothing is copied to the host.  Resets
 * the status word first.  d_out_perm[r] is the input index (order of
 * appearance) of output word r; d_src_off[i] the text offset of word i. */
bsort_status bsort_sort_text(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                             uint32_t max_words, bsort_alg alg, const bsort_tune* tune,
                             uint8_t* d_rec, uint8_t* d_len, uint32_t* d_src_off,
                             uint32_t* d_n_words, uint8_t* d_out_rec, uint32_t* d_out_perm,
                             uint32_t* d_off, void* d_ws, size_t ws_bytes, cudaStream_t s);

/* The paper's unbucketed variant (Table 2, second row: the whole file sorted
 * alphabetically by bubble sort, without the length sub-arrays), on a word
 * table: every word ordered by its bytes as an unsigned byte string, a proper
 * prefix before the longer word ("a" < "a\0" < "ab"), equal words in input
 * order.  d_out_rec[n*W] receives the sorted records (zero padded) and
 * d_out_perm[n] the input index of each output word.  alg picks the sort of
 * the length buckets the call goes through first (the order inside a bucket
 * is the same in both variants); the sorted buckets are then merged in
 * ceil(log2 W) stable merge levels, equal records taking the shorter length
 * first.  The bucket offsets stay inside the workspace.  Same workspace,
 * alignment and device errors as bsort_sort_records; resets the status word
 * first. */
bsort_status bsort_sort_records_whole(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                      uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                      uint8_t* d_out_rec, uint32_t* d_out_perm, void* d_ws,
                                      size_t ws_bytes, cudaStream_t s);

/* The unbucketed variant on raw text (phase 1 of §3, then the order of
 * bsort_sort_records_whole); arguments as bsort_sort_text without d_off. */
bsort_status bsort_sort_text_whole(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                                   uint32_t max_words, bsort_alg alg, const bsort_tune* tune,
                                   uint8_t* d_rec, uint8_t* d_len, uint32_t* d_src_off,
                                   uint32_t* d_n_words, uint8_t* d_out_rec, uint32_t* d_out_perm,
                                   void* d_ws, size_t ws_bytes, cudaStream_t s);

/* The paper's other data structure for the words (§3.1, "vectors of
 * string", against the fixed-width 3-D char array of the abstract): the n
 * sorted words of d_rec[n*W] (records in output order, as written by the
 * calls above) packed back to back without padding into d_bytes, word r at
 * d_bytes[d_offsets[r] .. d_offsets[r+1]-1], d_offsets[n] = total bytes.
 * Word r's length: with d_off (the W + 2 bucket offsets of a bucketed call)
 * the L with off[L] <= r < off[L+1], and n is then min(n, off[W+1]), so the
 * device-side word count of the text path applies; with d_off NULL it is
 * d_len[d_perm[r]] (input lengths through the permutation; any order, e.g.
 * the unbucketed one).  bytes_cap is the capacity of d_bytes: a larger total
 * records BSORT_E_CAPACITY in the workspace status, writes no bytes and sets
 * d_offsets[n] = 0.  n must be at most 2^28 words and n W below
 * 2^32 (else BSORT_E_CAPACITY).  The workspace (any size valid for W) holds
 * per-tile sums. */
bsort_status bsort_pack_words(uint32_t n, uint32_t W, const uint8_t* d_rec, const uint32_t* d_off,
                              const uint32_t* d_perm, const uint8_t* d_len, uint8_t* d_bytes,
                              uint64_t bytes_cap, uint32_t* d_offsets, void* d_ws,
                              size_t ws_bytes, cudaStream_t s);

/* bsort_sort_records with the answer in the "vectors of string" form of §3.1
 * instead of records: the sort's last kernel writes the sorted words (in the
 * bucketed order of the other calls) back to back without padding into
 * d_bytes, word r at d_bytes[d_offsets[r] .. d_offsets[r+1]-1], d_offsets[n] =
 * total bytes, and the permutation to d_out_perm[n] and the bucket offsets to
 * d_off as bsort_sort_records does; no fixed-width records are written.
 * Same bytes and offsets as bsort_sort_records followed by bsort_pack_words
 * with d_off.  bytes_cap is the capacity of d_bytes: a larger total records
 * BSORT_E_CAPACITY in the workspace status, writes no bytes and sets
 * d_offsets[n] = 0 (the other outputs are still written).  n must be at most
 * 2^28 words and n W below 2^32 (else BSORT_E_CAPACITY before any work).
 * d_bytes has no alignment requirement; d_rec as bsort_sort_records. */
bsort_status bsort_sort_records_packed(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                       uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                       uint8_t* d_bytes, uint64_t bytes_cap, uint32_t* d_offsets,
                                       uint32_t* d_out_perm, uint32_t* d_off, void* d_ws,
                                       size_t ws_bytes, cudaStream_t s);

/* bsort_sort_text with the packed answer of bsort_sort_records_packed
 * (phases 1-3 of §3, output as in §3.1): n = the device-side word count
 * *d_n_words, d_offsets[n] = total bytes; max_words bounds n for the 2^28 and
 * 2^32 limits.  The tokenised records still go to d_rec / d_len / d_src_off. */
bsort_status bsort_sort_text_packed(const uint8_t* d_text, uint64_t n_bytes, uint32_t W,
                                    uint32_t max_words, bsort_alg alg, const bsort_tune* tune,
                                    uint8_t* d_rec, uint8_t* d_len, uint32_t* d_src_off,
                                    uint32_t* d_n_words, uint8_t* d_bytes, uint64_t bytes_cap,
                                    uint32_t* d_offsets, uint32_t* d_out_perm, uint32_t* d_off,
                                    void* d_ws, size_t ws_bytes, cudaStream_t s);

/* The paper has no counterpart to this entry point.
 * bsort_sort_records without a workspace, for callers that may not allocate
 * device memory: code whose device memory belongs to a host framework's own
 * pool (plugins of inference servers or game engines that forbid raw
 * cudaMalloc), or latency-bound loops that cannot afford cudaMalloc / cudaFree
 * and the device synchronisation they may cause.  Same result as
 * bsort_sort_records for the same arguments.
 *  - Scratch is a static device array inside the library, sized for at most
 *    32,768 words (any W); every GPU that loads the library holds it (about
 *    3 MB) until the process exits.  n above 32,768 returns BSORT_E_CAPACITY
 *    before any work is queued.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call
 *    (with the optional profiler off, its default).
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  The address is kept with the id of the context it was
 *    taken in; after cudaDeviceReset the next call looks it up again.
 *  - Every call shares the array and finds the previous call's contents; the
 *    call clears what must start at zero.  Calls that overlap on the GPU (other
 *    streams or host threads) race on the array: serialise them.
 *  - d_status (device, may be NULL) receives the smallest device-detected
 *    error code (a bsort_status) once the call's work on s has run. */
bsort_status bsort_sort_records_noalloc(const uint8_t* d_rec, const uint8_t* d_len, uint32_t n,
                                        uint32_t W, bsort_alg alg, const bsort_tune* tune,
                                        uint8_t* d_out_rec, uint32_t* d_out_perm,
                                        uint32_t* d_off, int32_t* d_status, cudaStream_t s);

/* Batched form (not in the paper; its §4 MPI chunking sorts one text): sorts
 * n_lists independent lists with persistent kernels on stream s (two planning
 * kernels on the thread's helper stream, forked from s and joined back) that
 * can be captured in one CUDA graph (phases 1-3 of §3 for every list at once).
 * d_lists[n_lists] (device) describes each list.  Record mode
 * (lists_are_text = 0): d_text_or_rec / d_len hold all lists' records.  Text
 * mode: d_text_or_rec holds the texts, d_len must be NULL, and the tokenised
 * words go to the output slots only.  For list i the outputs are
 * d_out_rec[(word_off + r) * W], d_out_perm[word_off + r] (index within the
 * list), d_out_off[i * (W + 2) + L], and d_list_status[i] (a bsort_status).
 * max_list_words bounds every list's word count (it sets the number of merge
 * passes); a longer list gets BSORT_E_CAPACITY.  Every list's slots
 * word_off .. word_off + max_words - 1 must lie below the word capacity the
 * workspace was sized for (bsort_sort_many_workspace_size(total_words,
 * n_lists, W); a list outside it gets BSORT_E_WORKSPACE).  alg BSORT_AUTO
 * means BSORT_MERGE here.  Per-list statuses are written to d_list_status;
 * the call itself returns only argument and launch errors. */
size_t bsort_sort_many_workspace_size(uint64_t total_words, uint32_t n_lists, uint32_t W);
bsort_status bsort_sort_many(const uint8_t* d_text_or_rec, const uint8_t* d_len,
                             const bsort_list* d_lists, uint32_t n_lists, uint32_t W,
                             int lists_are_text, uint32_t max_list_words, bsort_alg alg,
                             const bsort_tune* tune, uint8_t* d_out_rec, uint32_t* d_out_perm,
                             uint32_t* d_out_off, int32_t* d_list_status, void* d_ws,
                             size_t ws_bytes, cudaStream_t s);

/* Copies the bucket contents left in the workspace by bsort_bucket_by_length
 * or bsort_sort_buckets (for inspection and tests): d_keys[k*n + r] is key
 * word k of bucket position r (0 beyond the word's ceil(L/8) keys),
 * d_idx[r] its input index. */
bsort_status bsort_export_buckets(uint32_t n, uint32_t W, const uint32_t* d_off,
                                  const void* d_ws, size_t ws_bytes, uint64_t* d_keys,
                                  uint32_t* d_idx, cudaStream_t s);

/* Per-kernel device timing (tracing; off by default).  While enabled, every
 * kernel launch of the library is bracketed by two CUDA events on its stream.
 * bsort_profile_read() waits for them and returns the number of distinct
 * kernels seen since the last reset; for entry i (i < max_entries) it writes
 * the launch count, the summed device milliseconds and the kernel name
 * (NUL-separated, packed into names[names_bytes]).  Host-side, thread-safe. */
bsort_status bsort_profile_enable(int on);
bsort_status bsort_profile_reset(void);
uint32_t bsort_profile_read(char* names, size_t names_bytes, uint64_t* launches, double* ms,
                            uint32_t max_entries);

/* Synchronises s and returns the smallest device-detected error recorded in
 * the workspace since the last reset (BSORT_OK if none). */
bsort_status bsort_get_status(const void* d_ws, cudaStream_t s);

/* Clears the workspace status word (asynchronously on s). */
bsort_status bsort_reset_status(void* d_ws, cudaStream_t s);

/* Bound of the kernels' device-side waits, for testing the timeout path
 * (the paper has no counterpart).  Every kernel that stages data with the
 * bulk-copy engine waits for the copy on an mbarrier, polling at most `polls`
 * times before it records BSORT_E_TIMEOUT and returns; the wait that then
 * lets the copy in flight land before the CTA exits always keeps the default
 * bound, so no copy outlives its CTA.  polls = 0 makes every such first wait
 * give up at once (the call then reports BSORT_E_TIMEOUT and leaves its
 * outputs undefined, and the context stays usable); BSORT_WAIT_DEFAULT
 * restores the default of 2^26 polls.  Process-wide; read when a call is
 * issued, so it does not change calls already queued or captured in a graph.
 * Not thread-safe against concurrent calls that rely on the default. */
#define BSORT_WAIT_DEFAULT 0xFFFFFFFFu
bsort_status bsort_set_wait_limit(uint32_t polls);

/* Human-readable name of a status code. */
const char* bsort_status_string(bsort_status st);

#ifdef __cplusplus
}
#endif

#endif /* BSORT_H_ */
