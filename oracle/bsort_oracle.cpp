// Reference oracle for the length-bucketed word sort -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU restatement of the method of Alyasseri et
// al., "Parallelize Bubble and Merge Sort Algorithms Using MPI" (arXiv 1411.5283),
// §3 Methodology, "Pre-processing":
//   phase 1  remove / ignore the special characters of the text;
//   phase 2  put the words into sub-arrays by character count, shorter lengths
//            before longer ones (abstract: sub-array sizes come from the number
//            of words of each length);
//   phase 3  sort each sub-array alphabetically with bubble sort (§2 and §3.2:
//            compare neighbours, swap when out of order, repeat passes until a
//            pass makes no swap; n(n-1)/2 compares in the worst case).
// The concatenation of the sub-arrays in ascending length is the answer.
// The paper also times the whole file sorted alphabetically by bubble sort
// without the sub-arrays (Table 2, second row); that variant is restated too.
//
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
// load this library. It shares no code, header or constant with the CUDA path.
//
// Readings of the paper taken here (the paper is silent on each):
//   * "removing / ignoring" special characters: a non-letter byte is a word
//     separator ("don't" -> "don", "t"), not deleted-and-joined;
//   * a letter is an ASCII byte in 'A'..'Z' or 'a'..'z'; every other byte,
//     including bytes >= 0x80, is a separator;
//   * no case folding: words compare as unsigned byte strings (memcmp);
//   * duplicate words are kept; bubble sort swaps only on a strict '>' so equal
//     words keep input order (ties broken by input index);
//   * the 3-D char array fixes a record width W; a word longer than W is an
//     error, never truncated.
//
// Status codes are this file's own (they coincide in value with the library's
// by design of the tests, not by a shared header):
//   0 ok, 1 invalid argument / zero-length record, 2 word longer than W,
//   3 more words than the capacity. When several errors are present the
//   smallest code is returned.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int ORC_OK = 0;
constexpr int ORC_E_INVALID = 1;
constexpr int ORC_E_WORD_TOO_LONG = 2;
constexpr int ORC_E_CAPACITY = 3;

// Phase 1: a letter is an ASCII Latin letter; anything else separates words.
inline bool is_letter(uint8_t b) {
  return (b >= 'A' && b <= 'Z') || (b >= 'a' && b <= 'z');
}

int smallest_error(unsigned flags) {
  for (int c = 1; c < 32; ++c)
    if (flags & (1u << c)) return c;
  return ORC_OK;
}

// Validates a table of records: every length must lie in 1..W.
unsigned check_lengths(const uint8_t* len, uint32_t n, uint32_t W) {
  unsigned flags = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (len[i] == 0) flags |= 1u << ORC_E_INVALID;
    else if (len[i] > W) flags |= 1u << ORC_E_WORD_TOO_LONG;
  }
  return flags;
}

// Phase 2: one sub-array per word length, members in input order.
std::vector<std::vector<uint32_t>> split_by_length(const uint8_t* len, uint32_t n,
                                                   uint32_t W) {
  std::vector<std::vector<uint32_t>> sub(W + 1);
  for (uint32_t i = 0; i < n; ++i) sub[len[i]].push_back(i);
  return sub;
}

// Concatenation in ascending length: out_rec gets the L letters of each word
// followed by zeros up to W; out_perm the input index; off[L] the number of
// words shorter than L (off[0] = off[1] = 0, off[W+1] = n).
void concatenate(const std::vector<std::vector<uint32_t>>& sub, const uint8_t* rec,
                 uint32_t W, uint8_t* out_rec, uint32_t* out_perm, uint32_t* off) {
  uint32_t r = 0;
  off[0] = 0;
  for (uint32_t L = 1; L <= W; ++L) {
    off[L] = r;
    for (uint32_t id : sub[L]) {
      if (out_rec) {
        std::memset(out_rec + (uint64_t)r * W, 0, W);
        std::memcpy(out_rec + (uint64_t)r * W, rec + (uint64_t)id * W, L);
      }
      if (out_perm) out_perm[r] = id;
      ++r;
    }
  }
  off[W + 1] = r;
}

}  // namespace

extern "C" {

// Phase 1 (§3, "Pre-processing", first phase). Scans text left to right; each
// maximal run of letters is a word, numbered in order of appearance. Writes up
// to max_words records (W bytes each, zero padded), their lengths and the byte
// offset of their first letter. *n_words receives the number of words found
// (even when it exceeds max_words).
int orc_tokenize(const uint8_t* text, uint64_t n_bytes, uint32_t W, uint32_t max_words,
                 uint8_t* rec, uint8_t* len, uint32_t* src_off, uint32_t* n_words) {
  if (W == 0 || W > 255 || (n_bytes > 0 && text == nullptr) || n_words == nullptr)
    return ORC_E_INVALID;
  unsigned flags = 0;
  uint32_t count = 0;
  uint64_t p = 0;
  while (p < n_bytes) {
    if (!is_letter(text[p])) { ++p; continue; }
    uint64_t start = p;
    while (p < n_bytes && is_letter(text[p])) ++p;
    uint64_t L = p - start;
    if (L > W) flags |= 1u << ORC_E_WORD_TOO_LONG;
    if (count < max_words) {
      if (rec) {
        std::memset(rec + (uint64_t)count * W, 0, W);
        std::memcpy(rec + (uint64_t)count * W, text + start, L > W ? W : L);
      }
      if (len) len[count] = (uint8_t)(L > 255 ? 255 : L);
      if (src_off) src_off[count] = (uint32_t)start;
    } else {
      flags |= 1u << ORC_E_CAPACITY;
    }
    ++count;
  }
  *n_words = count;
  return smallest_error(flags);
}

// Phase 2 alone: the sub-array of each length, in input order, concatenated in
// ascending length (bucket_ids), with the same off[] layout as concatenate().
int orc_split_by_length(const uint8_t* len, uint32_t n, uint32_t W, uint32_t* off,
                        uint32_t* bucket_ids) {
  if (W == 0 || W > 255) return ORC_E_INVALID;
  unsigned flags = check_lengths(len, n, W);
  if (flags) return smallest_error(flags);
  auto sub = split_by_length(len, n, W);
  concatenate(sub, nullptr, W, nullptr, bucket_ids, off);
  return ORC_OK;
}

// Phases 2 and 3 and the concatenation, with the paper's bubble sort: in each
// pass neighbouring words are compared and swapped when the left one sorts
// after the right one; passes repeat until one makes no swap (§2). swaps[L]
// receives the number of exchanges made in the sub-array of length L.
int orc_bubble_sort(const uint8_t* rec, const uint8_t* len, uint32_t n, uint32_t W,
                    uint8_t* out_rec, uint32_t* out_perm, uint32_t* off,
                    uint64_t* swaps) {
  if (W == 0 || W > 255) return ORC_E_INVALID;
  unsigned flags = check_lengths(len, n, W);
  if (flags) return smallest_error(flags);
  auto sub = split_by_length(len, n, W);
  for (uint32_t L = 1; L <= W; ++L) {
    std::vector<uint32_t>& b = sub[L];
    const uint64_t m = b.size();
    uint64_t exchanged = 0;
    for (uint64_t pass = 0; m > 1 && pass < m - 1; ++pass) {
      bool swapped = false;
      for (uint64_t j = 0; j + 1 < m - pass; ++j) {
        const uint8_t* a = rec + (uint64_t)b[j] * W;
        const uint8_t* c = rec + (uint64_t)b[j + 1] * W;
        if (std::memcmp(a, c, L) > 0) {
          std::swap(b[j], b[j + 1]);
          swapped = true;
          ++exchanged;
        }
      }
      if (!swapped) break;
    }
    if (swaps) swaps[L] = exchanged;
  }
  if (swaps) swaps[0] = 0;
  concatenate(sub, rec, W, out_rec, out_perm, off);
  return ORC_OK;
}

// Second formulation of the same result: one stable library sort of all word
// ids by (length, bytes). Used where bubble sort's n^2/2 compares are too slow.
int orc_stable_sort(const uint8_t* rec, const uint8_t* len, uint32_t n, uint32_t W,
                    uint8_t* out_rec, uint32_t* out_perm, uint32_t* off) {
  if (W == 0 || W > 255) return ORC_E_INVALID;
  unsigned flags = check_lengths(len, n, W);
  if (flags) return smallest_error(flags);
  std::vector<uint32_t> ids(n);
  for (uint32_t i = 0; i < n; ++i) ids[i] = i;
  std::stable_sort(ids.begin(), ids.end(), [&](uint32_t a, uint32_t b) {
    if (len[a] != len[b]) return len[a] < len[b];
    return std::memcmp(rec + (uint64_t)a * W, rec + (uint64_t)b * W, len[a]) < 0;
  });
  std::vector<std::vector<uint32_t>> sub(W + 1);
  for (uint32_t id : ids) sub[len[id]].push_back(id);
  concatenate(sub, rec, W, out_rec, out_perm, off);
  return ORC_OK;
}

// The paper's other experiment (Table 2, second row): the whole file's words
// sorted alphabetically by bubble sort, without the length sub-arrays.  Words
// compare as byte strings (a proper prefix first), ties by input index (the
// bubble sort swaps only on a strict '>').  out_rec, out_perm as above; swaps
// receives the number of exchanges.
int orc_bubble_sort_whole(const uint8_t* rec, const uint8_t* len, uint32_t n, uint32_t W,
                          uint8_t* out_rec, uint32_t* out_perm, uint64_t* swaps) {
  if (W == 0 || W > 255) return ORC_E_INVALID;
  unsigned flags = check_lengths(len, n, W);
  if (flags) return smallest_error(flags);
  std::vector<uint32_t> b(n);
  for (uint32_t i = 0; i < n; ++i) b[i] = i;
  const auto after = [&](uint32_t x, uint32_t y) {  // word x sorts after word y
    const uint8_t* a = rec + (uint64_t)x * W;
    const uint8_t* c = rec + (uint64_t)y * W;
    return std::lexicographical_compare(c, c + len[y], a, a + len[x]);
  };
  uint64_t exchanged = 0;
  for (uint64_t pass = 0; n > 1 && pass < (uint64_t)n - 1; ++pass) {
    bool swapped = false;
    for (uint64_t j = 0; j + 1 < (uint64_t)n - pass; ++j) {
      if (after(b[j], b[j + 1])) {
        std::swap(b[j], b[j + 1]);
        swapped = true;
        ++exchanged;
      }
    }
    if (!swapped) break;
  }
  if (swaps) *swaps = exchanged;
  for (uint32_t r = 0; r < n; ++r) {
    if (out_rec) {
      std::memset(out_rec + (uint64_t)r * W, 0, W);
      std::memcpy(out_rec + (uint64_t)r * W, rec + (uint64_t)b[r] * W, len[b[r]]);
    }
    if (out_perm) out_perm[r] = b[r];
  }
  return ORC_OK;
}

// The same answer by one stable library sort on the byte strings.
int orc_stable_sort_whole(const uint8_t* rec, const uint8_t* len, uint32_t n, uint32_t W,
                          uint8_t* out_rec, uint32_t* out_perm) {
  if (W == 0 || W > 255) return ORC_E_INVALID;
  unsigned flags = check_lengths(len, n, W);
  if (flags) return smallest_error(flags);
  std::vector<uint32_t> ids(n);
  for (uint32_t i = 0; i < n; ++i) ids[i] = i;
  std::stable_sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) {
    const uint8_t* a = rec + (uint64_t)x * W;
    const uint8_t* c = rec + (uint64_t)y * W;
    return std::lexicographical_compare(a, a + len[x], c, c + len[y]);
  });
  for (uint32_t r = 0; r < n; ++r) {
    if (out_rec) {
      std::memset(out_rec + (uint64_t)r * W, 0, W);
      std::memcpy(out_rec + (uint64_t)r * W, rec + (uint64_t)ids[r] * W, len[ids[r]]);
    }
    if (out_perm) out_perm[r] = ids[r];
  }
  return ORC_OK;
}

}  // extern "C"
