"""Seeded synthetic inputs shaped like the paper's workloads.

The paper sorts the words of two English prose files (§3 Methodology: about
190 KB and 1.38 MB of text).  Those texts are not used here; these generators
produce seeded stand-ins of the same shape instead.  This module only draws
random bytes: it does no tokenising, bucketing or sorting, so the CUDA path
and the CPU oracle can both take their inputs from it.

Random numbers: SplitMix64 (Steele, Lea and Flood, 2014) in counter mode.  The
value for counter ``c`` of stream ``key`` is the SplitMix64 output mix applied
to ``key + (c + 1) * 0x9E3779B97F4A7C15``.  Streams are keyed by (seed, tag),
so every array is a pure function of its seed and independent of chunking.

Recipe (all words are lowercase ``a``..``z``):

* word lengths 1..16 follow ``LENGTH_WEIGHTS_16`` (mean 4.49, mode 3);
  the 32-wide records extend this with 1 % mass on 17..32, geometric with
  ratio 0.75;
* a vocabulary holds V distinct random words (length from the weights,
  letters uniform); duplicates are redrawn;
* word identities follow Zipf(s = 1.1) over the vocabulary ranks, sampled by
  inverse CDF;
* batched lists share one V-word pool, each list relabelling its ranks by a
  seeded affine bijection;
* text: one space between words; after a word, with probability 0.08, one of
  ``,.;:!?'-`` follows directly; after ``'`` or ``-`` the next word follows
  with no space half of the time; once a line reaches 60 bytes the separator
  is a newline.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

LENGTH_WEIGHTS_16 = np.array(
    [3.3, 18.0, 21.8, 18.0, 11.4, 7.9, 6.7, 4.8, 3.1, 2.1, 1.25, 0.7, 0.4, 0.22, 0.12, 0.08])
PUNCT = b",.;:!?'-"
ZIPF_S = 1.1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

_TAGS = {"len": 1, "letters": 2, "zipf": 3, "mix": 4, "punct": 5, "pchar": 6, "glue": 7,
         "vocab_len": 8, "vocab_letters": 9, "size": 10, "arrive": 11, "kind": 12,
         "vocab": 13}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: str, sub: int = 0) -> np.uint64:
    """Key of the stream (seed, tag, sub): SplitMix64 of a fixed combination."""
    with np.errstate(over="ignore"):
        base = np.array([(seed * 0x100000001B3 + _TAGS[tag] * 0x1000193 + sub * 0x9E37)
                         & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return np.uint64(_mix(base + _GOLDEN)[0])


def raw64(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Counters start..start+count-1 of stream ``key`` as uint64."""
    with np.errstate(over="ignore"):
        c = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(key) + c * _GOLDEN)


def uniform01(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (raw64(key, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def letters(key: np.uint64, start_word: int, n: int, width: int) -> np.ndarray:
    """``n x width`` uniform letters a..z, four 16-bit draws per uint64."""
    per = (width + 3) // 4
    r = raw64(key, start_word * per, n * per).reshape(n, per)
    parts = [((r >> np.uint64(16 * j)) & np.uint64(0xFFFF)) for j in range(4)]
    u16 = np.stack(parts, axis=2).reshape(n, per * 4)[:, :width]
    return (ord("a") + ((u16 * np.uint64(26)) >> np.uint64(16))).astype(np.uint8)


def length_pmf(width: int) -> np.ndarray:
    """Probabilities of lengths 1..width (index 0 is length 1)."""
    w16 = LENGTH_WEIGHTS_16 / LENGTH_WEIGHTS_16.sum()
    if width <= 16:
        p = w16[:width]
        return p / p.sum()
    tail_n = width - 16
    r = 0.75
    tail = np.array([(1 - r) * r ** k for k in range(tail_n)])
    tail = 0.01 * tail / tail.sum()
    return np.concatenate([0.99 * w16, tail])


def sample_lengths(u: np.ndarray, pmf: np.ndarray) -> np.ndarray:
    cdf = np.cumsum(pmf)
    cdf[-1] = 1.0
    return (np.searchsorted(cdf, u, side="right") + 1).astype(np.uint8)


def random_words(seed: int, tag_len: str, tag_letters: str, start: int, n: int,
                 width: int, pmf: np.ndarray, sub: int = 0):
    """n random words: lengths from ``pmf``, letters uniform, zero padded."""
    ln = sample_lengths(uniform01(stream_key(seed, tag_len, sub), start, n), pmf)
    let = letters(stream_key(seed, tag_letters, sub), start, n, width)
    let[np.arange(width)[None, :] >= ln[:, None]] = 0
    return let, ln


@lru_cache(maxsize=16)
def _vocab_cached(seed: int, V: int, width: int, max_len: int):
    pmf = length_pmf(max_len)
    rec = np.zeros((0, width), dtype=np.uint8)
    ln = np.zeros(0, dtype=np.uint8)
    drawn = 0
    seen_keys = np.zeros(0, dtype=np.uint64)
    while rec.shape[0] < V:
        batch = max(1024, int((V - rec.shape[0]) * 1.15))
        r, l = random_words(seed, "vocab_len", "vocab_letters", drawn, batch, width, pmf,
                            sub=V)
        drawn += batch
        # identity of a word = its padded bytes; folded to 64 bits for de-duplication
        words64 = np.ascontiguousarray(r).view(np.uint64).reshape(batch, width // 8)
        with np.errstate(over="ignore"):
            h = np.zeros(batch, dtype=np.uint64)
            for j in range(words64.shape[1]):
                h = _mix(h ^ words64[:, j] + np.uint64(j + 1) * _GOLDEN)
        allk = np.concatenate([seen_keys, h])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keep_new = first[first >= seen_keys.size] - seen_keys.size
        rec = np.concatenate([rec, r[keep_new]])
        ln = np.concatenate([ln, l[keep_new]])
        seen_keys = np.concatenate([seen_keys, h[keep_new]])
    rec, ln = rec[:V], ln[:V]
    rec.setflags(write=False)
    ln.setflags(write=False)
    return rec, ln


def vocabulary(seed: int, V: int, width: int = 16, max_len: int | None = None):
    """V distinct random words (``rec[V, width]`` zero padded, ``len[V]``)."""
    assert width % 8 == 0
    return _vocab_cached(seed, V, width, max_len or width)


@lru_cache(maxsize=8)
def zipf_cdf(V: int, s: float = ZIPF_S) -> np.ndarray:
    w = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    c /= c[-1]
    c.setflags(write=False)
    return c


def zipf_ranks(u: np.ndarray, V: int) -> np.ndarray:
    """Zipf ranks 0..V-1 from uniforms by inverse CDF."""
    return np.minimum(np.searchsorted(zipf_cdf(V), u, side="right"), V - 1)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def zipf_words(seed: int, n: int, V: int, width: int = 16, vocab_seed: int | None = None):
    """n word records drawn by Zipf rank from a V-word vocabulary."""
    vrec, vlen = vocabulary(seed if vocab_seed is None else vocab_seed, V, width)
    ranks = zipf_ranks(uniform01(stream_key(seed, "zipf"), 0, n), V)
    return vrec[ranks].copy(), vlen[ranks].copy()


def prose(seed: int, n_words: int, V: int) -> bytes:
    """English-shaped text of exactly ``n_words`` words (lowercase, 1..16 letters)."""
    vrec, vlen = vocabulary(seed, V, 16)
    ranks = zipf_ranks(uniform01(stream_key(seed, "zipf"), 0, n_words), V)
    vocab_bytes = [bytes(vrec[i, :vlen[i]]) for i in range(V)]
    u_p = uniform01(stream_key(seed, "punct"), 0, n_words)
    pc = (raw64(stream_key(seed, "pchar"), 0, n_words) % np.uint64(len(PUNCT))).astype(int)
    u_g = uniform01(stream_key(seed, "glue"), 0, n_words)
    out = bytearray()
    line = 0
    for i in range(n_words):
        w = vocab_bytes[ranks[i]]
        out += w
        line += len(w)
        glue = False
        if u_p[i] < 0.08:
            c = PUNCT[pc[i]]
            out.append(c)
            line += 1
            glue = c in b"'-" and u_g[i] < 0.5
        if glue and i + 1 < n_words:
            continue
        if line >= 60 or i + 1 == n_words:
            out.append(0x0A)
            line = 0
        else:
            out.append(0x20)
            line += 1
    return bytes(out)


def large_records(seed: int, n: int, width: int = 32, V: int = 1 << 20,
                  zipf_frac: float = 0.30, chunk: int = 1 << 20):
    """Pre-tokenised records: ``zipf_frac`` of words from a V-word Zipf
    vocabulary, the rest random; lengths 1..width (16 + geometric tail)."""
    pmf = length_pmf(width)
    vrec, vlen = vocabulary(seed, V, width, width)
    rec = np.empty((n, width), dtype=np.uint8)
    ln = np.empty(n, dtype=np.uint8)
    kmix, kz = stream_key(seed, "mix"), stream_key(seed, "zipf")
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        r, l = random_words(seed, "len", "letters", s, m, width, pmf)
        pick = uniform01(kmix, s, m) < zipf_frac
        ranks = zipf_ranks(uniform01(kz, s, m), V)[pick]
        r[pick] = vrec[ranks]
        l[pick] = vlen[ranks]
        rec[s:s + m] = r
        ln[s:s + m] = l
    return rec, ln


def list_size(seed: int, lo: int = 64, hi: int = 65536) -> int:
    """Log-uniform size floor(exp(U[ln lo, ln(hi + 1))))."""
    u = uniform01(stream_key(seed, "size"), 0, 1)[0]
    return int(math.floor(math.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))))


def list_words(seed: int, n: int, V: int = 50_000, width: int = 16, vocab_seed: int = 0):
    """One list of the batched workload: n Zipf words over a per-list vocabulary.

    All lists share one V-word pool (drawn once from ``vocab_seed``); list
    ``seed`` relabels the pool's ranks by its own affine bijection
    ``k -> (a k + b) mod V`` (a coprime to V), so each list has its own
    rank-to-word assignment without drawing V new words per list."""
    vrec, vlen = vocabulary(vocab_seed, V, width)
    r = raw64(stream_key(seed, "vocab"), 0, 2)
    a = int(r[0] % np.uint64(V)) | 1
    while math.gcd(a, V) != 1:
        a = (a + 2) % V or 1
    b = int(r[1] % np.uint64(V))
    ranks = zipf_ranks(uniform01(stream_key(seed, "zipf"), 0, n), V)
    ids = (ranks.astype(np.int64) * a + b) % V
    return vrec[ids].copy(), vlen[ids].copy()


def batch_lists(n_lists: int, V: int = 50_000, width: int = 16, lo: int = 64,
                hi: int = 65536, seed0: int = 0):
    """Independent Zipf word lists; list i uses seed ``seed0 + i``.

    Returns ``(rec, len, sizes)`` with the lists concatenated in order."""
    sizes = [list_size(seed0 + i, lo, hi) for i in range(n_lists)]
    recs, lens = [], []
    for i, m in enumerate(sizes):
        r, l = list_words(seed0 + i, m, V, width)
        recs.append(r)
        lens.append(l)
    rec = np.concatenate(recs) if recs else np.zeros((0, width), np.uint8)
    ln = np.concatenate(lens) if lens else np.zeros(0, np.uint8)
    return rec, ln, np.array(sizes, dtype=np.int64)


def request_stream(seed: int, rate_per_s: float, duration_s: float, lo: int = 1024,
                   hi: int = 1 << 20, text_frac: float = 0.10):
    """Poisson arrivals: ``(arrival_times_s, sizes, is_text)`` for a served run."""
    n_max = int(rate_per_s * duration_s * 1.5 + 64)
    gaps = -np.log1p(-uniform01(stream_key(seed, "arrive"), 0, n_max)) / rate_per_s
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    k = t.size
    u = uniform01(stream_key(seed, "size"), 0, k)
    sizes = np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64)
    is_text = uniform01(stream_key(seed, "kind"), 0, k) < text_frac
    return t, sizes, is_text
