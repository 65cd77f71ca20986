/*
 * CPU oracle for TwoPaCo junction detection (arXiv 1602.05856).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header, table or constant with the CUDA library;
 * the two meet only in the seeded input generator.
 *
 * It is deliberately plain and slow: every k-mer is rebuilt from scratch at
 * every position, sets are std::unordered_map / std::unordered_set, and every
 * loop follows the text it cites.
 *
 * Entry points (extern "C", loaded with ctypes):
 *
 *   oracle_junctions   The definition of J(S, k): a vertex of G(S, k) is a
 *                      junction iff it is a bifurcation (more than one
 *                      distinct in-edge or out-edge) or a sentinel (first or
 *                      last k-mer of an input string) -- section
 *                      "Preliminaries". With both_strands the graph is the
 *                      comprehensive graph G(s) U G(s-bar) and every k-mer is
 *                      stored in its normalized form, the lexicographically
 *                      smaller of itself and its reverse complement (the
 *                      reverse-complement paragraph after Algorithm 2).
 *                      PINNED by the tests against the Fig. 1 example, a
 *                      brute-force explicit-graph compactor and invariants.
 *
 *   oracle_junctions_parallel  The same definition split over P threads:
 *                      thread p owns the normalized k-mers whose hash is p
 *                      mod P, scans all input, and decides the positions of
 *                      its own k-mers (the partition-parallel CPU timing the
 *                      benchmark reports). PINNED by equality with
 *                      oracle_junctions for several P.
 *
 *   oracle_alg1_exact  Algorithm 1 (Filter-Junctions) run naively: E is an
 *                      exact set of normalized (k+1)-mers. With every position
 *                      marked it must return J(S, k) (section "Single Round
 *                      Algorithm"). PINNED by equality with the definition
 *                      and by the brute-force compactor.
 *
 *   oracle_edges       Compacted-graph edges: one per pair of consecutive
 *                      junction positions of a string (section "Reduction to
 *                      the Problem of Finding Junction Positions").
 *                      PINNED by Observation 1 against the brute-force
 *                      maximal non-branching paths.
 *
 *   oracle_pass1       The first pass of Algorithm 2 with the vertex-keyed
 *                      split-block Bloom filter that the CUDA library uses as
 *                      E, restated here from its written specification (see
 *                      pass1_* below). It reproduces the candidate set C_temp
 *                      bit for bit. PINNED by invariants only: C_temp
 *                      contains J, is a candidate set (all occurrences of a
 *                      k-mer agree), and equals J when the filter has no
 *                      collisions; the exact bit layout is a design choice of
 *                      this project, not the paper's.
 *
 *   oracle_partition_cuts  The greedy class cut of the multiple-rounds
 *                      heuristic (section "Multiple Rounds") over given bin
 *                      counters. PINNED by worked examples and, on random
 *                      counters, by the greedy property: every class but the
 *                      last stays within the total / l bound and could not
 *                      take its next bin without passing it, unless it must
 *                      leave a bin to each later class.
 *
 * Conventions shared with the library (stated, not shared as code):
 *   bases A,C,G,T (either case) are 0,1,2,3; a k-mer is the integer with its
 *   first base most significant, so integer order is lexicographic order and
 *   the complement of base x is 3 - x. Positions are 0-based k-mer starts:
 *   i in [0, |s| - k]. Strings are never joined.
 *
 * N handling (split_n): the paper does not say what happens to an N. With
 * split_n = 1 every N (either case) ends its string there: the maximal
 * N-free pieces of each string are the strings of the definition (so the
 * first and last k-mers of every piece are sentinels, and no k-mer or edge
 * contains an N), while positions stay 0-based offsets into the original
 * string. With split_n = 0 an N is an invalid byte like any other.
 * PINNED by the tests against the brute-force compactor run on the pieces.
 */
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

typedef unsigned __int128 u128;

// Test builds define ORACLE_MUTANT = n to plant one known mistake, numbered
// where it is planted; each such build must fail a named pin of the tests
// (tests/test_oracle_mutations.py). Otherwise it is 0 and every planted
// branch compiles away.
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(n) (ORACLE_MUTANT == (n))

namespace {

// A k-mer of 64 to 128 bases: four 64-bit words, w[0] the most significant,
// with the same integer encoding as u128 holds for k <= 63 (k-mers of
// 64 <= k <= 127; the (k+1)-mers of Algorithm 1 fit as well).
struct U256 {
  uint64_t w[4] = {0, 0, 0, 0};
  U256() = default;
  explicit U256(uint64_t x) { w[3] = x; }
};

U256 operator<<(const U256& x, int s) {  // 0 <= s < 256
  U256 y;
  const int q = s / 64, r = s % 64;
  for (int i = 0; i < 4; ++i) {
    const int j = i + q;
    uint64_t v = j < 4 ? x.w[j] << r : 0;
    if (r && j + 1 < 4) v |= x.w[j + 1] >> (64 - r);
    y.w[i] = v;
  }
  return y;
}

U256 operator>>(const U256& x, int s) {  // 0 <= s < 256
  U256 y;
  const int q = s / 64, r = s % 64;
  for (int i = 0; i < 4; ++i) {
    const int j = i - q;
    uint64_t v = j >= 0 ? x.w[j] >> r : 0;
    if (r && j - 1 >= 0) v |= x.w[j - 1] << (64 - r);
    y.w[i] = v;
  }
  return y;
}

U256 operator|(const U256& a, const U256& b) {
  U256 y;
  for (int i = 0; i < 4; ++i) y.w[i] = a.w[i] | b.w[i];
  return y;
}

bool operator==(const U256& a, const U256& b) {
  for (int i = 0; i < 4; ++i)
    if (a.w[i] != b.w[i]) return false;
  return true;
}
bool operator!=(const U256& a, const U256& b) { return !(a == b); }
bool operator<(const U256& a, const U256& b) {
  for (int i = 0; i < 4; ++i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return false;
}

// Last base (two least significant bits) of a word.
unsigned last_base(u128 x) { return (unsigned)(x & 3); }
unsigned last_base(const U256& x) { return (unsigned)(x.w[3] & 3); }
// The 128 least significant bits, as (high, low) 64-bit halves.
uint64_t low_hi(u128 x) { return (uint64_t)(x >> 64); }
uint64_t low_lo(u128 x) { return (uint64_t)x; }
uint64_t low_hi(const U256& x) { return x.w[2]; }
uint64_t low_lo(const U256& x) { return x.w[3]; }

enum { ORACLE_OK = 0, ORACLE_EINVAL = -1, ORACLE_EBADBASE = -2 };
constexpr uint8_t kCodeN = 4;

int base_code(uint8_t c, int split_n) {
  switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    case 'N': case 'n': return split_n ? kCodeN : -1;
    default: return -1;
  }
}

struct KmerHash {
  size_t operator()(u128 x) const {
    uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
    return std::hash<uint64_t>()(lo ^ (lo >> 31) ^ (hi * 0x9E3779B97F4A7C15ull));
  }
  size_t operator()(const U256& x) const {
    uint64_t h = 0;
    for (int i = 0; i < 4; ++i) h = (h ^ x.w[i] ^ (x.w[i] >> 31)) * 0x9E3779B97F4A7C15ull;
    return std::hash<uint64_t>()(h);
  }
};

// The string of length len starting at codes[start], as an integer.
template <typename W>
W word_at(const std::vector<uint8_t>& codes, uint64_t start, int len) {
  W x{};
  for (int j = 0; j < len; ++j) x = (x << 2) | W(codes[start + j]);
  return x;
}

// Reverse complement of a len-base word: read backwards, complement each base.
template <typename W>
W reverse_complement(W x, int len) {
  W y{};
  for (int j = 0; j < len; ++j) {
    y = (y << 2) | W(3 - last_base(x));
    x = x >> 2;
  }
  return y;
}

// Normalized form (reverse-complement paragraph after Algorithm 2).
template <typename W>
W normalized(W x, int len, int both_strands) {
  if (!both_strands) return x;
  W r = reverse_complement(x, len);
  return r < x ? r : x;
}

int encode_all(const uint8_t* seq, uint64_t m, int split_n, std::vector<uint8_t>* codes) {
  codes->resize(m);
  for (uint64_t g = 0; g < m; ++g) {
    int c = base_code(seq[g], split_n);
    if (c < 0) return ORACLE_EBADBASE;
    (*codes)[g] = (uint8_t)c;
  }
  return ORACLE_OK;
}

// The strings of the definition: every input string, or with split_n its
// maximal N-free pieces. s0 is the piece's first global byte, len its length,
// string the input string it lies in.
struct Piece {
  uint64_t s0, len, string;
};

std::vector<Piece> pieces(const uint64_t* offsets, uint64_t n, const std::vector<uint8_t>& codes) {
  std::vector<Piece> out;
  for (uint64_t t = 0; t < n; ++t) {
    uint64_t g = offsets[t];
    while (g < offsets[t + 1]) {
      if (codes[g] == kCodeN) {
        ++g;
        continue;
      }
      const uint64_t a = g;
      while (g < offsets[t + 1] && codes[g] != kCodeN) ++g;
      out.push_back({a, g - a, t});
    }
    if (offsets[t] == offsets[t + 1]) out.push_back({offsets[t], 0, t});
  }
  return out;
}

int popcount4(uint8_t x) { return (x & 1) + ((x >> 1) & 1) + ((x >> 2) & 1) + ((x >> 3) & 1); }

struct Degrees {
  uint8_t in = 0;   // bit c set: edge c.v exists
  uint8_t out = 0;  // bit c set: edge v.c exists
};

/*
 * J(S, k) by definition ("Preliminaries"; normalized forms per the
 * reverse-complement paragraph after Algorithm 2).
 *   seq      all strings concatenated (ASCII, m = offsets[n] bytes)
 *   offsets  n + 1 entries; string t is seq[offsets[t] .. offsets[t+1])
 *   flags    m bytes, written: flags[g] = 1 iff the k-mer starting at
 *            global byte g is a junction (0 where no k-mer starts)
 *   n_distinct  optional: number of distinct (normalized) k-mers
 */
template <typename W>
int junctions_impl(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                   int both_strands, int split_n, uint8_t* flags, uint64_t* n_distinct) {
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  std::memset(flags, 0, m);
  const std::vector<Piece> S = pieces(offsets, n, codes);

  // Step 1-2: every occurrence contributes the edges that enter and leave
  // its k-mer, in the orientation of the normalized form.
  std::unordered_map<W, Degrees, KmerHash> deg;
  std::unordered_set<W, KmerHash> sentinels;
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    for (uint64_t i = 0; i + k <= len; ++i) {
      W v = word_at<W>(codes, s0 + i, k);
      W r = both_strands ? reverse_complement(v, k) : v;
      W key = (both_strands && r < v) ? r : v;
      if (MUTANT(3)) key = (both_strands && v < r) ? r : v;  // planted 3: stored under the maximum
      Degrees& d = deg[key];
      const bool has_pred = i >= 1, has_succ = i + k < len;
      const uint64_t succ_at = s0 + i + k - (MUTANT(5) ? 1 : 0);  // planted 5: successor one base early
      if (key == v) {  // forward occurrence of the normalized k-mer
        if (has_pred) d.in |= (uint8_t)(1u << codes[s0 + i - 1]);
        if (has_succ) d.out |= (uint8_t)(1u << codes[succ_at]);
      }
      // planted 7: a palindrome takes only its forward orientation
      if (both_strands && key == r && !(MUTANT(7) && key == v)) {  // occurrence on the other strand
        // planted 2: the other strand's predecessor not complemented
        if (has_succ) d.in |= (uint8_t)(1u << (MUTANT(2) ? codes[s0 + i + k] : 3 - codes[s0 + i + k]));
        if (has_pred) d.out |= (uint8_t)(1u << (3 - codes[s0 + i - 1]));
      }
    }
    // Step 3: first and last k-mer of the string are sentinels.
    if (MUTANT(1)) continue;  // planted 1: no sentinels
    sentinels.insert(normalized(word_at<W>(codes, s0, k), k, both_strands));
    sentinels.insert(normalized(word_at<W>(codes, s0 + len - k, k), k, both_strands));
  }
  // Step 4: junction = sentinel or bifurcation.
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    // planted 4: the last k-mer of a string never flagged
    for (uint64_t i = 0; MUTANT(4) ? i + k < len : i + k <= len; ++i) {
      W key = normalized(word_at<W>(codes, s0 + i, k), k, both_strands);
      const Degrees& d = deg[key];
      const int branch = MUTANT(6) ? 0 : 1;  // planted 6: one edge already counts as a branch
      bool junction = sentinels.count(key) || popcount4(d.in) > branch || popcount4(d.out) > branch;
      flags[s0 + i] = junction ? 1 : 0;
    }
  }
  if (n_distinct) *n_distinct = deg.size();
  return ORACLE_OK;
}

/*
 * Algorithm 1 (Filter-Junctions) with E an exact set of normalized
 * (k+1)-mers. marks (m bytes) is C on entry and the reduced C on exit.
 * Loop bounds follow the 0-based reading 1 <= i < |s| - k, which leaves
 * the two sentinel positions 0 and |s| - k untouched (they stay as given).
 * The sentinel test is on the k-mer, not the position.
 */
// The definition, for the normalized k-mers K with KmerHash(K) % threads ==
// part only: their degrees, their sentinel status, and the flags of the
// positions where they occur (no other thread writes those flags).
template <typename W>
void junctions_part(const std::vector<uint8_t>& codes, const std::vector<Piece>& S, int k,
                    int both_strands, int threads, int part, uint8_t* flags) {
  KmerHash hash;
  auto mine = [&](const W& key) { return (int)(hash(key) % (size_t)threads) == part; };
  std::unordered_map<W, Degrees, KmerHash> deg;
  std::unordered_set<W, KmerHash> sentinels;
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    for (uint64_t i = 0; i + k <= len; ++i) {
      W v = word_at<W>(codes, s0 + i, k);
      W r = both_strands ? reverse_complement(v, k) : v;
      W key = (both_strands && r < v) ? r : v;
      if (!mine(key)) continue;
      Degrees& d = deg[key];
      const bool has_pred = i >= 1, has_succ = i + k < len;
      if (key == v) {
        if (has_pred) d.in |= (uint8_t)(1u << codes[s0 + i - 1]);
        if (has_succ) d.out |= (uint8_t)(1u << codes[s0 + i + k]);
      }
      if (both_strands && key == r) {
        if (has_succ) d.in |= (uint8_t)(1u << (3 - codes[s0 + i + k]));
        if (has_pred) d.out |= (uint8_t)(1u << (3 - codes[s0 + i - 1]));
      }
    }
    const W first = normalized(word_at<W>(codes, s0, k), k, both_strands);
    const W last = normalized(word_at<W>(codes, s0 + len - k, k), k, both_strands);
    if (MUTANT(12)) continue;  // planted 12: the split definition forgets the sentinels
    if (mine(first)) sentinels.insert(first);
    if (mine(last)) sentinels.insert(last);
  }
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    for (uint64_t i = 0; i + k <= len; ++i) {
      W key = normalized(word_at<W>(codes, s0 + i, k), k, both_strands);
      if (!mine(key)) continue;
      const Degrees& d = deg[key];
      flags[s0 + i] = (sentinels.count(key) || popcount4(d.in) > 1 || popcount4(d.out) > 1) ? 1 : 0;
    }
  }
}

template <typename W>
int junctions_parallel_impl(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                            int both_strands, int split_n, int threads, uint8_t* flags) {
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  std::memset(flags, 0, m);
  const std::vector<Piece> S = pieces(offsets, n, codes);
  std::vector<std::thread> pool;
  for (int p = 0; p < threads; ++p)
    pool.emplace_back([&, p] { junctions_part<W>(codes, S, k, both_strands, threads, p, flags); });
  for (std::thread& t : pool) t.join();
  return ORACLE_OK;
}

template <typename W>
int alg1_impl(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
              int both_strands, int split_n, uint8_t* marks) {
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  const std::vector<Piece> S = pieces(offsets, n, codes);
  std::unordered_set<W, KmerHash> E, sentinels;
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    sentinels.insert(normalized(word_at<W>(codes, s0, k), k, both_strands));
    sentinels.insert(normalized(word_at<W>(codes, s0 + len - k, k), k, both_strands));
  }
  // Loop 1: insert the two (k+1)-mers that contain the k-mer at i.
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    for (uint64_t i = 1; i + k < len; ++i) {
      if (!marks[s0 + i]) continue;
      E.insert(normalized(word_at<W>(codes, s0 + i, k + 1), k + 1, both_strands));
      E.insert(normalized(word_at<W>(codes, s0 + i - 1, k + 1), k + 1, both_strands));
    }
  }
  // Loop 2: count existing edges around every marked non-sentinel k-mer.
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    for (uint64_t i = 1; i + k < len; ++i) {
      if (!marks[s0 + i]) continue;
      W v = word_at<W>(codes, s0 + i, k);
      // planted 8: the sentinel test skipped (it is on the k-mer, not the position)
      if (!MUTANT(8) && sentinels.count(normalized(v, k, both_strands))) continue;
      int in = 0, out = 0;
      for (int c = 0; c < 4; ++c) {
        W vc = (v << 2) | W(c);                    // v . c
        W cv = (W(c) << (2 * k)) | v;              // c . v
        if (E.count(normalized(vc, k + 1, both_strands))) ++out;
        if (E.count(normalized(cv, k + 1, both_strands))) ++in;
      }
      if (in == 1 && out == 1) marks[s0 + i] = 0;
    }
  }
  return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * First pass with the vertex-keyed split-block Bloom filter.
 *
 * Specification (restated independently by the CUDA library):
 *   mix64(z)  = splitmix64 finalizer (Steele, Lea & Flood 2014):
 *               z ^= z >> 30; z *= 0xbf58476d1ce4e5b9;
 *               z ^= z >> 27; z *= 0x94d049bb133111eb; z ^= z >> 31.
 *   V = hi * 2^64 + lo, the normalized k-mer (k <= 63), or
 *   V = w0 * 2^192 + w1 * 2^128 + w2 * 2^64 + w3 (64 <= k <= 127).
 *   H = mix64(lo ^ mix64(hi)), resp. mix64(w3 ^ mix64(w2 ^ mix64(w1 ^ mix64(w0))))
 *       (the same value when w0 = w1 = 0, as mix64(0) = 0);
 *   G = H * 0x9e3779b97f4a7c15 (mod 2^64)
 *   The filter has b bits = b/256 blocks of eight 32-bit words; a k-mer
 *   uses one 64-bit half-pair of its block: 32-bit words 2*o and 2*o + 1.
 *   block = H >> (64 - log2(b/256))  (0 when b = 256)
 *   o     = G >> 62
 *   for u < h: word t_u = 2*o + (u & 1), bit base base_u = (G >> (57 - 5u)) & 31
 *   item j sets / tests bit (base_u + j) & 31 of word t_u, for every u < h.
 *   items: j = 4a + c for the (predecessor a, successor c) pair of an
 *          occurrence read in the orientation of the normalized form
 *          (palindromes: both orientations); j = 16 marks a sentinel.
 *   round class: bin = H & (q - 1); a position is active iff its bin is in
 *          [bin_lo, bin_hi).
 *   Loop 1: every active position inserts item 16 if it is the first or
 *          last k-mer of its string (of its N-free piece under split_n),
 *          else its pair item(s).
 *   Loop 2: an active position stays marked iff it is a sentinel position,
 *          or item 16 is present, or at least two pair items are present.
 * ------------------------------------------------------------------------- */
namespace {

uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}

struct FilterSpot {
  uint64_t block;
  uint64_t H;
  uint32_t word[8];  // word index t_u for u < h
  uint32_t base[8];  // bit base for that word
};

uint64_t key_hash64(u128 V) { return mix64((uint64_t)V ^ mix64((uint64_t)(V >> 64))); }
uint64_t key_hash64(const U256& V) {
  return mix64(V.w[3] ^ mix64(V.w[2] ^ mix64(V.w[1] ^ mix64(V.w[0]))));
}

template <typename W>
FilterSpot locate(const W& V, int lg_blocks, int h) {
  FilterSpot f;
  f.H = key_hash64(V);
  uint64_t G = f.H * 0x9e3779b97f4a7c15ull;
  f.block = lg_blocks ? (f.H >> (64 - lg_blocks)) : 0;
  uint32_t o = (uint32_t)(G >> 62);
  for (int u = 0; u < h; ++u) {
    f.word[u] = 2 * o + ((uint32_t)u & 1u);
    f.base[u] = (uint32_t)(G >> (57 - 5 * u)) & 31u;
  }
  return f;
}

void filter_insert(std::vector<uint32_t>& F, const FilterSpot& f, int h, int item) {
  for (int u = 0; u < h; ++u)
    F[f.block * 8 + f.word[u]] |= 1u << ((f.base[u] + (uint32_t)item) & 31u);
}

bool filter_has(const std::vector<uint32_t>& F, const FilterSpot& f, int h, int item) {
  for (int u = 0; u < h; ++u)
    if (!((F[f.block * 8 + f.word[u]] >> ((f.base[u] + (uint32_t)item) & 31u)) & 1u)) return false;
  return true;
}

}  // namespace

template <typename W>
int pass1_impl(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
               int both_strands, int split_n, uint64_t filter_bits, int hashes, uint64_t q,
               uint64_t bin_lo, uint64_t bin_hi, uint8_t* marks, uint64_t* counters) {
  if (hashes < 1 || hashes > 8) return ORACLE_EINVAL;
  if (filter_bits < 256 || (filter_bits & (filter_bits - 1))) return ORACLE_EINVAL;
  if (q < 1 || (q & (q - 1))) return ORACLE_EINVAL;
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  std::memset(marks, 0, m);
  const std::vector<Piece> S = pieces(offsets, n, codes);
  int lg_blocks = 0;
  while ((256ull << lg_blocks) < filter_bits) ++lg_blocks;
  std::vector<uint32_t> F(filter_bits / 32, 0u);
  uint64_t active = 0, kept = 0;

  for (int loop = 1; loop <= 2; ++loop) {
    for (const Piece& pc : S) {
      const uint64_t s0 = pc.s0, len = pc.len;
      if (len < (uint64_t)k) continue;
      for (uint64_t i = 0; i + k <= len; ++i) {
        W v = word_at<W>(codes, s0 + i, k);
        W r = both_strands ? reverse_complement(v, k) : v;
        W key = (both_strands && r < v) ? r : v;
        FilterSpot f = locate(key, lg_blocks, hashes);
        uint64_t bin = f.H & (q - 1);
        if (bin < bin_lo || bin >= bin_hi) continue;
        const bool sentinel_pos = (i == 0) || (i + k == len);
        if (loop == 1) {
          ++active;
          if (sentinel_pos) {
            filter_insert(F, f, hashes, 16);
          } else {
            int a = codes[s0 + i - 1], c = codes[s0 + i + k];
            if (key == v) filter_insert(F, f, hashes, 4 * a + c);
            if (both_strands && key == r) filter_insert(F, f, hashes, 4 * (3 - c) + (3 - a));
          }
        } else {
          bool keep = sentinel_pos || filter_has(F, f, hashes, 16);
          if (!keep) {
            int present = 0;
            for (int j = 0; j < 16; ++j) present += filter_has(F, f, hashes, j) ? 1 : 0;
            keep = present >= (MUTANT(9) ? 1 : 2);  // planted 9: one present item keeps it
          }
          if (keep) {
            marks[s0 + i] = 1;
            ++kept;
          }
        }
      }
    }
  }
  if (counters) {
    counters[0] = active;
    counters[1] = kept;
  }
  return ORACLE_OK;
}

/*
 * Compacted-graph edges (section "Reduction to the Problem of Finding
 * Junction Positions"): for every two consecutive junction positions p < q of
 * a string (of a piece under split_n), one edge from the k-mer at p to the
 * k-mer at q. flags (m bytes)
 * is the output of oracle_junctions. Edges are written in string order, then
 * position order; for each: the normalized start and end k-mers (hi, lo
 * words), whether the string reads the reverse complement of each (0/1), the
 * start position p and the length q - p. Returns the number of edges, or a
 * negative error. The arrays hold at least (number of junctions) entries.
 */
template <typename W>
long long edges_impl(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                     int both_strands, int split_n, const uint8_t* flags, uint64_t* from_hi,
                     uint64_t* from_lo, uint64_t* to_hi, uint64_t* to_lo, uint8_t* from_rc,
                     uint8_t* to_rc, uint64_t* start, uint64_t* length, uint64_t* edges_per_string) {
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  if (edges_per_string)
    for (uint64_t t = 0; t < n; ++t) edges_per_string[t] = 0;
  long long e = 0;
  for (const Piece& pc : pieces(offsets, n, codes)) {
    const uint64_t s0 = pc.s0, len = pc.len, t = pc.string;
    bool have_prev = false;
    uint64_t prev = 0;
    for (uint64_t i = 0; i + k <= len && len >= (uint64_t)k; ++i) {
      if (!flags[s0 + i]) continue;
      if (have_prev) {
        W a = word_at<W>(codes, s0 + prev, k), b = word_at<W>(codes, s0 + i, k);
        W na = normalized(a, k, both_strands), nb = normalized(b, k, both_strands);
        from_hi[e] = low_hi(na);
        from_lo[e] = low_lo(na);
        to_hi[e] = low_hi(nb);
        to_lo[e] = low_lo(nb);
        from_rc[e] = (na != a) ? 1 : 0;
        to_rc[e] = (nb != b) ? 1 : 0;
        start[e] = s0 + prev - offsets[t];  // offset in the input string
        length[e] = i - prev + (MUTANT(11) ? 1 : 0);  // planted 11: length off by one
        ++e;
        if (edges_per_string) ++edges_per_string[t];
      }
      have_prev = true;
      prev = i;
    }
  }
  return e;
}

}  // namespace

extern "C" {

// Entry points: k-mers of up to 63 bases are held in 128-bit words, of 64 to
// 127 bases in 256-bit words (U256); the same code serves both.
int oracle_junctions(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                     int both_strands, int split_n, uint8_t* flags, uint64_t* n_distinct) {
  if (k >= 1 && k <= 63) return junctions_impl<u128>(seq, offsets, n, k, both_strands, split_n, flags, n_distinct);
  if (k >= 64 && k <= 127) return junctions_impl<U256>(seq, offsets, n, k, both_strands, split_n, flags, n_distinct);
  return ORACLE_EINVAL;
}

int oracle_junctions_parallel(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                              int both_strands, int split_n, int threads, uint8_t* flags) {
  if (threads < 1 || threads > 1024) return ORACLE_EINVAL;
  if (k >= 1 && k <= 63)
    return junctions_parallel_impl<u128>(seq, offsets, n, k, both_strands, split_n, threads, flags);
  if (k >= 64 && k <= 127)
    return junctions_parallel_impl<U256>(seq, offsets, n, k, both_strands, split_n, threads, flags);
  return ORACLE_EINVAL;
}

int oracle_alg1_exact(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                      int both_strands, int split_n, uint8_t* marks) {
  if (k >= 1 && k <= 63) return alg1_impl<u128>(seq, offsets, n, k, both_strands, split_n, marks);
  if (k >= 64 && k <= 127) return alg1_impl<U256>(seq, offsets, n, k, both_strands, split_n, marks);
  return ORACLE_EINVAL;
}

/*
 * marks: m bytes, written: 1 where the position is active and survives the
 * first pass, else 0. counters (optional, 2 entries): active positions,
 * surviving positions.
 */
int oracle_pass1(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                 int both_strands, int split_n, uint64_t filter_bits, int hashes, uint64_t q,
                 uint64_t bin_lo, uint64_t bin_hi, uint8_t* marks, uint64_t* counters) {
  if (k >= 1 && k <= 63)
    return pass1_impl<u128>(seq, offsets, n, k, both_strands, split_n, filter_bits, hashes, q, bin_lo,
                            bin_hi, marks, counters);
  if (k >= 64 && k <= 127)
    return pass1_impl<U256>(seq, offsets, n, k, both_strands, split_n, filter_bits, hashes, q, bin_lo,
                            bin_hi, marks, counters);
  return ORACLE_EINVAL;
}

/*
 * Compacted-graph edges: see edges_impl. For k > 63 the from/to words hold
 * the 128 least significant bits of the normalized k-mers (their last 64
 * bases).
 */
long long oracle_edges(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                       int both_strands, int split_n, const uint8_t* flags, uint64_t* from_hi,
                       uint64_t* from_lo, uint64_t* to_hi, uint64_t* to_lo, uint8_t* from_rc,
                       uint8_t* to_rc, uint64_t* start, uint64_t* length, uint64_t* edges_per_string) {
  if (k >= 1 && k <= 63)
    return edges_impl<u128>(seq, offsets, n, k, both_strands, split_n, flags, from_hi, from_lo, to_hi,
                            to_lo, from_rc, to_rc, start, length, edges_per_string);
  if (k >= 64 && k <= 127)
    return edges_impl<U256>(seq, offsets, n, k, both_strands, split_n, flags, from_hi, from_lo, to_hi,
                            to_lo, from_rc, to_rc, start, length, edges_per_string);
  return ORACLE_EINVAL;
}

/*
 * Greedy class cut of the multiple-rounds heuristic (section "Multiple
 * Rounds"): scan the q counters in order and close a class as soon as adding
 * the next counter would push its sum above (sum of all counters) / l, while
 * giving every class at least one bin; the last class takes what is left.
 * The comparison sum <= total / l is made exactly, as l * sum <= total.
 * cuts: l + 1 entries, class r owns bins [cuts[r], cuts[r+1]).
 */
int oracle_partition_cuts(const uint64_t* counts, uint64_t q, int l, uint64_t* cuts) {
  if (l < 1 || q < (uint64_t)l) return ORACLE_EINVAL;
  u128 total = 0;
  for (uint64_t j = 0; j < q; ++j) total += counts[j];
  uint64_t j = 0;
  cuts[0] = 0;
  for (int r = 0; r < l - 1; ++r) {
    u128 sum = 0;
    uint64_t start = j;
    // at least one bin, and leave at least one bin for each later class
    // planted 10: no bin left over for the later classes
    while (j < (MUTANT(10) ? q : q - (uint64_t)(l - 1 - r))) {
      if (j > start && (sum + counts[j]) * (u128)l > total) break;
      sum += counts[j];
      ++j;
    }
    cuts[r + 1] = j;
  }
  cuts[l] = q;
  return ORACLE_OK;
}

}  // extern "C"
