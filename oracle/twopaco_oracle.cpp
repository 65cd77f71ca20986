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
#include <unordered_map>
#include <unordered_set>
#include <vector>

typedef unsigned __int128 u128;

namespace {

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
};

// The string of length len starting at codes[start], as an integer.
u128 word_at(const std::vector<uint8_t>& codes, uint64_t start, int len) {
  u128 x = 0;
  for (int j = 0; j < len; ++j) x = (x << 2) | codes[start + j];
  return x;
}

// Reverse complement of a len-base word: read backwards, complement each base.
u128 reverse_complement(u128 x, int len) {
  u128 y = 0;
  for (int j = 0; j < len; ++j) {
    y = (y << 2) | (u128)(3 - (int)(x & 3));
    x >>= 2;
  }
  return y;
}

// Normalized form (reverse-complement paragraph after Algorithm 2).
u128 normalized(u128 x, int len, int both_strands) {
  if (!both_strands) return x;
  u128 r = reverse_complement(x, len);
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

}  // namespace

extern "C" {

/*
 * J(S, k) by definition ("Preliminaries"; normalized forms per the
 * reverse-complement paragraph after Algorithm 2).
 *   seq      all strings concatenated (ASCII, m = offsets[n] bytes)
 *   offsets  n + 1 entries; string t is seq[offsets[t] .. offsets[t+1])
 *   flags    m bytes, written: flags[g] = 1 iff the k-mer starting at
 *            global byte g is a junction (0 where no k-mer starts)
 *   n_distinct  optional: number of distinct (normalized) k-mers
 */
int oracle_junctions(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                     int both_strands, int split_n, uint8_t* flags, uint64_t* n_distinct) {
  if (k < 1 || k > 63) return ORACLE_EINVAL;
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  std::memset(flags, 0, m);
  const std::vector<Piece> S = pieces(offsets, n, codes);

  // Step 1-2: every occurrence contributes the edges that enter and leave
  // its k-mer, in the orientation of the normalized form.
  std::unordered_map<u128, Degrees, KmerHash> deg;
  std::unordered_set<u128, KmerHash> sentinels;
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    for (uint64_t i = 0; i + k <= len; ++i) {
      u128 v = word_at(codes, s0 + i, k);
      u128 r = both_strands ? reverse_complement(v, k) : v;
      u128 key = (both_strands && r < v) ? r : v;
      Degrees& d = deg[key];
      const bool has_pred = i >= 1, has_succ = i + k < len;
      if (key == v) {  // forward occurrence of the normalized k-mer
        if (has_pred) d.in |= (uint8_t)(1u << codes[s0 + i - 1]);
        if (has_succ) d.out |= (uint8_t)(1u << codes[s0 + i + k]);
      }
      if (both_strands && key == r) {  // occurrence on the other strand
        if (has_succ) d.in |= (uint8_t)(1u << (3 - codes[s0 + i + k]));
        if (has_pred) d.out |= (uint8_t)(1u << (3 - codes[s0 + i - 1]));
      }
    }
    // Step 3: first and last k-mer of the string are sentinels.
    sentinels.insert(normalized(word_at(codes, s0, k), k, both_strands));
    sentinels.insert(normalized(word_at(codes, s0 + len - k, k), k, both_strands));
  }
  // Step 4: junction = sentinel or bifurcation.
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    for (uint64_t i = 0; i + k <= len; ++i) {
      u128 key = normalized(word_at(codes, s0 + i, k), k, both_strands);
      const Degrees& d = deg[key];
      bool junction = sentinels.count(key) || popcount4(d.in) > 1 || popcount4(d.out) > 1;
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
int oracle_alg1_exact(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                      int both_strands, int split_n, uint8_t* marks) {
  if (k < 1 || k > 63) return ORACLE_EINVAL;
  const uint64_t m = offsets[n];
  std::vector<uint8_t> codes;
  int rc = encode_all(seq, m, split_n, &codes);
  if (rc) return rc;
  const std::vector<Piece> S = pieces(offsets, n, codes);
  std::unordered_set<u128, KmerHash> E, sentinels;
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    if (len < (uint64_t)k) continue;
    sentinels.insert(normalized(word_at(codes, s0, k), k, both_strands));
    sentinels.insert(normalized(word_at(codes, s0 + len - k, k), k, both_strands));
  }
  // Loop 1: insert the two (k+1)-mers that contain the k-mer at i.
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    for (uint64_t i = 1; i + k < len; ++i) {
      if (!marks[s0 + i]) continue;
      E.insert(normalized(word_at(codes, s0 + i, k + 1), k + 1, both_strands));
      E.insert(normalized(word_at(codes, s0 + i - 1, k + 1), k + 1, both_strands));
    }
  }
  // Loop 2: count existing edges around every marked non-sentinel k-mer.
  for (const Piece& pc : S) {
    const uint64_t s0 = pc.s0, len = pc.len;
    for (uint64_t i = 1; i + k < len; ++i) {
      if (!marks[s0 + i]) continue;
      u128 v = word_at(codes, s0 + i, k);
      if (sentinels.count(normalized(v, k, both_strands))) continue;
      int in = 0, out = 0;
      for (int c = 0; c < 4; ++c) {
        u128 vc = (v << 2) | (u128)c;                    // v . c
        u128 cv = ((u128)c << (2 * k)) | v;              // c . v
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
 *   V = hi * 2^64 + lo, the normalized k-mer.
 *   H = mix64(lo ^ mix64(hi));  G = H * 0x9e3779b97f4a7c15 (mod 2^64)
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

FilterSpot locate(u128 V, int lg_blocks, int h) {
  FilterSpot f;
  uint64_t lo = (uint64_t)V, hi = (uint64_t)(V >> 64);
  f.H = mix64(lo ^ mix64(hi));
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

/*
 * marks: m bytes, written: 1 where the position is active and survives the
 * first pass, else 0. counters (optional, 2 entries): active positions,
 * surviving positions.
 */
int oracle_pass1(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                 int both_strands, int split_n, uint64_t filter_bits, int hashes, uint64_t q,
                 uint64_t bin_lo, uint64_t bin_hi, uint8_t* marks, uint64_t* counters) {
  if (k < 1 || k > 63 || hashes < 1 || hashes > 8) return ORACLE_EINVAL;
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
        u128 v = word_at(codes, s0 + i, k);
        u128 r = both_strands ? reverse_complement(v, k) : v;
        u128 key = (both_strands && r < v) ? r : v;
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
            keep = present >= 2;
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
 * a string, one edge from the k-mer at p to the k-mer at q. flags (m bytes)
 * is the output of oracle_junctions. Edges are written in string order, then
 * position order; for each: the normalized start and end k-mers (hi, lo
 * words), whether the string reads the reverse complement of each (0/1), the
 * start position p and the length q - p. Returns the number of edges, or a
 * negative error. The arrays hold at least (number of junctions) entries.
 */
long long oracle_edges(const uint8_t* seq, const uint64_t* offsets, uint64_t n, int k,
                       int both_strands, int split_n, const uint8_t* flags, uint64_t* from_hi,
                       uint64_t* from_lo, uint64_t* to_hi, uint64_t* to_lo, uint8_t* from_rc,
                       uint8_t* to_rc, uint64_t* start, uint64_t* length, uint64_t* edges_per_string) {
  if (k < 1 || k > 63) return ORACLE_EINVAL;
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
        u128 a = word_at(codes, s0 + prev, k), b = word_at(codes, s0 + i, k);
        u128 na = normalized(a, k, both_strands), nb = normalized(b, k, both_strands);
        from_hi[e] = (uint64_t)(na >> 64);
        from_lo[e] = (uint64_t)na;
        to_hi[e] = (uint64_t)(nb >> 64);
        to_lo[e] = (uint64_t)nb;
        from_rc[e] = (na != a) ? 1 : 0;
        to_rc[e] = (nb != b) ? 1 : 0;
        start[e] = s0 + prev - offsets[t];  // offset in the input string
        length[e] = i - prev;
        ++e;
        if (edges_per_string) ++edges_per_string[t];
      }
      have_prev = true;
      prev = i;
    }
  }
  return e;
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
    while (j < q - (uint64_t)(l - 1 - r)) {
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
