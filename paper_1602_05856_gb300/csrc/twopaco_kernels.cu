// CUDA kernels of the junction-detection library (sm_103a).
//
// One run = pack, then per round (Algorithm 3, section "Multiple Rounds")
// the two passes of Algorithm 2 (Filter-Junctions-Two-Pass), each an
// instance of Algorithm 1 (Filter-Junctions): an insert loop and a probe
// loop, separated by a kernel boundary (the barrier of section
// "Parallelization Scheme"); then one emit of the junction positions.
//
// The first pass visits every position. An insert thread takes kInsertR
// consecutive positions and rolls the forward and reverse-complement k-mer
// words from one to the next; besides its filter OR it leaves an 8-byte
// descriptor per position, which the probe streams (4 rows of 32 positions
// per warp and step) instead of walking again. The second pass visits only
// the candidates the first pass left, from a compact list.
//
// Encoding: A,C,G,T = 0,1,2,3, 16 bases per 32-bit word, first base in the
// two most significant bits. A k-mer is the integer with its first base most
// significant, so integer order is lexicographic order (the normalized form
// of a k-mer is min(k-mer, reverse complement)), and complement is 3 - x.
#include "twopaco_internal.h"

#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

// This file is compiled twice: on its own (every kernel but the k > 63
// ones, and the library's entry points), and with TWOPACO_WIDE_ONLY from
// twopaco_kernels_wide.cu (only the k > 63 instances, launch_round_wide and
// launch_partition_count_wide), so that the two halves build in parallel.

namespace twopaco {

// Optional per-kernel timing: CUDA events recorded on the launch stream
// right before and after every kernel (state shared by both halves).
struct ProfRecord {
  const char* name;
  cudaEvent_t start, stop;
};
extern std::atomic<unsigned long long> g_launches;
extern std::mutex g_prof_mu;
extern bool g_prof_on;
extern std::vector<ProfRecord> g_prof;
extern std::vector<cudaEvent_t> g_event_pool;
#ifndef TWOPACO_WIDE_ONLY
std::atomic<unsigned long long> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_prof;
std::vector<cudaEvent_t> g_event_pool;
#endif

namespace {

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Scope that brackets one kernel launch with events when profiling is on.
struct Timed {
  ProfRecord rec{nullptr, nullptr, nullptr};
  cudaStream_t s;
  unsigned flags = cudaEventRecordDefault;
  Timed(const char* name, cudaStream_t st) : s(st) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on) return;
    rec.name = name;
    rec.start = take_event();
    rec.stop = take_event();
    // inside a stream capture the events must become graph nodes of their own
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      flags = cudaEventRecordExternal;
    cudaEventRecordWithFlags(rec.start, s, flags);
  }
  ~Timed() {
    if (!rec.name) return;
    cudaEventRecordWithFlags(rec.stop, s, flags);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back(rec);
  }
};

// Consecutive positions per thread (at most 16: one 32-bit word of successor
// bases) in the first-pass kernels and the partition pre-pass.
constexpr int kInsertR = 16;
constexpr int kProbeR = 8;
// Loads issued one step ahead (measured: the probe's descriptors and the
// classify's records gain; the second-pass insert's records lose).
constexpr bool kProbePrefetch = true;
constexpr bool kInsertPrefetch = false;
constexpr bool kClassifyPrefetch = true;
constexpr int kR = 8;  // partition pre-pass

using Ranges = std::vector<std::pair<uint64_t, uint64_t>>;

// ---------------------------------------------------------------------------
// k-mer words
// ---------------------------------------------------------------------------

struct Key {
  uint64_t hi, lo;  // value = hi * 2^64 + lo; hi == 0 for k <= 31
};

// k-mers of 64 to 127 bases: four words, w[0] the most significant.
struct Key4 {
  uint64_t w[4];
};

// The k-mer word of KW = 1 (k <= 31), 2 (k <= 63) or 4 (k <= 127).
template <int KW>
struct KeyOf {
  using T = Key;
};
template <>
struct KeyOf<4> {
  using T = Key4;
};
template <int KW>
using KeyT = typename KeyOf<KW>::T;

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

__device__ __forceinline__ bool key_less(const Key4& a, const Key4& b) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return false;
}

__device__ __forceinline__ bool key_eq(const Key4& a, const Key4& b) {
  return a.w[0] == b.w[0] && a.w[1] == b.w[1] && a.w[2] == b.w[2] && a.w[3] == b.w[3];
}

// a0:a1:a2:a3 (a0 most significant) shifted right by s bits, 0 <= s <= 128.
__device__ __forceinline__ Key4 shr256(uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3, int s) {
  if (s >= 64) {
    a3 = a2; a2 = a1; a1 = a0; a0 = 0; s -= 64;
  }
  if (s >= 64) {
    a3 = a2; a2 = a1; a1 = a0; a0 = 0; s -= 64;
  }
  if (s) {
    a3 = (a3 >> s) | (a2 << (64 - s));
    a2 = (a2 >> s) | (a1 << (64 - s));
    a1 = (a1 >> s) | (a0 << (64 - s));
    a0 >>= s;
  }
  return Key4{{a0, a1, a2, a3}};
}

// splitmix64 output finalizer (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}

// H of a k-mer: mix64(lo), mix64(lo ^ mix64(hi)), or for four words
// mix64(w3 ^ mix64(w2 ^ mix64(w1 ^ mix64(w0)))) -- the same value whenever the
// higher words are zero, as mix64(0) = 0.
template <int KW>
__device__ __forceinline__ uint64_t key_hash(const KeyT<KW>& v) {
  if constexpr (KW == 4) return mix64(v.w[3] ^ mix64(v.w[2] ^ mix64(v.w[1] ^ mix64(v.w[0]))));
  else return KW == 1 ? mix64(v.lo) : mix64(v.lo ^ mix64(v.hi));
}

// Second hash word: H times the 64-bit golden ratio; only its high bits are used.
__device__ __forceinline__ uint64_t second_hash(uint64_t H) { return H * 0x9e3779b97f4a7c15ull; }

// Start slot of a k-mer in the pass-2 table (bits above the partition bins).
__device__ __forceinline__ uint64_t slot_hash(uint64_t H) { return H >> 16; }

// Start slot of a k-mer in a pass-2 table of cap slots (any capacity): bits
// 16-47 of H scaled to [0, cap) by a multiply-high (Lemire, "Fast random
// integer generation in an interval", 2019); larger tables take a remainder.
__device__ __forceinline__ uint64_t slot_start(uint64_t H, uint64_t cap) {
  if (cap <= 0xFFFFFFFFull) return __umulhi((uint32_t)(H >> 16), (uint32_t)cap);
  return slot_hash(H) % cap;
}

// The slot after i in linear probing, wrapping at cap.
__device__ __forceinline__ uint64_t next_slot(uint64_t i, uint64_t cap) { return i + 1 == cap ? 0 : i + 1; }

// Reverse the order of the 32 two-bit groups of x.
__device__ __forceinline__ uint64_t rev_pairs(uint64_t x) {
  const uint64_t b = __brevll(x);
  return ((b >> 1) & 0x5555555555555555ull) | ((b & 0x5555555555555555ull) << 1);
}

__device__ __forceinline__ uint32_t base_at(const uint32_t* __restrict__ packed, uint64_t g) {
  return (__ldg(packed + (g >> 4)) >> (30u - 2u * (uint32_t)(g & 15))) & 3u;
}

// 32 bases starting at base g, first base in the two most significant bits.
__device__ __forceinline__ uint64_t bases32(const uint32_t* __restrict__ packed, uint64_t g) {
  const uint32_t* p = packed + (g >> 4);
  const uint32_t o2 = 2u * (uint32_t)(g & 15);
  const uint32_t w0 = __ldg(p), w1 = __ldg(p + 1);
  uint64_t a = ((uint64_t)w0 << 32) | w1;
  if (o2) a = (a << o2) | (__ldg(p + 2) >> (32u - o2));
  return a;
}

// The k-mer starting at base g. KW = 1 for k <= 31 (one 64-bit word), 2 for
// 32 <= k <= 63, 4 for 64 <= k <= 127.
template <int KW>
__device__ __forceinline__ KeyT<KW> load_kmer(const uint32_t* __restrict__ packed, uint64_t g, int k) {
  if constexpr (KW == 4) {
    // 128 bases from g, then the first k of them
    return shr256(bases32(packed, g), bases32(packed, g + 32), bases32(packed, g + 64),
                  bases32(packed, g + 96), 256 - 2 * k);
  } else {
    const uint64_t a = bases32(packed, g);
    Key v;
    if (KW == 1) {
      v.hi = 0;
      v.lo = a >> (64 - 2 * k);
    } else {
      const uint64_t b = bases32(packed, g + 32);
      const int sh = 128 - 2 * k;  // 2 .. 64
      if (sh == 64) {
        v.hi = 0;
        v.lo = a;
      } else {
        v.hi = a >> sh;
        v.lo = (b >> sh) | (a << (64 - sh));
      }
    }
    return v;
  }
}

// Reverse complement of a k-mer.
template <int KW>
__device__ __forceinline__ KeyT<KW> revcomp(const KeyT<KW>& v, int k) {
  if constexpr (KW == 4) {
    return shr256(rev_pairs(~v.w[3]), rev_pairs(~v.w[2]), rev_pairs(~v.w[1]), rev_pairs(~v.w[0]),
                  256 - 2 * k);
  } else {
    Key r;
    if (KW == 1) {
      r.hi = 0;
      r.lo = rev_pairs(~v.lo) >> (64 - 2 * k);
    } else {
      const uint64_t nh = rev_pairs(~v.lo), nl = rev_pairs(~v.hi);
      const int sh = 128 - 2 * k;
      if (sh == 64) {
        r.hi = 0;
        r.lo = nh;
      } else {
        r.hi = nh >> sh;
        r.lo = (nl >> sh) | (nh << (64 - sh));
      }
    }
    return r;
  }
}

// Slide the k-mer one base to the right: f gains base b at its end, r (the
// reverse complement) gains 3 - b at its start.
template <int KW>
__device__ __forceinline__ void roll(KeyT<KW>& f, KeyT<KW>& r, uint32_t b, int k) {
  if constexpr (KW == 4) {
    f.w[0] = (f.w[0] << 2) | (f.w[1] >> 62);
    f.w[1] = (f.w[1] << 2) | (f.w[2] >> 62);
    f.w[2] = (f.w[2] << 2) | (f.w[3] >> 62);
    f.w[3] = (f.w[3] << 2) | b;
    const int hb = 2 * k - 128;  // bits above the two low words, 0 .. 126
    if (hb > 64) {
      f.w[0] &= (1ull << (hb - 64)) - 1ull;
    } else {
      f.w[0] = 0;
      if (hb < 64) f.w[1] &= (1ull << hb) - 1ull;
    }
    r.w[3] = (r.w[3] >> 2) | (r.w[2] << 62);
    r.w[2] = (r.w[2] >> 2) | (r.w[1] << 62);
    r.w[1] = (r.w[1] >> 2) | (r.w[0] << 62);
    r.w[0] >>= 2;
    const int top = 2 * k - 2;  // bit of the first base, from the least significant
    const uint64_t c = 3u - b;
    if (top >= 192) r.w[0] |= c << (top - 192);
    else if (top >= 128) r.w[1] |= c << (top - 128);
    else r.w[2] |= c << (top - 64);
  } else if (KW == 1) {
    f.lo = ((f.lo << 2) | b) & ((1ull << (2 * k)) - 1ull);
    r.lo = (r.lo >> 2) | ((uint64_t)(3u - b) << (2 * k - 2));
  } else {
    const int hb = 2 * k - 64;  // bits of the high word, 0 .. 62
    f.hi = ((f.hi << 2) | (f.lo >> 62)) & ((1ull << hb) - 1ull);
    f.lo = (f.lo << 2) | b;
    r.lo = (r.lo >> 2) | (r.hi << 62);
    r.hi >>= 2;
    if (hb >= 2) r.hi |= (uint64_t)(3u - b) << (hb - 2);
    else r.lo |= (uint64_t)(3u - b) << 62;
  }
}

// First base of a k-mer.
template <int KW>
__device__ __forceinline__ uint32_t first_base(const KeyT<KW>& f, int k) {
  if constexpr (KW == 4) {
    const int top = 2 * k - 2;
    const uint64_t x = top >= 192 ? f.w[0] >> (top - 192) : (top >= 128 ? f.w[1] >> (top - 128) : f.w[2] >> (top - 64));
    return (uint32_t)x & 3u;
  } else if (KW == 1) {
    return (uint32_t)(f.lo >> (2 * k - 2)) & 3u;
  } else {
    return (uint32_t)(k == 32 ? f.lo >> 62 : f.hi >> (2 * k - 66)) & 3u;
  }
}

// ---------------------------------------------------------------------------
// Positions and occurrences
// ---------------------------------------------------------------------------

struct Bounds {
  uint64_t start, end;
};

// [start, end) of the string that holds base g (largest t with offsets[t] <= g).
__device__ __forceinline__ Bounds seq_bounds(const RunView& v, uint64_t g) {
  uint32_t lo = 0, hi = v.n_seqs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(v.offsets + mid) <= g) lo = mid; else hi = mid;
  }
  return {__ldg(v.offsets + lo), __ldg(v.offsets + lo + 1)};
}

// The string bounds a k-mer at g must lie in. Without N splitting these are
// the input string's; with it, the N-free piece holding g, or the empty
// range [g, g) when base g is N (no k-mer starts there, and the next
// position looks its bounds up again).
__device__ __forceinline__ Bounds kmer_bounds(const RunView& v, uint64_t g) {
  if (!v.nmask) return seq_bounds(v, g);
  if ((__ldg(v.nmask + (g >> 5)) >> (g & 31)) & 1u) return {g, g};
  const uint64_t n = __ldcg(&v.hdr->n_runs);  // runs[n] = m
  uint64_t lo = 0, hi = n;                    // largest j < n with runs[j] <= g
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(v.runs + mid) <= g) lo = mid; else hi = mid;
  }
  return {__ldg(v.runs + lo), __ldg(v.runs + lo + 1)};
}

// One k-mer occurrence, read in the orientation of its normalized form.
template <int KW>
struct OccT {
  KeyT<KW> key;    // normalized k-mer
  uint64_t H;      // key_hash(key)
  uint32_t items;  // filter items this occurrence inserts (bit j = item j)
  uint32_t tbits;  // pass-2 bits: in-bases 0-3, out-bases 4-7, sentinel 8
  bool sentinel;   // first or last k-mer of its string
  bool rc;         // the string reads the reverse complement of key here
};

// The filter items and pass-2 bits of one occurrence: its (predecessor,
// successor) pair read in the orientation of the normalized form (both
// orientations of a palindrome), or the sentinel item and bit.
__device__ __forceinline__ void occ_bits(uint32_t pred, uint32_t succ, bool use_f, bool use_r, bool sentinel,
                                         uint32_t* items_out, uint32_t* tbits_out) {
  if (sentinel) {
    *items_out = 1u << 16;
    *tbits_out = 1u << 8;
    return;
  }
  uint32_t items = 0, tb = 0;
  if (use_f) {
    items |= 1u << (4 * pred + succ);
    tb |= (1u << pred) | (16u << succ);
  }
  if (use_r) {
    const uint32_t a = 3u - succ, c = 3u - pred;  // predecessor / successor on the other strand
    items |= 1u << (4 * a + c);
    tb |= (1u << a) | (16u << c);
  }
  *items_out = items;
  *tbits_out = tb;
}

template <int KW>
__device__ __forceinline__ void make_occ(const RunView& v, const KeyT<KW>& f, const KeyT<KW>& r,
                                         uint32_t pred, uint32_t succ, bool sentinel, OccT<KW>* oc) {
  const bool use_f = !v.both || !key_less(r, f);  // f is the normalized form
  const bool use_r = v.both && !key_less(f, r);   // r is (palindromes: both)
  oc->key = use_f ? f : r;
  oc->H = key_hash<KW>(oc->key);
  oc->sentinel = sentinel;
  oc->rc = !use_f;
  occ_bits(pred, succ, use_f, use_r, sentinel, &oc->items, &oc->tbits);
}

// The occurrence at global position g, read from scratch; false if no k-mer
// starts at g.
template <int KW>
__device__ __forceinline__ bool read_occurrence(const RunView& v, uint64_t g, OccT<KW>* oc) {
  const Bounds b = kmer_bounds(v, g);
  if (g + (uint64_t)v.k > b.end) return false;
  const KeyT<KW> f = load_kmer<KW>(v.packed, g, v.k);
  const bool has_pred = g > b.start, has_succ = g + (uint64_t)v.k < b.end;
  const uint32_t pred = has_pred ? base_at(v.packed, g - 1) : 0u;
  const uint32_t succ = has_succ ? base_at(v.packed, g + v.k) : 0u;
  const KeyT<KW> r = v.both ? revcomp<KW>(f, v.k) : f;
  make_occ<KW>(v, f, r, pred, succ, !has_pred || !has_succ, oc);
  return true;
}

// Distance from p0 to x, clamped to [-2^30, 2^30] (positions within one
// thread's chunk are compared in 32 bits).
__device__ __forceinline__ int32_t rel(uint64_t x, uint64_t p0) {
  constexpr int64_t kClamp = 1ll << 30;
  const int64_t d = (int64_t)(x - p0);
  return (int32_t)(d > kClamp ? kClamp : (d < -kClamp ? -kClamp : d));
}

// The occurrence of a listed candidate: its string bounds are not needed,
// because the list marks candidates at a string end (sentinel positions)
// and every other candidate has a predecessor and a successor.
template <int KW>
__device__ __forceinline__ void read_listed(const RunView& v, uint64_t g, bool sentinel, OccT<KW>* oc) {
  const KeyT<KW> f = load_kmer<KW>(v.packed, g, v.k);
  const KeyT<KW> r = v.both ? revcomp<KW>(f, v.k) : f;
  const uint32_t pred = sentinel ? 0u : base_at(v.packed, g - 1);
  const uint32_t succ = sentinel ? 0u : base_at(v.packed, g + v.k);
  make_occ<KW>(v, f, r, pred, succ, sentinel, oc);
}

// Visit the R consecutive positions p0 .. p0 + R - 1 (p0 < m), rolling the
// k-mer from each position to the next within a string and reading it from
// scratch after a string boundary. fn(i, p, valid, occ) runs for every i,
// with i a compile-time constant once unrolled.
template <int KW, int R, typename F>
__device__ __forceinline__ void walk(const RunView& v, uint64_t p0, F&& fn) {
  static_assert(R >= 1 && R <= 16, "successor bases come from one 32-bit word");
  const int k = v.k;
  Bounds b = kmer_bounds(v, p0);
  int32_t s_rel = rel(b.start, p0), e_rel = rel(b.end, p0);  // string bounds relative to p0
  const int32_t m_rel = rel(v.m, p0);
  // bases p0 + k .. p0 + k + R - 1: the successor of each position, which is
  // also the base that enters the k-mer when it slides to the next position
  const uint32_t next = (uint32_t)(bases32(v.packed, p0 + (uint64_t)k) >> 32);
  KeyT<KW> f{}, r{};
  bool fresh = true;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const uint64_t p = p0 + i;
    OccT<KW> oc;
    bool valid = false;
    if (i < m_rel) {
      if (i >= e_rel) {  // p starts a later string (or piece)
        b = kmer_bounds(v, p);
        s_rel = rel(b.start, p0);
        e_rel = rel(b.end, p0);
        fresh = true;
      }
      if (i + k <= e_rel) {
        valid = true;
        uint32_t pred;
        if (fresh) {
          f = load_kmer<KW>(v.packed, p, k);
          if (v.both) r = revcomp<KW>(f, k);
          pred = i > s_rel ? base_at(v.packed, p - 1) : 0u;
          fresh = false;
        } else {
          pred = first_base<KW>(f, k);  // the first base of the previous k-mer
          roll<KW>(f, r, i > 0 ? (next >> (32 - 2 * i)) & 3u : 0u, k);
        }
        const uint32_t succ = (next >> (30 - 2 * i)) & 3u;
        const bool sentinel = i == s_rel || i + k == e_rel;
        make_occ<KW>(v, f, v.both ? r : f, pred, succ, sentinel, &oc);
      } else {
        fresh = true;
      }
    }
    fn(i, p, valid, oc);
  }
}

__device__ __forceinline__ bool in_round(const RunView& v, uint64_t H, int round) {
  const uint32_t bin = (uint32_t)H & v.qmask;
  return bin >= __ldg(v.cuts + round) && bin < __ldg(v.cuts + round + 1);
}

// ---------------------------------------------------------------------------
// First-pass filter: b bits = b/256 blocks of four 64-bit words. A k-mer owns
// one 64-bit word: block from the top bits of H, word o from the top two bits
// of G. Each of its h bits u has a 5-bit base cut from G, in the low (u even)
// or high (u odd) half; item j sets bit (base_u + j) & 31 of that half. All 17
// items of a k-mer live in one word: an insert is one 64-bit atomic OR and a
// probe is one 8-byte load that answers all of its items at once.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long* filter_word(const RunView& v, uint64_t H, uint64_t G) {
  // b <= 2^40 bits: the block index has at most 32 bits
  const uint32_t block = v.lg_blocks ? (uint32_t)(H >> (64 - v.lg_blocks)) : 0u;
  return v.filter + ((uint64_t)block * 4u + (uint32_t)(G >> 62));
}

__device__ __forceinline__ uint32_t bit_base(uint64_t G, int u) {
  const int sh = 57 - 5 * u;  // u is a compile-time constant once unrolled
  if (sh >= 32) return ((uint32_t)(G >> 32) >> (sh - 32)) & 31u;
  return (uint32_t)(G >> sh) & 31u;
}

// The bits of item 0 in each half of the word; item j is both halves
// rotated left by j (bit (base_u + j) mod 32).
struct ItemPattern {
  uint32_t lo, hi;
};

// HB > 0: that many bits per item, a compile-time constant; HB = 0: hb bits,
// a run-time value (the k > 63 kernels, to keep their instances few).
template <int HB>
__device__ __forceinline__ ItemPattern item_pattern(uint64_t G, int hb) {
  ItemPattern p{0u, 0u};
#pragma unroll
  for (int u = 0; u < (HB ? HB : 8); ++u) {
    if (!HB && u >= hb) break;
    const uint32_t b = 1u << bit_base(G, u);
    if (u & 1) p.hi |= b; else p.lo |= b;
  }
  return p;
}

__device__ __forceinline__ uint64_t item_bits(const ItemPattern& p, uint32_t j) {
  return ((uint64_t)__funnelshift_l(p.hi, p.hi, j) << 32) | __funnelshift_l(p.lo, p.lo, j);
}

template <int HB>
__device__ __forceinline__ uint64_t item_bits(uint64_t G, uint32_t j, int hb) {
  return item_bits(item_pattern<HB>(G, hb), j);
}

// Bit j of the result: item j is present (all of its bits are set).
template <int HB>
__device__ __forceinline__ uint32_t present_items(uint64_t G, uint64_t w, int hb) {
  const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
  uint32_t pres = 0x1FFFFu;
#pragma unroll
  for (int u = 0; u < (HB ? HB : 8); ++u) {
    if (!HB && u >= hb) break;
    const uint32_t x = (u & 1) ? hi : lo;
    pres &= __funnelshift_r(x, x, bit_base(G, u));
  }
  return pres & 0x1FFFFu;
}

// Index of a k-mer's filter word (the word filter_word points to).
__device__ __forceinline__ uint64_t filter_index(const RunView& v, uint64_t H, uint64_t G) {
  const uint32_t block = v.lg_blocks ? (uint32_t)(H >> (64 - v.lg_blocks)) : 0u;
  return (uint64_t)block * 4u + (uint32_t)(G >> 62);
}

// ---------------------------------------------------------------------------
// Region-bucketed first-pass inserts. A filter far larger than L2 takes its
// random ORs at DRAM's random-access rate, about a tenth of the rate L2 takes
// them at. So for such a filter the insert loop turns every OR into an 8-byte
// record in the bucket of its filter region (32 MiB, which L2 holds), and the
// apply kernel then performs the ORs bucket by bucket, while the region stays
// in L2. A record: bits 0-21 the word within its region, 22-51 the bits 32-61
// of G (the bit bases of up to 6 bits per item), 52-56 and 57-61 the items (two
// for a palindrome's orientations). A full bucket takes the OR directly.
// ---------------------------------------------------------------------------

constexpr uint32_t kApplyPiece = 4096;  // records per apply work item
constexpr uint32_t kFillStride = 32;    // bucket counters 128 bytes apart (one L2 line each)

// A region's records go to one of its sub-buckets (chosen by the warp, so
// that every region has at least 256 counters between them): the bucket
// index is region * n_sub + sub, region-major, so that the apply's order
// still takes one region after the other.
__device__ __forceinline__ void stage_or(const RunView& v, uint64_t word, uint64_t G, uint32_t j1, uint32_t j2,
                                         uint64_t mask) {
  const uint32_t warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const uint32_t b = (uint32_t)(word >> v.lg_region_words) * v.n_sub + (warp & (v.n_sub - 1u));
  const unsigned grp = __match_any_sync(__activemask(), b);
  const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(v.bucket_fill + (uint64_t)b * kFillStride, (uint32_t)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  const uint64_t slot = (uint64_t)base + __popc(grp & ((1u << lane) - 1u));
  if (slot < v.bucket_cap) {
    const uint64_t local = word & ((1ull << v.lg_region_words) - 1ull);
    v.bucket_recs[(uint64_t)b * v.bucket_cap + slot] =
        local | (((G >> 32) & 0x3FFFFFFFull) << 22) | ((uint64_t)j1 << 52) | ((uint64_t)j2 << 57);
  } else {
    atomicOr(v.filter + word, (unsigned long long)mask);
  }
}

// The ORs of the staged records, in work items of kApplyPiece records taken in
// bucket order from a ticket (so that the blocks in flight work on one or two
// regions at a time). The counter after the last bucket's is the ticket.
template <int HB>
__global__ void __launch_bounds__(kBlock) filter_apply_kernel(RunView v) {
  __shared__ uint32_t first_s[kMaxBuckets + 1];  // first work item of every bucket
  __shared__ uint32_t item_s;
  const uint32_t R = v.n_regions * v.n_sub;  // buckets
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t b = 0; b < R; ++b) {
      first_s[b] = acc;
      const uint64_t n = min((uint64_t)__ldcg(v.bucket_fill + (uint64_t)b * kFillStride), v.bucket_cap);
      acc += (uint32_t)((n + kApplyPiece - 1) / kApplyPiece);
    }
    first_s[R] = acc;
  }
  __syncthreads();
  const uint32_t total = first_s[R];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(v.bucket_fill + (uint64_t)R * kFillStride, 1u);
    __syncthreads();
    const uint32_t item = item_s;
    __syncthreads();
    if (item >= total) break;
    uint32_t lo = 0, hi = R;  // the bucket b with first_s[b] <= item < first_s[b + 1]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (first_s[mid] <= item) lo = mid; else hi = mid;
    }
    const uint32_t b = lo;
    const uint64_t n = min((uint64_t)__ldcg(v.bucket_fill + (uint64_t)b * kFillStride), v.bucket_cap);
    const uint64_t i0 = (uint64_t)(item - first_s[b]) * kApplyPiece;
    const uint64_t i1 = min(i0 + kApplyPiece, n);
    const uint64_t* recs = v.bucket_recs + (uint64_t)b * v.bucket_cap;
    const uint64_t region = (uint64_t)(b / v.n_sub) << v.lg_region_words;
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += kBlock) {
      const uint64_t r = __ldcs(recs + i);
      const uint64_t G = ((r >> 22) & 0x3FFFFFFFull) << 32;  // the bits bit_base reads for u < 6
      const ItemPattern pat = item_pattern<HB>(G, v.hashes);
      const uint32_t j1 = (uint32_t)(r >> 52) & 31u, j2 = (uint32_t)(r >> 57) & 31u;
      uint64_t m = item_bits(pat, j1);
      if (j2 != j1) m |= item_bits(pat, j2);
      atomicOr(v.filter + (region | (r & ((1ull << 22) - 1ull))), (unsigned long long)m);
    }
  }
}

// ---------------------------------------------------------------------------
// Pass-2 table: open addressing with linear probing, keyed by the normalized
// k-mer; the value is the 9-bit pass-2 mask. Empty keys are all ones, which
// no k-mer of k <= 63 can be.
// ---------------------------------------------------------------------------

struct alignas(16) Slot1 {
  unsigned long long key;
  unsigned int mask;
  unsigned int pad;
};

struct alignas(32) Slot2 {
  unsigned long long w0, w1;  // key.lo, key.hi (one 128-bit word, w0 low)
  unsigned int mask;
  unsigned int pad;
  unsigned long long pad2;
};

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kMaskBits = 9;

__device__ __forceinline__ void cas128(unsigned long long* addr, uint64_t cmp_lo, uint64_t cmp_hi,
                                       uint64_t new_lo, uint64_t new_hi, uint64_t* old_lo,
                                       uint64_t* old_hi) {
  uint64_t ol, oh;
  asm volatile(
      "{\n\t.reg .b128 c, n, d;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 n, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], c, n;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(ol), "=l"(oh)
      : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(addr)
      : "memory");
  *old_lo = ol;
  *old_hi = oh;
}

constexpr uint64_t kNoSlot = ~0ull;

// Insert (key, bits) into a table of cap TS-kind slots (table_slot_kind),
// probing from slot start (< cap); the key's slot, or kNoSlot if every slot
// was tried (the table is full). Bits already present are not written again.
template <int TS>
__device__ __forceinline__ uint64_t table_insert(const RunView& v, uint64_t cap, const Key& key,
                                             uint64_t start, uint32_t bits) {
  uint64_t i = start;
  for (uint64_t probe = 0; probe < cap; ++probe, i = next_slot(i, cap)) {
    if (TS == 0) {
      // one word: key << 9 | mask bits; never all ones for a key < 2^54. A
      // plain load first: most candidates meet their k-mer already in the
      // table, and a random load costs less than a random atomic
      unsigned long long* s = static_cast<unsigned long long*>(v.table) + i;
      unsigned long long cur = __ldcg(s);
      if (cur == kEmpty) {
        cur = atomicCAS(s, kEmpty, (key.lo << kMaskBits) | bits);
        if (cur == kEmpty) return i;
      }
      if ((cur >> kMaskBits) != key.lo) continue;
      if ((cur & bits) != bits) atomicOr(s, (unsigned long long)bits);
      return i;
    } else if (TS == 1) {
      Slot1* s = static_cast<Slot1*>(v.table) + i;
      const ulonglong2 w = __ldcg(reinterpret_cast<const ulonglong2*>(s));
      unsigned long long cur = w.x;
      uint32_t have = (uint32_t)w.y;
      if (cur == kEmpty) {
        cur = atomicCAS(&s->key, kEmpty, (unsigned long long)key.lo);
        if (cur == kEmpty) cur = key.lo;
        have = 0;
      }
      if (cur != key.lo) continue;
      if ((have & bits) != bits) atomicOr(&s->mask, bits);
      return i;
    } else {
      Slot2* s = static_cast<Slot2*>(v.table) + i;
      uint64_t ol, oh;
      cas128(&s->w0, kEmpty, kEmpty, key.lo, key.hi, &ol, &oh);
      const bool mine = (ol == kEmpty && oh == kEmpty) || (ol == key.lo && oh == key.hi);
      if (!mine) continue;
      if ((__ldcg(&s->mask) & bits) != bits) atomicOr(&s->mask, bits);
      return i;
    }
  }
  return kNoSlot;
}

// Mask of key, or -1 if absent.
template <int TS>
__device__ __forceinline__ int table_find(const RunView& v, uint64_t cap, const Key& key, uint64_t start) {
  uint64_t i = start;
  for (uint64_t probe = 0; probe < cap; ++probe, i = next_slot(i, cap)) {
    if (TS == 0) {
      const unsigned long long cur = __ldcg(static_cast<const unsigned long long*>(v.table) + i);
      if (cur == kEmpty) return -1;
      if ((cur >> kMaskBits) == key.lo) return (int)(cur & ((1u << kMaskBits) - 1u));
    } else if (TS == 1) {
      const Slot1* s = static_cast<const Slot1*>(v.table) + i;
      const ulonglong2 w = __ldcg(reinterpret_cast<const ulonglong2*>(s));
      if (w.x == key.lo) return (int)(unsigned int)w.y;
      if (w.x == kEmpty) return -1;
    } else {
      const Slot2* s = static_cast<const Slot2*>(v.table) + i;
      const ulonglong2 w = __ldcg(reinterpret_cast<const ulonglong2*>(&s->w0));
      if (w.x == key.lo && w.y == key.hi) return (int)__ldcg(&s->mask);
      if (w.x == kEmpty && w.y == kEmpty) return -1;
    }
  }
  return -1;
}

// Slots of k-mers of 64 to 127 bases (kind 3): instead of the key, a
// reference to one occurrence of it -- bits 0-47 its position + 1, bit 48
// whether the string reads the key's reverse complement there, bits 49-63
// the top 15 bits of H as a tag. 0 is empty. Keys are compared by reading the
// referenced occurrence back from the packed input, so one 64-bit CAS claims
// a slot for a key of any length.
struct alignas(16) Slot3 {
  unsigned long long ref;
  unsigned int mask;
  unsigned int pad;
};

constexpr uint64_t kRefPos = (1ull << 48) - 1;

__device__ __forceinline__ bool ref_holds(const RunView& v, uint64_t ref, const Key4& key) {
  Key4 x = load_kmer<4>(v.packed, (ref & kRefPos) - 1, v.k);
  if ((ref >> 48) & 1u) x = revcomp<4>(x, v.k);
  return key_eq(x, key);
}

__device__ __forceinline__ uint64_t table_insert_ref(const RunView& v, uint64_t cap, const Key4& key,
                                                     uint64_t H, uint32_t bits, uint64_t g, bool rc) {
  const uint64_t tag = H >> 49;
  const unsigned long long mine = (tag << 49) | ((uint64_t)rc << 48) | (g + 1);
  uint64_t i = slot_start(H, cap);
  for (uint64_t probe = 0; probe < cap; ++probe, i = next_slot(i, cap)) {
    Slot3* s = static_cast<Slot3*>(v.table) + i;
    unsigned long long cur = __ldcg(&s->ref);
    if (cur == 0) {
      cur = atomicCAS(&s->ref, 0ull, mine);
      if (cur == 0) {
        atomicOr(&s->mask, bits);
        return i;
      }
    }
    if ((cur >> 49) != tag || !ref_holds(v, cur, key)) continue;
    if ((__ldcg(&s->mask) & bits) != bits) atomicOr(&s->mask, bits);
    return i;
  }
  return kNoSlot;
}

__device__ __forceinline__ int table_find_ref(const RunView& v, uint64_t cap, const Key4& key, uint64_t H) {
  const uint64_t tag = H >> 49;
  uint64_t i = slot_start(H, cap);
  for (uint64_t probe = 0; probe < cap; ++probe, i = next_slot(i, cap)) {
    const Slot3* s = static_cast<const Slot3*>(v.table) + i;
    const unsigned long long cur = __ldcg(&s->ref);
    if (cur == 0) return -1;
    if ((cur >> 49) == tag && ref_holds(v, cur, key)) return (int)__ldcg(&s->mask);
  }
  return -1;
}

// The table slot of an occurrence at g (inserted), or its mask (found).
template <int KW, int TS>
__device__ __forceinline__ uint64_t insert_occurrence(const RunView& v, uint64_t cap, const OccT<KW>& oc,
                                                      uint64_t g) {
  if constexpr (TS == 3) return table_insert_ref(v, cap, oc.key, oc.H, oc.tbits, g, oc.rc);
  else return table_insert<TS>(v, cap, oc.key, slot_start(oc.H, cap), oc.tbits);
}

template <int KW, int TS>
__device__ __forceinline__ int find_occurrence(const RunView& v, uint64_t cap, const OccT<KW>& oc) {
  if constexpr (TS == 3) return table_find_ref(v, cap, oc.key, oc.H);
  else return table_find<TS>(v, cap, oc.key, slot_start(oc.H, cap));
}

// Mask held by slot i (a slot that table_insert returned).
template <int TS>
__device__ __forceinline__ int table_mask(const RunView& v, uint64_t i) {
  if (TS == 0) return (int)(__ldcg(static_cast<const unsigned long long*>(v.table) + i) & ((1u << kMaskBits) - 1u));
  if (TS == 1) return (int)__ldcg(&(static_cast<const Slot1*>(v.table) + i)->mask);
  if (TS == 3) return (int)__ldcg(&(static_cast<const Slot3*>(v.table) + i)->mask);
  return (int)__ldcg(&(static_cast<const Slot2*>(v.table) + i)->mask);
}

__device__ __forceinline__ bool is_junction_mask(int mk) {
  return ((mk >> 8) & 1) || __popc(mk & 15) > 1 || __popc((mk >> 4) & 15) > 1;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Exclusive scan of x over the block (blockDim.x == kBlock); *total gets the sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* total) {
  __shared__ uint32_t warp_tot[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kBlock / 32; ++w) {
    const uint32_t t = warp_tot[w];
    before += (w < wid) ? t : 0u;
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + inc - x;
}

// Sum a counter over the block's threads into *dst (one atomic per block).
__device__ __forceinline__ void block_add(unsigned long long x, unsigned long long* dst) {
  __shared__ unsigned long long part[kBlock / 32];
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kBlock / 32; ++w) t += part[w];
    if (t) atomicAdd(dst, t);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Four ASCII bytes -> four 2-bit codes (first byte in bits 7-6); *bad gets
// 0xFF in every byte that is not one of ACGTacgt.
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t* bad, uint32_t* is_n) {
  const uint32_t low = x | 0x20202020u;
  const uint32_t ok = __vcmpeq4(low, 0x61616161u) | __vcmpeq4(low, 0x63636363u) |
                      __vcmpeq4(low, 0x67676767u) | __vcmpeq4(low, 0x74747474u);
  *bad = ~ok;
  *is_n = __vcmpeq4(low, 0x6e6e6e6eu);
  // a=0x61 c=0x63 g=0x67 t=0x74: bits 2-1 are 00 01 11 10; fold to 0 1 2 3
  const uint32_t t = (low >> 1) & 0x03030303u;
  const uint32_t c = t ^ ((t >> 1) & 0x01010101u);
  return ((c & 3u) << 6) | (((c >> 8) & 3u) << 4) | (((c >> 16) & 3u) << 2) | ((c >> 24) & 3u);
}

// Bit j of the result: the top bit of byte j of e (for a __vcmpeq4 mask:
// byte j matched).
__device__ __forceinline__ uint32_t byte_bits(uint32_t e) {
  // the top bit of every byte to bits 0-3: the multiply moves bits 7, 15, 23
  // and 31 to bits 28-31, every other partial product lands elsewhere
  return ((e & 0x80808080u) * 0x00204081u) >> 28;
}

// Sixteen ASCII bytes at g (or fewer at the end of the input) -> one word;
// *bad_at gets the index of the first invalid byte. With N splitting (v.nmask)
// an N is valid and *nbits gets bit i for an N at g + i.
__device__ __forceinline__ uint32_t pack16(const RunView& v, uint64_t g, uint4 q, bool full,
                                           uint64_t* bad_at, uint32_t* nbits) {
  uint32_t out = 0, nb = 0;
  const bool split = v.nmask != nullptr;
  if (full) {
    const uint32_t part[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t bad, is_n;
      out |= pack4(part[c], &bad, &is_n) << (24 - 8 * c);
      if (split) {
        bad &= ~is_n;
        nb |= byte_bits(is_n) << (4 * c);
      }
      if (bad && *bad_at == ~0ull) *bad_at = g + 4 * c + (__ffs(bad) - 1) / 8;
    }
  } else if (g < v.m) {
    for (int i = 0; i < 16 && g + i < v.m; ++i) {
      const uint32_t c = v.bases[g + i];
      uint32_t bad, is_n;
      const uint32_t code = pack4(c | 0x61616100u, &bad, &is_n) >> 6;  // pad bytes are 'a'
      if (split && (is_n & 0xFFu)) {
        bad = 0;
        nb |= 1u << i;
      }
      if ((bad & 0xFFu) && *bad_at == ~0ull) *bad_at = g + i;
      out |= code << (30 - 2 * i);
    }
  }
  *nbits = nb;
  return out;
}

// ASCII -> 2-bit words: 64 bytes (four 128-bit loads in flight) per thread,
// for the packed words [w_begin, w_end) (w_begin a multiple of 4; the input
// bytes of those words are read at v.bases + 16 * w, so that a chunk of the
// input staged elsewhere can be packed by passing v.bases offset back by the
// chunk's start). With `first`, block 0 also records where this run keeps its
// bitmaps (for inspection), and the grid clears the filter, the
// linear-counting bitmap, C_final and the emit's tile status for the first
// round.
__global__ void __launch_bounds__(kBlock) pack_kernel(RunView v, uint64_t w_begin, uint64_t w_end, int first) {
  if (first && blockIdx.x == 0 && threadIdx.x == 0) {
    DevHeader* h = v.hdr;
    h->ctemp = v.ctemp;
    h->cfinal = v.cfinal;
    h->bins = v.bins;
    h->cuts = v.cuts;
    h->bitmap_words = v.bitmap_words;
    h->q = (unsigned long long)v.qmask + 1ull;
    h->rounds = (unsigned long long)v.rounds;
    h->packed = v.packed;
    h->m = v.m;
    h->k = v.k;
    h->both = v.both;
    h->nmask = v.nmask;
    h->runs = v.runs;
    h->run_rank = v.run_rank;
    h->run_cap = v.run_cap;
    h->offsets = v.offsets;
    h->n_seqs = v.n_seqs;
    h->hashes = v.hashes;
    h->lg_blocks = v.lg_blocks;
    h->partial = v.partial;
    h->packed_words = v.packed_words;
  }
  const bool vec = (reinterpret_cast<uintptr_t>(v.bases) & 15) == 0;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * 4;
  uint64_t bad_at = ~0ull;
  for (uint64_t w0 = w_begin + ((uint64_t)blockIdx.x * kBlock + threadIdx.x) * 4; w0 < w_end; w0 += stride) {
    uint4 q[4];
    bool full[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t g = (w0 + j) * 16;
      full[j] = vec && g + 16 <= v.m;
      if (full[j]) q[j] = __ldcs(reinterpret_cast<const uint4*>(v.bases + g));
    }
    uint32_t out[4], nb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = pack16(v, (w0 + j) * 16, q[j], full[j], &bad_at, &nb[j]);
    if (v.nmask) {  // two packed words per N-mask word (w0 is a multiple of 4)
      v.nmask[w0 / 2] = nb[0] | (nb[1] << 16);
      v.nmask[w0 / 2 + 1] = nb[2] | (nb[3] << 16);
    }
    if (w0 + 4 <= w_end) {
      *reinterpret_cast<uint4*>(v.packed + w0) = make_uint4(out[0], out[1], out[2], out[3]);
    } else {
      for (int j = 0; j < 4 && w0 + j < w_end; ++j) v.packed[w0 + j] = out[j];
    }
  }
  if (bad_at != ~0ull) atomicMax(&v.hdr->bad_inv, ~(unsigned long long)bad_at);
  if (!first) return;
  // clear what the first round and the emit need to start at zero
  const uint64_t tid = (uint64_t)blockIdx.x * kBlock + threadIdx.x, nthreads = (uint64_t)gridDim.x * kBlock;
  auto zero = [&](void* p, uint64_t bytes) {  // 16-byte multiples at 16-byte aligned addresses
    uint4* q = static_cast<uint4*>(p);
    for (uint64_t i = tid; i < bytes / 16; i += nthreads) q[i] = make_uint4(0u, 0u, 0u, 0u);
  };
  zero(v.filter, v.filter_words64 * 8);
  zero(v.lc_bits, (1ull << v.lc_log2) / 8);
  zero(v.cfinal, (v.bitmap_words + 3) / 4 * 16);
  zero(v.tile_prefix, (v.n_tiles + 1) / 2 * 16);
}

// Digest of the input (checkpoints record it and check it on resume): the
// packed words, the string offsets and the N mask, each term tagged with its
// kind and index.
__global__ void __launch_bounds__(kBlock) digest_kernel(DevHeader* hdr, const uint32_t* packed, uint64_t words,
                                                        const uint64_t* offsets, uint64_t n_off,
                                                        const uint32_t* nmask, uint64_t nmask_words) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  const uint64_t tid = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  unsigned long long d = 0;
  for (uint64_t w = tid; w < words; w += stride) d += mix64((w << 32) ^ packed[w]);
  for (uint64_t t = tid; t < n_off; t += stride) d += mix64(mix64(t ^ 0x6f66667365747321ull) ^ offsets[t]);
  if (nmask)
    for (uint64_t w = tid; w < nmask_words; w += stride) d += mix64(mix64(w ^ 0x6e6d61736b212121ull) ^ nmask[w]);
  block_add(d, &hdr->input_digest);
}

// ---------------------------------------------------------------------------
// N splitting: the sorted boundaries of the N-free pieces and of the N runs.
// Bit g of the boundary bitmap is set iff g starts a string or base g is N
// and base g - 1 is not, or the other way round, inside one string. The set
// bits, in order, are runs[0 .. n_runs); runs[n_runs] = m.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock) runs_mark_kernel(RunView v) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t w = (uint64_t)blockIdx.x * kBlock + threadIdx.x; w < v.bitmap_words; w += stride) {
    const uint32_t cur = v.nmask[w], prev = w ? v.nmask[w - 1] : 0u;
    uint32_t b = cur ^ ((cur << 1) | (prev >> 31));
    if (w == v.bitmap_words - 1 && (v.m & 31)) b &= (1u << (v.m & 31)) - 1u;
    v.bound_bits[w] = b;
  }
}

__global__ void __launch_bounds__(kBlock) runs_starts_kernel(RunView v) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t t = (uint64_t)blockIdx.x * kBlock + threadIdx.x; t < v.n_seqs; t += stride) {
    const uint64_t g = __ldg(v.offsets + t);
    if (g < v.m) atomicOr(v.bound_bits + (g >> 5), 1u << (g & 31));
  }
}

// Set bits of every chunk of kRunChunkWords boundary words.
__global__ void __launch_bounds__(kBlock) runs_count_kernel(RunView v) {
  __shared__ unsigned long long part[kBlock / 32];
  for (uint64_t c = blockIdx.x; c < v.n_chunks; c += gridDim.x) {
    unsigned long long n = 0;
    for (uint64_t w = c * kRunChunkWords + threadIdx.x; w < (c + 1) * kRunChunkWords && w < v.bitmap_words;
         w += kBlock)
      n += __popc(v.bound_bits[w]);
    n = warp_sum(n);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
      for (int i = 0; i < kBlock / 32; ++i) tot += part[i];
      v.chunk_counts[c] = tot;
    }
    __syncthreads();
  }
}

// Exclusive scan of the chunk counts (in place, one block); records the
// number of boundaries (at most run_cap, else the overflow flag) and closes
// the list with m.
__global__ void __launch_bounds__(1024) runs_scan_kernel(RunView v) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t base = 0; base < v.n_chunks; base += 1024) {
    const uint64_t c = base + threadIdx.x;
    const unsigned long long x = c < v.n_chunks ? v.chunk_counts[c] : 0ull;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      before += (w < wid) ? wsum[w] : 0ull;
      all += wsum[w];
    }
    const unsigned long long c0 = carry_s;
    if (c < v.n_chunks) v.chunk_counts[c] = c0 + before + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = c0 + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = carry_s;
    const unsigned long long n = total < v.run_cap ? total : v.run_cap;
    if (total > v.run_cap) v.hdr->overflow = 1;
    v.hdr->n_runs = n;
    v.runs[n] = v.m;
  }
}

// Positions of the set boundary bits, in order (chunk by chunk).
__global__ void __launch_bounds__(kBlock) runs_write_kernel(RunView v) {
  constexpr int kPer = (int)(kRunChunkWords / kBlock);  // consecutive words per thread
  for (uint64_t c = blockIdx.x; c < v.n_chunks; c += gridDim.x) {
    const uint64_t w0 = c * kRunChunkWords + (uint64_t)threadIdx.x * kPer;
    uint32_t words[kPer];
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      words[j] = (w0 + j < v.bitmap_words) ? v.bound_bits[w0 + j] : 0u;
      n += __popc(words[j]);
    }
    uint32_t tot;
    uint64_t at = v.chunk_counts[c] + block_exclusive_scan(n, &tot);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      uint32_t bits = words[j];
      while (bits) {
        const uint32_t b = __ffs(bits) - 1;
        bits &= bits - 1;
        if (at < v.run_cap) v.runs[at] = (w0 + j) * 32 + b;
        ++at;
      }
    }
  }
}

// Probe descriptor of a position (64 bits): bit 63 active (probe it), bit 62
// sentinel position, bits 32-61 the bit bases of its k-mer (G >> 32, bases
// of u < 6), bits 0-31 its filter word index. 1 marks a position whose
// k-mer is in another round's class, 0 a position without a k-mer.
constexpr uint64_t kDescActive = 1ull << 63, kDescSentinel = 1ull << 62;

__device__ __forceinline__ uint64_t make_desc(const RunView& v, uint64_t H, uint64_t G, bool sentinel) {
  const uint64_t block = v.lg_blocks ? (H >> (64 - v.lg_blocks)) : 0ull;
  const uint64_t index = block * 4 + (G >> 62);  // < 2^32 for b <= 2^37
  return kDescActive | (sentinel ? kDescSentinel : 0ull) | (((G >> 32) & 0x3FFFFFFFull) << 32) | index;
}

// Algorithm 1, insert loop, first pass: every active position records its
// item(s) in its k-mer's filter word with one atomic OR. With DESC it also
// leaves the position's probe descriptor for the probe loop: the block's
// descriptors are staged in shared memory (16-byte pairs, columns swizzled by
// the owning thread so that neither side conflicts) and written out in
// order, whole sectors at a time.
template <int KW, bool ROUNDS, int HB, bool DESC, bool BKT = false>
__global__ void __launch_bounds__(kBlock) pass1_insert_kernel(RunView v, int round) {
  constexpr int kTile = kBlock * kInsertR;  // positions per block per pass
  constexpr int kPairs = kInsertR / 2;      // 16-byte descriptor pairs per thread
  __shared__ ulonglong2 stage[DESC ? kTile / 2 : 1];
  const uint64_t stride = (uint64_t)gridDim.x * kTile;
  const int t = threadIdx.x;
  for (uint64_t base = v.p_begin + (uint64_t)blockIdx.x * kTile; base < v.p_end; base += stride) {
    const uint64_t p0 = base + (uint64_t)t * kInsertR;
    if (p0 < v.m) {
      uint64_t prev = 0;
      walk<KW, kInsertR>(v, p0, [&](int i, uint64_t, bool valid, const auto& oc) {
        uint64_t d = 0;
        if (valid) {
          if (ROUNDS && !in_round(v, oc.H, round)) {
            d = 1;
          } else {
            const uint64_t G = second_hash(oc.H);
            const ItemPattern pat = item_pattern<HB>(G, v.hashes);
            const uint32_t j1 = __ffs(oc.items) - 1, j2 = 31 - __clz(oc.items);
            uint64_t m = item_bits(pat, j1);
            if (j2 != j1) m |= item_bits(pat, j2);  // a palindrome's two orientations
            if (BKT) stage_or(v, filter_index(v, oc.H, G), G, j1, j2, m);
            else atomicOr(filter_word(v, oc.H, G), (unsigned long long)m);
            if (DESC) d = make_desc(v, oc.H, G, oc.sentinel);
          }
        }
        if (DESC) {
          if (i & 1) stage[t * kPairs + ((i >> 1) ^ (t % kPairs))] = make_ulonglong2(prev, d);
          else prev = d;
        }
      });
    }
    if (DESC) {
      __syncthreads();
      // pair j covers positions base + 2j, base + 2j + 1; its owner is thread
      // j / kPairs (which wrote 0 for any of them past m). The region holds
      // m + 16 descriptors, so a pair that starts before m fits.
      for (int j = t; j < kTile / 2; j += kBlock) {
        const uint64_t p = base + 2 * (uint64_t)j;
        if (p >= v.m) break;
        const int owner = j / kPairs, c = j % kPairs;
        __stcs(reinterpret_cast<ulonglong2*>(v.desc + p), stage[owner * kPairs + (c ^ (owner % kPairs))]);
      }
      __syncthreads();
    }
  }
}

// Algorithm 1, probe loop, first pass: a position stays a candidate iff it is
// a sentinel position, its k-mer's sentinel item is present, or at least two
// of its 16 (predecessor, successor) items are present -- i.e. the filter
// does not show exactly one in-edge and one out-edge. Writes C_temp, appends
// every candidate's position to the warp's own segment of the pass-2 list,
// and sets the candidate's bit in a linear-counting bitmap that estimates how
// many distinct k-mers survive.
template <int KW, bool ROUNDS, int HB>
__global__ void __launch_bounds__(kBlock, 3) pass1_probe_kernel(RunView v, int round) {
  const int lane = threadIdx.x & 31;
  constexpr int kR = kProbeR;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * kR;
  constexpr int kLanesPerWord = 32 / kR;
  unsigned long long kept = 0, valid_n = 0;
  const uint32_t warp_id = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  uint64_t* seg = v.cands + (uint64_t)warp_id * v.seg_cap;  // wide records
  uint32_t* seg32 = reinterpret_cast<uint32_t*>(v.cands) + (uint64_t)warp_id * v.seg_cap;
  uint64_t seg_used = 0;
  for (uint64_t wbase = v.p_begin + ((uint64_t)blockIdx.x * kBlock + (threadIdx.x & ~31u)) * kR;
       wbase < v.p_end; wbase += stride) {
    const uint64_t p0 = wbase + (uint64_t)lane * kR;
    uint64_t word[kR], G[kR];
    uint32_t probe_bits = 0, sent_bits = 0, valid_bits = 0;
    if (p0 < v.m) {
      walk<KW, kR>(v, p0, [&](int i, uint64_t, bool valid, const auto& oc) {
        if (!valid) return;
        valid_bits |= 1u << i;
        if (ROUNDS && !in_round(v, oc.H, round)) return;
        G[i] = second_hash(oc.H);
        if (oc.sentinel) {
          sent_bits |= 1u << i;
        } else {
          word[i] = __ldcg(filter_word(v, oc.H, G[i]));
          probe_bits |= 1u << i;
        }
      });
    }
    uint32_t keep_bits = sent_bits;
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      if ((probe_bits >> i) & 1u) {
        const uint32_t pres = present_items<HB>(G[i], word[i], v.hashes);
        if ((pres >> 16) || __popc(pres & 0xFFFFu) >= 2) keep_bits |= 1u << i;
      }
      if (((keep_bits >> i) & 1u) && !v.partial) {
        const uint64_t idx = (G[i] * 0xff51afd7ed558ccdull) >> (64 - v.lc_log2);
        atomicOr(v.lc_bits + (idx >> 5), 1u << (idx & 31));
      }
    }
    // C_temp: kLanesPerWord lanes make up one 32-bit word
    uint32_t wv = keep_bits << (kR * (lane % kLanesPerWord));
#pragma unroll
    for (int o = 1; o < kLanesPerWord; o <<= 1) wv |= __shfl_xor_sync(0xffffffffu, wv, o);
    if (lane % kLanesPerWord == 0) {
      const uint64_t w = (wbase >> 5) + lane / kLanesPerWord;
      if (w < v.bitmap_words) {
        v.ctemp[w] = wv;
        if (v.partial) v.cfinal[w] |= wv;  // rounds own disjoint positions; one writer per word
      }
    }
    if (v.partial) {
      kept += __popc(keep_bits);
      valid_n += __popc(valid_bits);
      continue;
    }
    // candidate list: the warp appends to its own segment, in position order
    const uint32_t c = __popc(keep_bits);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    uint64_t at = seg_used + (inc - c);
    uint32_t bits = keep_bits;
    while (bits) {
      const int i = __ffs(bits) - 1;
      bits &= bits - 1;
      if (at < v.seg_cap) {
        const uint64_t sent = (sent_bits >> i) & 1u;  // a string's first or last k-mer
        if (v.narrow) seg32[at] = (uint32_t)(p0 + (uint64_t)i) | ((uint32_t)sent << 31);
        else seg[at] = (p0 + (uint64_t)i) | (sent << 63);
      }
      ++at;
    }
    seg_used += __shfl_sync(0xffffffffu, inc, 31);
    kept += c;
    valid_n += __popc(valid_bits);
  }
  if (lane == 0) {
    v.seg_count[warp_id] = (uint32_t)(seg_used < v.seg_cap ? seg_used : v.seg_cap);
    if (seg_used > v.seg_cap) v.hdr->cand_overflow = 1;
  }
  block_add(kept, &v.hdr->pass1_kept);
  block_add(kept, v.partial ? &v.hdr->pass2_kept : &v.hdr->round_kept);
  if (round == v.count_round) block_add(valid_n, &v.hdr->positions);
}

// The probe loop from descriptors (same decisions and outputs as
// pass1_probe_kernel). A warp takes kProbeR rows of 32 consecutive
// positions; lane l reads the descriptor of position row + l (one coalesced
// 256-byte load per row), loads the filter words of its active non-sentinel
// positions, then decides. A row's ballot is its C_temp word, and its kept
// positions go to the warp's list segment in order.
template <int HB>
__global__ void __launch_bounds__(kBlock) pass1_probe_desc_kernel(RunView v, int round) {
  static_assert(HB <= 6, "descriptors carry the bases of six bits");
  constexpr int kRows = 4;  // rows of 32 positions per warp and step (4 measured faster than 8 or 16)
  static_assert(kRows <= 32, "one C_temp word per lane");
  const int lane = threadIdx.x & 31;
  const uint32_t below = (1u << lane) - 1u;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * kRows;
  unsigned long long kept = 0, valid_n = 0;
  const uint32_t warp_id = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  uint64_t* seg = v.cands + (uint64_t)warp_id * v.seg_cap;
  uint32_t* seg32 = reinterpret_cast<uint32_t*>(v.cands) + (uint64_t)warp_id * v.seg_cap;
  uint64_t seg_used = 0;
  // the descriptors of a step are loaded one step ahead (kProbePrefetch), so
  // that their stream overlaps the previous step's filter loads
  uint64_t dn[kRows];
  const uint64_t wfirst = v.p_begin + ((uint64_t)blockIdx.x * kBlock + (threadIdx.x & ~31u)) * kRows;
  if (kProbePrefetch) {
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const uint64_t p = wfirst + 32 * q + lane;
      dn[q] = p < v.m ? __ldcs(v.desc + p) : 0ull;
    }
  }
  for (uint64_t wbase = wfirst; wbase < v.p_end; wbase += stride) {
    uint64_t d[kRows], word[kRows];
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const uint64_t p = wbase + 32 * q + lane;
      if (kProbePrefetch) d[q] = dn[q];
      else d[q] = p < v.m ? __ldcs(v.desc + p) : 0ull;
    }
#pragma unroll
    for (int q = 0; q < kRows; ++q)
      if ((d[q] & (kDescActive | kDescSentinel)) == kDescActive) word[q] = __ldcg(v.filter + (uint32_t)d[q]);
    if (kProbePrefetch) {
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const uint64_t p = wbase + stride + 32 * q + lane;
        dn[q] = p < v.m ? __ldcs(v.desc + p) : 0ull;
      }
    }
    uint32_t my_word = 0;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      bool keep = false;
      if (d[q] & kDescActive) {
        if (d[q] & kDescSentinel) {
          keep = true;
        } else {
          // descriptor bits 32-61 are G's, the only bits bit_base reads for u < 6
          const uint32_t pres = present_items<HB>(d[q], word[q], v.hashes);
          keep = (pres >> 16) || __popc(pres & 0xFFFFu) >= 2;
        }
      }
      valid_n += d[q] != 0;
      const uint32_t row = __ballot_sync(0xffffffffu, keep);
      if (lane == q) my_word = row;
      if (v.partial) {
        kept += keep;
        continue;
      }
      if (keep) {
        const uint64_t idx = ((d[q] & ~(kDescActive | kDescSentinel)) * 0xff51afd7ed558ccdull) >> (64 - v.lc_log2);
        atomicOr(v.lc_bits + (idx >> 5), 1u << (idx & 31));
        const uint64_t at = seg_used + __popc(row & below);
        if (at < v.seg_cap) {
          const uint64_t p = wbase + 32 * q + lane;
          const uint64_t sent = (d[q] >> 62) & 1u;
          if (v.narrow) seg32[at] = (uint32_t)p | ((uint32_t)sent << 31);
          else seg[at] = p | (sent << 63);
        }
        ++kept;
      }
      seg_used += __popc(row);
    }
    if (lane < kRows) {
      const uint64_t w = (wbase >> 5) + lane;
      if (w < v.bitmap_words) {
        v.ctemp[w] = my_word;
        if (v.partial) v.cfinal[w] |= my_word;  // rounds own disjoint positions; one writer per word
      }
    }
  }
  if (lane == 0) {
    v.seg_count[warp_id] = (uint32_t)(seg_used < v.seg_cap ? seg_used : v.seg_cap);
    if (seg_used > v.seg_cap) v.hdr->cand_overflow = 1;
  }
  block_add(kept, &v.hdr->pass1_kept);
  block_add(kept, v.partial ? &v.hdr->pass2_kept : &v.hdr->round_kept);
  if (round == v.count_round) block_add(valid_n, &v.hdr->positions);
}

// ---------------------------------------------------------------------------
// Class map (rounds > 1, at most kMaxMapRounds of them): Algorithm 3 marks,
// in round i, the positions whose k-mer is in class i. Instead of walking and
// hashing every position again in every round, one pass after the class cut
// records per position one byte -- bit 7: no k-mer starts here, bit 6: a
// sentinel position (the first or last k-mer of its string or N-free piece),
// bits 0-5: the class -- and each round's two first-pass loops then visit only
// the positions of their class, reading each k-mer from scratch. A warp takes
// a window of 512 consecutive positions, compacts the indices of the active
// ones in shared memory and shares them out evenly over its lanes.
// ---------------------------------------------------------------------------

constexpr uint32_t kCmNone = 0x80u, kCmSentinel = 0x40u, kCmClass = 0x3Fu;
constexpr int kCmWindow = 32 * 16;  // positions per warp window

// Class of a bin: the r with cuts[r] <= bin < cuts[r + 1] (cuts in shared memory).
__device__ __forceinline__ uint32_t class_of_bin(const uint32_t* cuts, int rounds, uint32_t bin) {
  int lo = 0, hi = rounds;  // cuts[lo] <= bin < cuts[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cuts[mid] <= bin) lo = mid; else hi = mid;
  }
  return (uint32_t)lo;
}

// Filter region of a k-mer's word (region-ordered first pass).
__device__ __forceinline__ uint32_t ord_region(const RunView& v, uint64_t H, uint64_t G) {
  return (uint32_t)(filter_index(v, H, G) >> v.o_lg_region_words);
}

template <int KW>
__global__ void __launch_bounds__(kBlock) class_map_kernel(RunView v) {
  __shared__ uint32_t cuts_s[kMaxMapRounds + 1];
  for (int i = threadIdx.x; i <= v.rounds; i += kBlock) cuts_s[i] = v.cuts[i];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * kInsertR;
  for (uint64_t p0 = ((uint64_t)blockIdx.x * kBlock + threadIdx.x) * kInsertR; p0 < v.m; p0 += stride) {
    uint32_t w[4] = {0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u};
    walk<KW, kInsertR>(v, p0, [&](int i, uint64_t, bool valid, const auto& oc) {
      if (!valid) return;
      const uint32_t c = class_of_bin(cuts_s, v.rounds, (uint32_t)oc.H & v.qmask) |
                         (oc.sentinel ? kCmSentinel : 0u);
      w[i >> 2] = (w[i >> 2] & ~(0xFFu << (8 * (i & 3)))) | (c << (8 * (i & 3)));
    });
    *reinterpret_cast<uint4*>(v.cmap + p0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// The class map of a run with the region-ordered first pass, a tile of
// kOrdTile positions per block: also the region plane (the filter region of
// every position's k-mer) and, per tile, its positions of every (class,
// region) pair (o_thist, tile-major) and of every (class, warp chunk of
// kOrdTile / 8 positions) (o_wcount, class-major) and of every class
// (o_tcount, class-major).
template <int KW>
__global__ void __launch_bounds__(kBlock) class_map_ord_kernel(RunView v) {
  constexpr int kChunks = (int)(kOrdTile / ((uint64_t)kBlock * kInsertR));  // 4
  constexpr int kWarpChunks = kBlock / 32;                                   // 8
  __shared__ uint32_t cuts_s[kMaxMapRounds + 1];
  __shared__ uint32_t thist_s[kOrdMaxHist];
  __shared__ uint32_t wcnt_s[kWarpChunks * kMaxMapRounds];
  for (int i = threadIdx.x; i <= v.rounds; i += kBlock) cuts_s[i] = v.cuts[i];
  const uint32_t R = v.o_regions, L = (uint32_t)v.rounds, nh = L * R;
  for (uint64_t t = blockIdx.x; t < v.o_tiles; t += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < nh; i += kBlock) thist_s[i] = 0;
    for (uint32_t i = threadIdx.x; i < kWarpChunks * L; i += kBlock) wcnt_s[i] = 0;
    __syncthreads();
    for (int c = 0; c < kChunks; ++c) {
      const uint64_t p0 = t * kOrdTile + ((uint64_t)c * kBlock + threadIdx.x) * kInsertR;
      if (p0 >= v.m) break;
      // the warp chunk of these positions: kOrdTile / 8 = 2048 positions, 128 threads' worth
      const uint32_t wc = (uint32_t)((((uint64_t)c * kBlock + threadIdx.x) * kInsertR) / (kOrdTile / kWarpChunks));
      uint32_t w[4] = {0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u};
      uint32_t r[4] = {0u, 0u, 0u, 0u};
      walk<KW, kInsertR>(v, p0, [&](int i, uint64_t, bool valid, const auto& oc) {
        if (!valid) return;
        const uint32_t cls = class_of_bin(cuts_s, v.rounds, (uint32_t)oc.H & v.qmask);
        w[i >> 2] = (w[i >> 2] & ~(0xFFu << (8 * (i & 3)))) | ((cls | (oc.sentinel ? kCmSentinel : 0u)) << (8 * (i & 3)));
        const uint32_t reg = ord_region(v, oc.H, second_hash(oc.H));
        r[i >> 2] |= reg << (8 * (i & 3));
        atomicAdd(thist_s + cls * R + reg, 1u);
        atomicAdd(wcnt_s + wc * L + cls, 1u);
      });
      *reinterpret_cast<uint4*>(v.cmap + p0) = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(v.rplane + p0) = make_uint4(r[0], r[1], r[2], r[3]);
    }
    __syncthreads();
    // at most kOrdTile = 16384 positions per tile: every count fits 16 bits
    uint16_t* th = v.o_thist + t * nh;
    for (uint32_t i = threadIdx.x; i < nh; i += kBlock) th[i] = (uint16_t)thist_s[i];
    for (uint32_t i = threadIdx.x; i < kWarpChunks * L; i += kBlock) {
      const uint32_t cls = i % L, wc = i / L;
      v.o_wcount[((uint64_t)cls * v.o_tiles + t) * kWarpChunks + wc] = (uint16_t)wcnt_s[i];
    }
    for (uint32_t cls = threadIdx.x; cls < L; cls += kBlock) {
      uint32_t tot = 0;
      for (int wc = 0; wc < kWarpChunks; ++wc) tot += wcnt_s[wc * L + cls];
      v.o_tcount[(uint64_t)cls * v.o_tiles + t] = tot;
    }
    __syncthreads();
  }
}

// The positions of this round's class in the warp's window [wbase, wbase + 512):
// their offsets (bits 0-8) with the sentinel flag (bit 9) go to idx[0 .. n), in
// position order; *valid gets the number of positions with a k-mer.
__device__ __forceinline__ uint32_t compact_window(const RunView& v, uint64_t wbase, int round, uint16_t* idx,
                                                   uint32_t* valid) {
  const int lane = threadIdx.x & 31;
  const uint64_t p0 = wbase + 16 * (uint64_t)lane;
  uint4 q = make_uint4(0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u);
  if (p0 < v.m) q = __ldcs(reinterpret_cast<const uint4*>(v.cmap + p0));
  const uint32_t part[4] = {q.x, q.y, q.z, q.w};
  const uint32_t want = (uint32_t)round * 0x01010101u;
  uint32_t act = 0, sent = 0, val = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    act |= byte_bits(__vcmpeq4(part[c] & 0xBFBFBFBFu, want)) << (4 * c);  // valid and in this class
    sent |= byte_bits(part[c] << 1) << (4 * c);  // bit 6: a sentinel
    val |= byte_bits(~part[c]) << (4 * c);       // bit 7 clear: a k-mer
  }
  const uint32_t n = __popc(act);
  uint32_t inc = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  uint32_t at = inc - n;
  while (act) {
    const uint32_t i = __ffs(act) - 1;
    act &= act - 1;
    idx[at++] = (uint16_t)((16 * lane + i) | (((sent >> i) & 1u) << 9));
  }
  *valid = __popc(val);
  __syncwarp();
  return __shfl_sync(0xffffffffu, inc, 31);
}

// The region-ordered kernels take the current round (its records fit).
__device__ __forceinline__ bool ordered_round(const RunView& v) {
  return v.o_regions && *reinterpret_cast<volatile const unsigned int*>(&v.hdr->ord_ok);
}

// Algorithm 1, insert loop, first pass, over this round's class only.
template <int KW, int HB, bool BKT = false>
__global__ void __launch_bounds__(kBlock) pass1_insert_cm_kernel(RunView v, int round) {
  __shared__ uint16_t idx_s[kBlock / 32][kCmWindow];
  if (ordered_round(v)) return;  // the region-ordered kernels take this round
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint16_t* idx = idx_s[wid];
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * 16;
  for (uint64_t wbase = v.p_begin + ((uint64_t)blockIdx.x * kBlock + (threadIdx.x & ~31u)) * 16; wbase < v.p_end;
       wbase += stride) {
    uint32_t valid;
    const uint32_t n = compact_window(v, wbase, round, idx, &valid);
    for (uint32_t j = lane; j < n; j += 32) {
      const uint32_t e = idx[j];
      OccT<KW> oc;
      read_listed<KW>(v, wbase + (e & 511u), (e >> 9) & 1u, &oc);
      const uint64_t G = second_hash(oc.H);
      const ItemPattern pat = item_pattern<HB>(G, v.hashes);
      const uint32_t j1 = __ffs(oc.items) - 1, j2 = 31 - __clz(oc.items);
      uint64_t m = item_bits(pat, j1);
      if (j2 != j1) m |= item_bits(pat, j2);  // a palindrome's two orientations
      if (BKT) stage_or(v, filter_index(v, oc.H, G), G, j1, j2, m);
      else atomicOr(filter_word(v, oc.H, G), (unsigned long long)m);
    }
    __syncwarp();
  }
}

// Algorithm 1, probe loop, first pass, over this round's class only: the same
// decisions and outputs as pass1_probe_kernel (C_temp words of the window, the
// candidate list segment of the warp, the linear-counting bits).
template <int KW, int HB>
__global__ void __launch_bounds__(kBlock) pass1_probe_cm_kernel(RunView v, int round) {
  __shared__ uint16_t idx_s[kBlock / 32][kCmWindow];
  __shared__ uint32_t keep_s[kBlock / 32][kCmWindow / 32];
  if (ordered_round(v)) return;  // the region-ordered kernels take this round
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint16_t* idx = idx_s[wid];
  uint32_t* keep_w = keep_s[wid];
  const uint32_t below = (1u << lane) - 1u;
  unsigned long long kept = 0, valid_n = 0;
  const uint32_t warp_id = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  uint64_t* seg = v.cands + (uint64_t)warp_id * v.seg_cap;
  uint32_t* seg32 = reinterpret_cast<uint32_t*>(v.cands) + (uint64_t)warp_id * v.seg_cap;
  uint64_t seg_used = 0;
  if (lane < kCmWindow / 32) keep_w[lane] = 0;
  __syncwarp();
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * 16;
  for (uint64_t wbase = v.p_begin + ((uint64_t)blockIdx.x * kBlock + (threadIdx.x & ~31u)) * 16; wbase < v.p_end;
       wbase += stride) {
    uint32_t valid;
    const uint32_t n = compact_window(v, wbase, round, idx, &valid);
    valid_n += valid;
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
      const uint32_t j = j0 + lane;
      bool keep = false;
      uint64_t G = 0, g = 0;
      uint32_t sentinel = 0;
      if (j < n) {
        const uint32_t e = idx[j];
        g = wbase + (e & 511u);
        sentinel = (e >> 9) & 1u;
        if (sentinel) {
          keep = true;
          OccT<KW> oc;
          read_listed<KW>(v, g, true, &oc);
          G = second_hash(oc.H);
        } else {
          OccT<KW> oc;
          read_listed<KW>(v, g, false, &oc);
          G = second_hash(oc.H);
          const uint64_t word = __ldcg(filter_word(v, oc.H, G));
          const uint32_t pres = present_items<HB>(G, word, v.hashes);
          keep = (pres >> 16) || __popc(pres & 0xFFFFu) >= 2;
        }
        if (keep) atomicOr(keep_w + ((e & 511u) >> 5), 1u << (e & 31u));
      }
      if (v.partial) {
        kept += keep;
        continue;
      }
      const uint32_t row = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const uint64_t x = (G * 0xff51afd7ed558ccdull) >> (64 - v.lc_log2);
        atomicOr(v.lc_bits + (x >> 5), 1u << (x & 31));
        const uint64_t at = seg_used + __popc(row & below);
        if (at < v.seg_cap) {
          if (v.narrow) seg32[at] = (uint32_t)g | (sentinel << 31);
          else seg[at] = g | ((uint64_t)sentinel << 63);
        }
        ++kept;
      }
      seg_used += __popc(row);
    }
    __syncwarp();
    if (lane < kCmWindow / 32) {
      const uint64_t w = (wbase >> 5) + lane;
      const uint32_t word = keep_w[lane];
      keep_w[lane] = 0;
      if (w < v.bitmap_words) {
        v.ctemp[w] = word;
        if (v.partial) v.cfinal[w] |= word;  // rounds own disjoint positions; one writer per word
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    v.seg_count[warp_id] = (uint32_t)(seg_used < v.seg_cap ? seg_used : v.seg_cap);
    if (seg_used > v.seg_cap) v.hdr->cand_overflow = 1;
  }
  block_add(kept, &v.hdr->pass1_kept);
  block_add(kept, v.partial ? &v.hdr->pass2_kept : &v.hdr->round_kept);
  if (round == v.count_round) block_add(valid_n, &v.hdr->positions);
}

// ---------------------------------------------------------------------------
// Region-ordered first pass (class-map rounds). A filter far beyond L2 takes
// every random OR and every random probe at DRAM's random-access rate (about
// 64 bytes moved per 8-byte access). Here a round instead writes one 8-byte
// record per position of its class into the bucket of the position's filter
// region (at most 2^22 words: 32 MiB, which L2 holds), applies the ORs and
// then the probes bucket by bucket -- so that the random accesses of a region
// all hit L2 -- and gathers the probe's decisions back in position order.
//
// Buckets: the class map counted the positions of every (class, region)
// pair per tile, so a round's buckets are laid out exactly (each a multiple
// of 32 slots). Tiles: kOrdTile consecutive positions, each warp of the block
// taking kOrdTile / 8 of them (kOrdTileWindows / 8 windows). A tile's records
// for a bucket are consecutive in the bucket, in tile order: a scan over the
// tiles' counts gives every tile its room in every bucket (o_meta). The
// members of a round are numbered in position order (o_tbase holds every
// tile's first number); o_perm[member] is the member's rank within its
// tile's room, so that the gather finds the member's decision bit at
// o_start[bucket] + room + rank.
//
// A record: bits 0-21 the word within its region, 22-51 the bits 32-61 of G
// (the bit bases of up to 6 bits per item), 52-56 and 57-61 the items (two
// for a palindrome's orientations), bit 62 the sentinel flag. With pass 2 on
// the records (k <= 27) a record holds the occurrence instead (fused_record).
// ---------------------------------------------------------------------------

constexpr int kOrdWarpWindows = kOrdTileWindows / (kBlock / 32);  // windows per warp and tile
constexpr uint32_t kOrdPiece = 4096;  // records per apply or probe work item (a multiple of 32)
constexpr unsigned long long kOrdSentinel = 1ull << 62;

// Fused records (k <= 27, o_fused): the round's pass 2 runs on the same
// records. A record then holds the occurrence itself -- bits 7-60 the
// normalized k-mer, 6 the sentinel flag, 5 and 4 whether the string reads the
// k-mer's reverse complement and the k-mer itself there (both for a
// palindrome), 2-3 and 0-1 the predecessor and successor bases -- and the
// kernels that apply it recompute H, G, the filter word and the items.
__device__ __forceinline__ unsigned long long fused_record(const RunView& v, uint64_t g, bool sentinel) {
  const Key f = load_kmer<1>(v.packed, g, v.k);
  const Key r = v.both ? revcomp<1>(f, v.k) : f;
  const uint32_t pred = sentinel ? 0u : base_at(v.packed, g - 1);
  const uint32_t succ = sentinel ? 0u : base_at(v.packed, g + v.k);
  const bool use_f = !v.both || !key_less(r, f);
  const bool use_r = v.both && !key_less(f, r);
  const uint64_t key = use_f ? f.lo : r.lo;
  return (key << 7) | ((uint64_t)sentinel << 6) | ((uint64_t)use_r << 5) | ((uint64_t)use_f << 4) |
         ((uint64_t)pred << 2) | succ;
}

struct FusedOcc {
  uint64_t key, H, G;
  uint32_t items, tbits;
  bool sentinel;
};

__device__ __forceinline__ FusedOcc fused_occ(unsigned long long rec) {
  FusedOcc o;
  o.key = rec >> 7;
  o.sentinel = (rec >> 6) & 1u;
  occ_bits((uint32_t)(rec >> 2) & 3u, (uint32_t)rec & 3u, (rec >> 4) & 1u, (rec >> 5) & 1u, o.sentinel, &o.items,
           &o.tbits);
  o.H = mix64(o.key);  // key_hash of a one-word k-mer
  o.G = second_hash(o.H);
  return o;
}

// The fused pass-2 table: bucket b owns the o_tcap one-word slots (key << 9 |
// mask) from b * o_tcap, so that its inserts and lookups stay in L2 beside
// the filter region; a k-mer starts at bits 16-47 of H scaled to o_tcap
// (Lemire's multiply-high) and probes linearly within the region.
__device__ __forceinline__ bool fused_table_insert(const RunView& v, uint32_t b, uint64_t key, uint64_t H,
                                                   uint32_t tbits) {
  const uint32_t cap = v.o_tcap;
  unsigned long long* T = static_cast<unsigned long long*>(v.table) + (uint64_t)b * cap;
  uint32_t i = __umulhi((uint32_t)(H >> 16), cap);
  for (uint32_t probe = 0; probe < cap; ++probe, i = i + 1 == cap ? 0u : i + 1) {
    unsigned long long cur = __ldcg(T + i);
    if (cur == kEmpty) {
      cur = atomicCAS(T + i, kEmpty, (key << kMaskBits) | tbits);
      if (cur == kEmpty) return true;
    }
    if ((cur >> kMaskBits) != key) continue;
    if ((cur & tbits) != tbits) atomicOr(T + i, (unsigned long long)tbits);
    return true;
  }
  return false;
}

// Mask of key in the fused table, or -1 if absent.
__device__ __forceinline__ int fused_table_find(const RunView& v, uint32_t b, uint64_t key, uint64_t H) {
  const uint32_t cap = v.o_tcap;
  const unsigned long long* T = static_cast<const unsigned long long*>(v.table) + (uint64_t)b * cap;
  uint32_t i = __umulhi((uint32_t)(H >> 16), cap);
  for (uint32_t probe = 0; probe < cap; ++probe, i = i + 1 == cap ? 0u : i + 1) {
    const unsigned long long cur = __ldcg(T + i);
    if (cur == kEmpty) return -1;
    if ((cur >> kMaskBits) == key) return (int)(cur & ((1u << kMaskBits) - 1u));
  }
  return -1;
}

// A lane's 16 positions of the window at wbase: their class and region bytes.
__device__ __forceinline__ void ord_lane_bytes(const RunView& v, uint64_t wbase, uint4* cls, uint4* reg) {
  const uint64_t p0 = wbase + 16 * (uint64_t)(threadIdx.x & 31);
  *cls = make_uint4(0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u);
  *reg = make_uint4(0u, 0u, 0u, 0u);
  if (p0 < v.m) {
    *cls = __ldcg(reinterpret_cast<const uint4*>(v.cmap + p0));
    *reg = __ldcg(reinterpret_cast<const uint4*>(v.rplane + p0));
  }
}

// Bit i: the lane's position i is of this round's class (act), a sentinel
// (sent), has a k-mer (val).
__device__ __forceinline__ void ord_lane_bits(const uint4& q, int round, uint32_t* act, uint32_t* sent,
                                              uint32_t* val) {
  const uint32_t part[4] = {q.x, q.y, q.z, q.w};
  const uint32_t want = (uint32_t)round * 0x01010101u;
  uint32_t a = 0, s = 0, l = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    a |= byte_bits(__vcmpeq4(part[c] & 0xBFBFBFBFu, want)) << (4 * c);
    s |= byte_bits(part[c] << 1) << (4 * c);
    l |= byte_bits(~part[c]) << (4 * c);
  }
  *act = a;
  *sent = s;
  *val = l;
}

__device__ __forceinline__ uint32_t uint4_byte(const uint4& q, uint32_t i) {
  const uint32_t w = i < 8 ? (i < 4 ? q.x : q.y) : (i < 12 ? q.z : q.w);
  return (w >> (8 * (i & 3))) & 0xFFu;
}

// compact_window with the region of every listed position in reg[0 .. n).
__device__ __forceinline__ uint32_t compact_window_ord(const RunView& v, uint64_t wbase, int round, uint16_t* idx,
                                                       uint8_t* reg) {
  const int lane = threadIdx.x & 31;
  uint4 q, rq;
  ord_lane_bytes(v, wbase, &q, &rq);
  uint32_t act, sent, val;
  ord_lane_bits(q, round, &act, &sent, &val);
  const uint32_t n = __popc(act);
  uint32_t inc = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  uint32_t at = inc - n;
  while (act) {
    const uint32_t i = __ffs(act) - 1;
    act &= act - 1;
    idx[at] = (uint16_t)((16 * lane + i) | (((sent >> i) & 1u) << 9));
    reg[at] = (uint8_t)uint4_byte(rq, i);
    ++at;
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, inc, 31);
}

// Members of every (round, tile): thread blocks of the scan below take
// kOrdScanTiles tiles of one round each.

// o_tsum[round * chunks + c] = members of the round in tiles [c * 1024, (c + 1) * 1024).
__global__ void __launch_bounds__(kBlock) ord_tile_sum_kernel(RunView v, uint64_t chunks) {
  const uint64_t r = blockIdx.x / chunks, c = blockIdx.x % chunks;
  const uint32_t* cnt = v.o_tcount + r * v.o_tiles;
  unsigned long long s = 0;
  for (uint64_t t = c * kOrdScanTiles + threadIdx.x; t < min((c + 1) * kOrdScanTiles, v.o_tiles); t += kBlock)
    s += cnt[t];
  __shared__ unsigned long long part[kBlock / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kBlock / 32; ++w) t += part[w];
    v.o_tsum[blockIdx.x] = t;
  }
}

// o_tbase[round * tiles + t] = members of the round in tiles before t.
__global__ void __launch_bounds__(kBlock) ord_tile_scan_kernel(RunView v, uint64_t chunks) {
  const uint64_t r = blockIdx.x / chunks, c = blockIdx.x % chunks;
  unsigned long long before = 0;
  for (uint64_t i = threadIdx.x; i < c; i += kBlock) before += v.o_tsum[r * chunks + i];
  __shared__ unsigned long long part[kBlock / 32];
  __shared__ unsigned long long carry_s;
  before = warp_sum(before);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = before;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kBlock / 32; ++w) t += part[w];
    carry_s = t;
  }
  __syncthreads();
  const uint32_t* cnt = v.o_tcount + r * v.o_tiles;
  unsigned long long* base = v.o_tbase + r * v.o_tiles;
  for (uint64_t t0 = c * kOrdScanTiles; t0 < min((c + 1) * kOrdScanTiles, v.o_tiles); t0 += kBlock) {
    const uint64_t t = t0 + threadIdx.x;
    const uint32_t x = t < v.o_tiles ? cnt[t] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(x, &tot);
    if (t < v.o_tiles) base[t] = carry_s + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry_s += tot;
    __syncthreads();
  }
}

// Exclusive scan of x over the block (blockDim.x == kBlock), 64-bit.
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long x, unsigned long long* total) {
  __shared__ unsigned long long warp_tot[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  unsigned long long before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kBlock / 32; ++w) {
    const unsigned long long t = warp_tot[w];
    before += (w < wid) ? t : 0ull;
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + inc - x;
}

// The rooms of a round's tiles in its buckets, in tile order: o_meta[t * R + b]
// = the round's members of bucket b in the tiles before t. Three steps over
// chunks of kOrdScanTiles tiles: the chunks' sums, their prefix per bucket
// (with every bucket's total, o_btot), then every tile's room.
__global__ void __launch_bounds__(kBlock) ord_room_sum_kernel(RunView v, int round) {
  const uint32_t R = v.o_regions, b = threadIdx.x, nh = (uint32_t)v.rounds * R;
  if (b >= R) return;
  const uint64_t c = blockIdx.x, t1 = min((c + 1) * kOrdScanTiles, v.o_tiles);
  const uint16_t* th = v.o_thist + (uint64_t)round * R + b;
  uint32_t s = 0;
#pragma unroll 8
  for (uint64_t t = c * kOrdScanTiles; t < t1; ++t) s += th[t * nh];
  v.o_csum[c * R + b] = s;
}

__global__ void __launch_bounds__(kBlock) ord_room_prefix_kernel(RunView v, uint64_t chunks) {
  const uint32_t R = v.o_regions, b = blockIdx.x;
  __shared__ unsigned long long carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint64_t c0 = 0; c0 < chunks; c0 += kBlock) {
    const uint64_t c = c0 + threadIdx.x;
    const unsigned long long x = c < chunks ? v.o_csum[c * R + b] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan64(x, &tot);
    if (c < chunks) v.o_cpre[c * R + b] = carry_s + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) v.o_btot[b] = carry_s;
}

__global__ void __launch_bounds__(kBlock) ord_room_scan_kernel(RunView v, int round) {
  const uint32_t R = v.o_regions, b = threadIdx.x, nh = (uint32_t)v.rounds * R;
  if (b >= R) return;
  const uint64_t c = blockIdx.x, t1 = min((c + 1) * kOrdScanTiles, v.o_tiles);
  const uint16_t* th = v.o_thist + (uint64_t)round * R + b;
  unsigned long long run = v.o_cpre[c * R + b];
  for (uint64_t t = c * kOrdScanTiles; t < t1; ++t) {
    v.o_meta[t * R + b] = (uint32_t)run;  // within a bucket below 2^32 (the setup checks)
    run += th[t * nh];
  }
}

// Before a round's scatter: the buckets' starts (each a multiple of 32), the
// work tickets cleared, and whether the round's records fit (else the direct
// kernels take the round). One block.
__global__ void __launch_bounds__(kBlock) ord_setup_kernel(RunView v, int round) {
  const uint32_t R = v.o_regions;
  for (uint32_t b = threadIdx.x; b < R; b += kBlock) v.o_fill[(uint64_t)b * kOrdFillStride] = (uint32_t)v.o_btot[b];
  if (threadIdx.x == 0) {
    uint64_t at = 0;
    bool fits = true;
    for (uint32_t b = 0; b < R; ++b) {
      v.o_start[b] = at;
      const uint64_t n = v.o_btot[b];
      fits = fits && n < (1ull << 32);  // slots within a bucket are 32-bit
      at += (n + 31) & ~31ull;
    }
    v.o_start[R] = at;
    v.hdr->ord_ok = (fits && at <= v.o_rec_cap) ? 1u : 0u;
    v.hdr->ord_rounds += v.hdr->ord_ok;
    v.hdr->ord_ticket[0] = 0;
    v.hdr->ord_ticket[1] = 0;
    v.hdr->ord_ticket[2] = 0;
  }
}

// Records a tile stages in shared memory, sorted by bucket, before writing
// them out run by run (a tile with more members writes them one by one).
constexpr uint32_t kOrdStage = 4352;  // four blocks of 256 threads per SM (228 KB of shared memory)
constexpr size_t kOrdStageBytes = (size_t)kOrdStage * 9;  // the records, then their buckets

// Algorithm 1, insert loop, first pass, over this round's class: one record
// per position into the bucket of its filter region (tiles grid-strided).
template <int KW, int HB, bool FUSED>
__global__ void __launch_bounds__(kBlock) ord_scatter_kernel(RunView v, int round) {
  extern __shared__ __align__(16) unsigned char ord_dyn_s[];
  unsigned long long* stage_rec = reinterpret_cast<unsigned long long*>(ord_dyn_s);
  uint8_t* stage_b = ord_dyn_s + (size_t)kOrdStage * 8;
  __shared__ uint16_t idx_s[kBlock / 32][kCmWindow];
  __shared__ uint8_t reg_s[kBlock / 32][kCmWindow];
  __shared__ uint32_t cur_s[kOrdMaxRegions];   // members per bucket, then the next rank
  __shared__ uint32_t room_s[kOrdMaxRegions];  // where the tile's room starts in every bucket
  __shared__ uint32_t off_s[kOrdMaxRegions];   // where every bucket's run starts in the stage
  __shared__ unsigned long long start_s[kOrdMaxRegions];
  __shared__ uint32_t wcnt_s[kBlock / 32];
  if (!ordered_round(v)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t R = v.o_regions;
  for (uint32_t b = threadIdx.x; b < R; b += kBlock) start_s[b] = v.o_start[b];
  const uint64_t local_mask = (1ull << v.o_lg_region_words) - 1ull;
  const unsigned long long* tbase = v.o_tbase + (uint64_t)round * v.o_tiles;
  const uint64_t n_tiles = (v.p_end - v.p_begin + kOrdTile - 1) / kOrdTile;
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint64_t tpos = v.p_begin + t * kOrdTile;
    // the tile's members per bucket (o_thist) and per warp chunk (o_wcount),
    // and its rooms (o_meta)
    const uint32_t mine = threadIdx.x < R ? v.o_thist[(t * v.rounds + round) * R + threadIdx.x] : 0u;
    uint32_t total;
    const uint32_t off = block_exclusive_scan(mine, &total);
    if (threadIdx.x < R) {
      room_s[threadIdx.x] = __ldg(v.o_meta + t * R + threadIdx.x);
      off_s[threadIdx.x] = off;
      cur_s[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
      const uint16_t* wcnt = v.o_wcount + ((uint64_t)round * v.o_tiles + t) * (kBlock / 32);
      uint32_t run = 0;
      for (int w = 0; w < kBlock / 32; ++w) {
        wcnt_s[w] = run;
        run += wcnt[w];
      }
    }
    __syncthreads();
    const bool staged = total <= kOrdStage;
    uint64_t mi = tbase[t] + wcnt_s[wid];  // number of the warp's next member
    for (int q = 0; q < kOrdWarpWindows; ++q) {
      const uint64_t wbase = tpos + (uint64_t)(wid * kOrdWarpWindows + q) * kCmWindow;
      if (wbase >= v.p_end) break;
      const uint32_t n = compact_window_ord(v, wbase, round, idx_s[wid], reg_s[wid]);
      for (uint32_t j = lane; j < n; j += 32) {
        const uint32_t e = idx_s[wid][j], b = reg_s[wid][j];
        const uint32_t rank = atomicAdd(&cur_s[b], 1u);
        v.o_perm[mi + j] = (uint16_t)rank;
        const bool sentinel = (e >> 9) & 1u;
        unsigned long long rec;
        if constexpr (FUSED) {
          rec = fused_record(v, wbase + (e & 511u), sentinel);
        } else {
          OccT<KW> oc;
          read_listed<KW>(v, wbase + (e & 511u), sentinel, &oc);
          const uint64_t G = second_hash(oc.H);
          const uint32_t j1 = __ffs(oc.items) - 1, j2 = 31 - __clz(oc.items);
          const uint64_t word = filter_index(v, oc.H, G);
          rec = (word & local_mask) | (((G >> 32) & 0x3FFFFFFFull) << 22) | ((uint64_t)j1 << 52) |
                ((uint64_t)j2 << 57) | (sentinel ? kOrdSentinel : 0ull);
        }
        if (staged) {
          stage_rec[off_s[b] + rank] = rec;
          stage_b[off_s[b] + rank] = (uint8_t)b;
        } else {
          v.o_recs[start_s[b] + room_s[b] + rank] = rec;
        }
      }
      mi += n;
      __syncwarp();
    }
    __syncthreads();
    if (staged) {  // consecutive threads on consecutive records of a run
      for (uint32_t i = threadIdx.x; i < total; i += kBlock) {
        const uint32_t b = stage_b[i];
        v.o_recs[start_s[b] + room_s[b] + (i - off_s[b])] = stage_rec[i];
      }
      __syncthreads();
    }
  }
}

// Work items of kOrdPiece records, taken in bucket order from a ticket, so
// that the blocks in flight work on one or two regions at a time. first_s[b]:
// the first item of bucket b (first_s[R]: the number of items).
__device__ __forceinline__ void ord_items(const RunView& v, uint32_t* first_s) {
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t b = 0; b < v.o_regions; ++b) {
      first_s[b] = acc;
      const uint64_t n = __ldcg(v.o_fill + (uint64_t)b * kOrdFillStride);
      acc += (uint32_t)((n + kOrdPiece - 1) / kOrdPiece);
    }
    first_s[v.o_regions] = acc;
  }
  __syncthreads();
}

// Warm L2 with this work item's share of the next bucket's filter region, so
// that the region's first accesses do not wait on DRAM one random sector at
// a time (the items of a bucket together cover the whole next region).
__device__ __forceinline__ void ord_prefetch_next(const RunView& v, const uint32_t* first_s, uint32_t b,
                                                  uint32_t item) {
  if (b + 1 >= v.o_regions) return;
  const uint64_t rbytes = 8ull << v.o_lg_region_words;
  const uint64_t share = (rbytes / (first_s[b + 1] - first_s[b]) + 127) & ~127ull;
  const uint64_t off = (uint64_t)(item - first_s[b]) * share, end = min(off + share, rbytes);
  const char* next = reinterpret_cast<const char*>(v.filter + ((uint64_t)(b + 1) << v.o_lg_region_words));
  for (uint64_t o = off + 128 * (uint64_t)threadIdx.x; o < end; o += 128 * (uint64_t)kBlock)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(next + o));
}

__device__ __forceinline__ uint32_t ord_item_bucket(const uint32_t* first_s, uint32_t R, uint32_t item) {
  uint32_t lo = 0, hi = R;  // the bucket b with first_s[b] <= item < first_s[b + 1]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (first_s[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// The ORs of the round's records, bucket by bucket (four records in flight
// per thread).
template <int HB, bool FUSED>
__global__ void __launch_bounds__(kBlock) ord_or_kernel(RunView v) {
  __shared__ uint32_t first_s[kOrdMaxRegions + 1];
  __shared__ uint32_t item_s;
  if (!ordered_round(v)) return;
  ord_items(v, first_s);
  const uint32_t R = v.o_regions, total = first_s[R];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(&v.hdr->ord_ticket[0], 1u);
    __syncthreads();
    const uint32_t item = item_s;
    __syncthreads();
    if (item >= total) break;
    const uint32_t b = ord_item_bucket(first_s, R, item);
    ord_prefetch_next(v, first_s, b, item);
    const uint64_t n = __ldcg(v.o_fill + (uint64_t)b * kOrdFillStride);
    const uint64_t i0 = (uint64_t)(item - first_s[b]) * kOrdPiece, i1 = min(i0 + kOrdPiece, n);
    const uint64_t* recs = v.o_recs + __ldg(v.o_start + b);
    unsigned long long* region = v.filter + ((uint64_t)b << v.o_lg_region_words);
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += 4 * kBlock) {
      uint64_t r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) r[u] = i + u * kBlock < i1 ? __ldcs(recs + i + u * kBlock) : ~0ull;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (r[u] == ~0ull) continue;
        if constexpr (FUSED) {
          const FusedOcc o = fused_occ(r[u]);
          const ItemPattern pat = item_pattern<HB>(o.G, v.hashes);
          const uint32_t j1 = __ffs(o.items) - 1, j2 = 31 - __clz(o.items);
          uint64_t m = item_bits(pat, j1);
          if (j2 != j1) m |= item_bits(pat, j2);
          atomicOr(v.filter + filter_index(v, o.H, o.G), (unsigned long long)m);
        } else {
          const uint64_t G = ((r[u] >> 22) & 0x3FFFFFFFull) << 32;  // the bits bit_base reads for u < 6
          const ItemPattern pat = item_pattern<HB>(G, v.hashes);
          const uint32_t j1 = (uint32_t)(r[u] >> 52) & 31u, j2 = (uint32_t)(r[u] >> 57) & 31u;
          uint64_t m = item_bits(pat, j1);
          if (j2 != j1) m |= item_bits(pat, j2);
          atomicOr(region + (r[u] & 0x3FFFFFull), (unsigned long long)m);
        }
      }
    }
  }
}

// Algorithm 1, probe loop, first pass, over the round's records, bucket by
// bucket: a record's decision (its k-mer is a candidate: a sentinel, or its
// filter word holds a sentinel item or two distinct items) goes to its slot's
// bit; the linear-counting bit of every candidate is set from the k-mer's
// filter word index and bit bases. FUSED: instead, every candidate inserts
// its in/out bases into its region's part of the pass-2 table (Algorithm 1's
// insert loop, second pass) while the region is in L2.
template <int HB, bool FUSED>
__global__ void __launch_bounds__(kBlock) ord_probe_kernel(RunView v) {
  __shared__ uint32_t first_s[kOrdMaxRegions + 1];
  __shared__ uint32_t item_s;
  if (!ordered_round(v)) return;
  ord_items(v, first_s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t R = v.o_regions, total = first_s[R];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(&v.hdr->ord_ticket[1], 1u);
    __syncthreads();
    const uint32_t item = item_s;
    __syncthreads();
    if (item >= total) break;
    const uint32_t b = ord_item_bucket(first_s, R, item);
    ord_prefetch_next(v, first_s, b, item);
    const uint64_t n = __ldcg(v.o_fill + (uint64_t)b * kOrdFillStride);
    const uint64_t i0 = (uint64_t)(item - first_s[b]) * kOrdPiece, i1 = min(i0 + kOrdPiece, n);
    const uint64_t start = __ldg(v.o_start + b);  // a multiple of 32, as is i0
    const uint64_t* recs = v.o_recs + start;
    const uint64_t region = (uint64_t)b << v.o_lg_region_words;
    for (uint64_t w0 = i0 + 32 * wid; w0 < i1; w0 += kBlock) {
      const uint64_t i = w0 + lane;
      bool keep = false;
      if (FUSED && i < i1) {  // the decision, and the candidate's edges into the region's table
        const FusedOcc o = fused_occ(__ldcs(recs + i));
        if (o.sentinel) {
          keep = true;
        } else {
          const uint64_t word = __ldcg(v.filter + filter_index(v, o.H, o.G));
          const uint32_t pres = present_items<HB>(o.G, word, v.hashes);
          keep = (pres >> 16) || __popc(pres & 0xFFFFu) >= 2;
        }
        if (keep && !fused_table_insert(v, b, o.key, o.H, o.tbits)) v.hdr->overflow = 1;
      } else if (i < i1) {
        const uint64_t r = __ldcs(recs + i);
        const uint64_t word_index = region | (r & 0x3FFFFFull);
        if (r & kOrdSentinel) {
          keep = true;
        } else {
          const uint64_t G = ((r >> 22) & 0x3FFFFFFFull) << 32;
          const uint64_t word = __ldcg(v.filter + word_index);
          const uint32_t pres = present_items<HB>(G, word, v.hashes);
          keep = (pres >> 16) || __popc(pres & 0xFFFFu) >= 2;
        }
        if (keep && !v.partial) {  // linear counting over a 2^-lc_sample_log2 sample of the k-mers
          const uint64_t id = (word_index << 30) | ((r >> 22) & 0x3FFFFFFFull);
          const uint64_t h = id * 0xff51afd7ed558ccdull;
          if (((uint32_t)(h >> 24) & ((1u << v.lc_sample_log2) - 1u)) == 0) {
            const uint64_t x = h >> (64 - v.lc_log2);
            atomicOr(v.lc_bits + (x >> 5), 1u << (x & 31));
          }
        }
      }
      const uint32_t row = __ballot_sync(0xffffffffu, keep);
      // fused: word pairs, the candidates' bits then the junctions' (ord_classify)
      if (lane == 0) v.o_dec[((start + w0) >> 5) << (FUSED ? 1 : 0)] = row;
    }
  }
}

// Algorithm 1, probe loop, second pass, on fused records, bucket by bucket:
// every candidate record (decision bit set) looks its k-mer up in the
// region's table; its bit in the junction word of o_dec says whether the
// k-mer is a junction (the table mask holds the sentinel bit or more than
// one in- or out-base).
__global__ void __launch_bounds__(kBlock) ord_classify_kernel(RunView v) {
  __shared__ uint32_t first_s[kOrdMaxRegions + 1];
  __shared__ uint32_t item_s;
  if (!ordered_round(v)) return;
  ord_items(v, first_s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t R = v.o_regions, total = first_s[R];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(&v.hdr->ord_ticket[2], 1u);
    __syncthreads();
    const uint32_t item = item_s;
    __syncthreads();
    if (item >= total) break;
    const uint32_t b = ord_item_bucket(first_s, R, item);
    const uint64_t n = __ldcg(v.o_fill + (uint64_t)b * kOrdFillStride);
    const uint64_t i0 = (uint64_t)(item - first_s[b]) * kOrdPiece, i1 = min(i0 + kOrdPiece, n);
    const uint64_t start = __ldg(v.o_start + b);  // a multiple of 32, as is i0
    const uint64_t* recs = v.o_recs + start;
    // four chunks of 32 records per warp and step: their loads all in flight at once
    constexpr int U = 4;
    for (uint64_t w0 = i0 + 32 * wid; w0 < i1; w0 += U * kBlock) {
      uint32_t cand[U];
      unsigned long long rec[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t c = w0 + (uint64_t)u * kBlock;
        cand[u] = c < i1 ? __ldcg(v.o_dec + (((start + c) >> 5) << 1)) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t i = w0 + (uint64_t)u * kBlock + lane;
        rec[u] = (i < i1 && ((cand[u] >> lane) & 1u)) ? __ldcs(recs + i) : ~0ull;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t c = w0 + (uint64_t)u * kBlock;
        bool junction = false;
        if (rec[u] != ~0ull) {
          const FusedOcc o = fused_occ(rec[u]);
          const int mk = fused_table_find(v, b, o.key, o.H);
          if (mk < 0) v.hdr->overflow = 1;
          junction = mk < 0 || is_junction_mask(mk);
        }
        const uint32_t row = __ballot_sync(0xffffffffu, junction);
        if (lane == 0 && c < i1) v.o_dec[(((start + c) >> 5) << 1) + 1] = row;
      }
    }
  }
}

// The probe loop's outputs in position order: every member of the round's
// class takes its decision from its record's slot (its tile's room in its
// bucket plus its rank, o_perm); C_temp words, the candidate list segment of
// the warp and the counts are as pass1_probe_cm_kernel writes them (with
// fused records: C_temp words, and the junction bits ORed into C_final
// instead of a list). Every
// lane takes its own 16 positions of a window (at most 40 registers: six
// blocks per SM).
__global__ void __launch_bounds__(kBlock, 6) ord_gather_kernel(RunView v, int round) {
  __shared__ uint32_t room_s[kOrdMaxRegions];
  __shared__ unsigned long long start_s[kOrdMaxRegions];
  __shared__ uint32_t wcnt_s[kBlock / 32];
  if (!ordered_round(v)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t R = v.o_regions;
  for (uint32_t b = threadIdx.x; b < R; b += kBlock) start_s[b] = v.o_start[b];
  unsigned long long kept = 0, valid_n = 0, junctions = 0;
  const uint32_t warp_id = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  uint64_t* seg = v.cands + (uint64_t)warp_id * v.seg_cap;
  uint32_t* seg32 = reinterpret_cast<uint32_t*>(v.cands) + (uint64_t)warp_id * v.seg_cap;
  uint64_t seg_used = 0;
  const unsigned long long* tbase = v.o_tbase + (uint64_t)round * v.o_tiles;
  const uint64_t n_tiles = (v.p_end - v.p_begin + kOrdTile - 1) / kOrdTile;
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint64_t tpos = v.p_begin + t * kOrdTile;
    for (uint32_t b = threadIdx.x; b < R; b += kBlock) room_s[b] = __ldg(v.o_meta + t * R + b);
    if (threadIdx.x == 0) {
      const uint16_t* wcnt = v.o_wcount + ((uint64_t)round * v.o_tiles + t) * (kBlock / 32);
      uint32_t run = 0;
      for (int w = 0; w < kBlock / 32; ++w) {
        wcnt_s[w] = run;
        run += wcnt[w];
      }
    }
    __syncthreads();
    uint64_t mi = tbase[t] + wcnt_s[wid];  // number of the warp's next member
    for (int q = 0; q < kOrdWarpWindows; ++q) {
      const uint64_t wbase = tpos + (uint64_t)(wid * kOrdWarpWindows + q) * kCmWindow;
      if (wbase >= v.p_end) break;
      uint4 cq, rq;
      ord_lane_bytes(v, wbase, &cq, &rq);
      uint32_t act, sent, val;
      ord_lane_bits(cq, round, &act, &sent, &val);
      valid_n += __popc(val);
      const uint32_t n = __popc(act);
      uint32_t inc = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      uint64_t at = mi + inc - n;  // number of the lane's first member
      uint32_t keep = 0, jun = 0;
      for (uint32_t a = act; a; a &= a - 1, ++at) {
        const uint32_t i = __ffs(a) - 1, b = uint4_byte(rq, i);
        const uint64_t s = start_s[b] + room_s[b] + __ldg(v.o_perm + at);
        if (v.o_fused) {  // the candidate and junction words of the slot, in one load
          const uint2 d = __ldg(reinterpret_cast<const uint2*>(v.o_dec) + (s >> 5));
          keep |= ((d.x >> (s & 31)) & 1u) << i;
          jun |= ((d.y >> (s & 31)) & 1u) << i;
        } else {
          keep |= ((__ldg(v.o_dec + (s >> 5)) >> (s & 31)) & 1u) << i;
        }
      }
      mi += __shfl_sync(0xffffffffu, inc, 31);
      // C_temp (and, fused, C_final): lanes 2i and 2i + 1 hold the halves of the window's word i
      const uint32_t hi = __shfl_down_sync(0xffffffffu, keep, 1);
      const uint32_t jhi = __shfl_down_sync(0xffffffffu, jun, 1);
      if (!(lane & 1)) {
        const uint64_t w = (wbase >> 5) + (lane >> 1);
        const uint32_t word = keep | (hi << 16);
        if (w < v.bitmap_words) {
          v.ctemp[w] = word;
          // rounds own disjoint positions; one writer per word
          if (v.partial) {
            v.cfinal[w] |= word;
          } else if (v.o_fused) {
            const uint32_t jw = jun | (jhi << 16);
            if (jw) atomicOr(v.cfinal + w, jw);  // no wait on the word's other rounds' bits
          }
        }
      }
      const uint32_t kc = __popc(keep);
      kept += kc;
      junctions += __popc(jun);
      if (v.partial || v.o_fused) continue;
      uint32_t kinc = kc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, kinc, o);
        if (lane >= o) kinc += y;
      }
      uint64_t o = seg_used + kinc - kc;
      for (uint32_t k = keep; k; k &= k - 1, ++o) {
        const uint32_t i = __ffs(k) - 1;
        const uint64_t g = wbase + 16 * (uint64_t)lane + i;
        const uint32_t sentinel = (sent >> i) & 1u;
        if (o < v.seg_cap) {
          if (v.narrow) seg32[o] = (uint32_t)g | (sentinel << 31);
          else seg[o] = g | ((uint64_t)sentinel << 63);
        }
      }
      seg_used += __shfl_sync(0xffffffffu, kinc, 31);
    }
    __syncthreads();  // room_s and wcnt_s serve the next tile
  }
  if (lane == 0) {
    v.seg_count[warp_id] = (uint32_t)(seg_used < v.seg_cap ? seg_used : v.seg_cap);
    if (seg_used > v.seg_cap) v.hdr->cand_overflow = 1;
  }
  block_add(kept, &v.hdr->pass1_kept);
  block_add(kept, v.partial ? &v.hdr->pass2_kept : &v.hdr->round_kept);
  if (v.o_fused) block_add(junctions, &v.hdr->pass2_kept);
  if (round == v.count_round) block_add(valid_n, &v.hdr->positions);
}

// Table slots per estimated distinct candidate: 2.5 for one-word slots
// (k <= 27), where probe chains cost more than memory, 2 for the wider slots,
// where a smaller table stays in L2 (measured at k = 25, 31 and 63).
constexpr double kTableLoadWord = 2.5, kTableLoad = 2.0;
// pass-2 list work: parts of about this many records, at most kMaxParts per segment
constexpr unsigned long long kPartRecords = 128, kMaxParts = 4096;

// Size the pass-2 table of this round: 2.5 or 2 times the number of distinct
// candidate k-mers, estimated by linear counting (Whang, Vander-Zanden &
// Taylor 1990) from the bits the probe set (at least 1024 slots, a multiple
// of 32, not rounded to a power of two), capped by the workspace. A saturated bitmap falls back to
// twice the number of candidate positions. The estimate only sets the table's
// size; an undersized table is detected and reported, never silently wrong.
// Every block counts its share of the bitmap; the last block to finish sizes
// the table.
__global__ void __launch_bounds__(kBlock) table_setup_kernel(RunView v) {
  if (v.o_fused && ordered_round(v)) {  // the round's table was the fused one: nothing left to size or clear
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long used = (unsigned long long)v.o_tcap * v.o_regions;
      v.hdr->table_slots = 0;
      if (used > v.hdr->table_max) v.hdr->table_max = used;
      v.hdr->cand_overflow = 0;
      v.hdr->round_kept = 0;
      v.hdr->lc_set = 0;
      v.hdr->lc_blocks_done = 0;
    }
    return;
  }
  const uint64_t words = (1ull << v.lc_log2) / 32;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  unsigned long long c = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < words; i += stride)
    c += __popc(__ldcg(v.lc_bits + i));
  block_add(c, &v.hdr->lc_set);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&v.hdr->lc_blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  const unsigned long long kept = *(volatile unsigned long long*)&v.hdr->round_kept;
  const unsigned long long set = *(volatile unsigned long long*)&v.hdr->lc_set;
  const double M = (double)(1ull << v.lc_log2);
  unsigned long long distinct = kept;
  if ((double)set < M - M / 1024.0) {  // at least 1/1024 of the bits still clear: about 7 per bit
    // a region-ordered round counted a 2^-s sample of the k-mers: scale it up,
    // with eight standard deviations of the sample's size to spare
    const int sl = (v.o_regions && *(volatile unsigned int*)&v.hdr->ord_ok) ? v.lc_sample_log2 : 0;
    const double f = (double)(1u << sl);
    const double est = -M * log1p(-(double)set / M) * f;
    const unsigned long long e = (unsigned long long)(est * 1.1 + (sl ? 8.0 * sqrt(est * f) : 0.0)) + 64ull;
    if (e < distinct) distinct = e;
  }
  unsigned long long cap =
      (unsigned long long)((v.k <= 27 ? kTableLoadWord : kTableLoad) * (double)distinct);
  if (cap < 1024ull) cap = 1024ull;
  cap = (cap + 31) / 32 * 32;  // any capacity works (slot_start); whole 32-slot groups
  if (cap > v.table_max_slots) cap = v.table_max_slots;
  v.hdr->table_slots = cap;
  if (cap > v.hdr->table_max) v.hdr->table_max = cap;
  v.hdr->round_listed = *(volatile unsigned int*)&v.hdr->cand_overflow ? 0u : 1u;
  // pass 2 cuts every list segment into parts of about kPartRecords records
  unsigned long long parts = (kept / v.n_segments + kPartRecords) / kPartRecords;
  v.hdr->list_parts = (unsigned int)(parts < kMaxParts ? parts : kMaxParts);
  v.hdr->cand_overflow = 0;
  v.hdr->round_kept = 0;
  v.hdr->lc_set = 0;
  v.hdr->lc_blocks_done = 0;
}

template <int TS>
__global__ void __launch_bounds__(kBlock) table_clear_kernel(RunView v) {
  const uint64_t cap = *(volatile unsigned long long*)&v.hdr->table_slots;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < cap; i += stride) {
    if (TS == 0) {
      static_cast<unsigned long long*>(v.table)[i] = kEmpty;
    } else if (TS == 1) {
      Slot1* s = static_cast<Slot1*>(v.table) + i;
      *reinterpret_cast<ulonglong2*>(s) = make_ulonglong2(kEmpty, 0ull);
    } else if (TS == 3) {
      reinterpret_cast<ulonglong2*>(v.table)[i] = make_ulonglong2(0ull, 0ull);
    } else {
      Slot2* s = static_cast<Slot2*>(v.table) + i;
      reinterpret_cast<ulonglong2*>(s)[0] = make_ulonglong2(kEmpty, kEmpty);
      reinterpret_cast<ulonglong2*>(s)[1] = make_ulonglong2(0ull, 0ull);
    }
  }
}

// Candidate i of the list: its position, and whether it is a sentinel
// position (the record's top bit; 32-bit records when the input has fewer
// than 2^31 bases).
__device__ __forceinline__ uint64_t list_at(const RunView& v, uint64_t i, bool* sentinel, bool last_use) {
  if (v.narrow) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(v.cands) + i;
    const uint32_t r = last_use ? __ldcs(p) : __ldcg(p);
    *sentinel = r >> 31;
    return r & 0x7FFFFFFFu;
  }
  const uint64_t r = last_use ? __ldcs(v.cands + i) : __ldcg(v.cands + i);
  *sentinel = r >> 63;
  return r & ~(1ull << 63);
}

// Pass-2 work over the candidate list. Every list segment is cut into
// list_parts parts (interleaved 32-record rows), and the launched warps take
// the (segment, part) pairs in turn, so that the work spreads evenly over a
// grid that is resident all at once. fn(i) runs for list index i.
template <typename F>
__device__ __forceinline__ void for_listed(const RunView& v, F&& fn) {
  // 32-bit arithmetic: at most kMaxSegments segments of at most kMaxParts parts
  const uint32_t parts = *(volatile unsigned int*)&v.hdr->list_parts;
  const uint32_t pairs = v.n_segments * parts;
  const uint32_t warps = gridDim.x * (kBlock / 32);
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t w = (blockIdx.x * kBlock + threadIdx.x) >> 5; w < pairs; w += warps) {
    const uint32_t sgm = w / parts, part = w - sgm * parts;
    const uint32_t n = __ldcg(v.seg_count + sgm);
    const uint64_t first = (uint64_t)sgm * v.seg_cap;
    for (uint32_t j = part * 32 + lane; j < n; j += 32 * parts) fn(first + j);
  }
}

// for_listed that reads each record one ahead: fn(i, g, sentinel, slot)
// gets list index i with its position (and with SLOT its kept table slot)
// already loaded, while the lane's next record is in flight.
template <bool SLOT, typename F>
__device__ __forceinline__ void for_listed_ahead(const RunView& v, bool last_use, F&& fn) {
  const uint32_t parts = *(volatile unsigned int*)&v.hdr->list_parts;
  const uint32_t pairs = v.n_segments * parts;
  const uint32_t warps = gridDim.x * (kBlock / 32);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t row = 32 * parts;
  for (uint32_t w = (blockIdx.x * kBlock + threadIdx.x) >> 5; w < pairs; w += warps) {
    const uint32_t sgm = w / parts, part = w - sgm * parts;
    const uint32_t n = __ldcg(v.seg_count + sgm);
    const uint64_t first = (uint64_t)sgm * v.seg_cap;
    uint32_t j = part * 32 + lane;
    bool sent = false;
    uint64_t g = j < n ? list_at(v, first + j, &sent, last_use) : 0;
    uint32_t slot = (SLOT && j < n) ? __ldcs(v.cand_slot + first + j) : 0u;
    while (j < n) {
      const uint32_t jn = j + row;
      bool sent_n = false;
      const uint64_t gn = jn < n ? list_at(v, first + jn, &sent_n, last_use) : 0;
      const uint32_t slot_n = (SLOT && jn < n) ? __ldcs(v.cand_slot + first + jn) : 0u;
      fn(first + j, g, sent, slot);
      j = jn;
      g = gn;
      sent = sent_n;
      slot = slot_n;
    }
  }
}

// Algorithm 1, insert loop, second pass: every candidate ORs its in/out bases
// (or the sentinel bit) into the exact table entry of its k-mer. Reads the
// candidate list and keeps the slot of each listed candidate for the probe
// loop; if the list overflowed, walks C_temp instead.
template <int KW, int TS>
__global__ void __launch_bounds__(kBlock) pass2_insert_kernel(RunView v) {
  if (v.o_fused && ordered_round(v)) return;  // the fused records took this round's pass 2
  const uint64_t cap = *(volatile unsigned long long*)&v.hdr->table_slots;
  if (*(volatile unsigned int*)&v.hdr->round_listed) {
    auto insert_one = [&](uint64_t i, uint64_t g, bool sent, uint32_t) {
      OccT<KW> oc;
      read_listed<KW>(v, g, sent, &oc);
      const uint64_t slot = insert_occurrence<KW, TS>(v, cap, oc, g);
      if (slot == kNoSlot) v.hdr->overflow = 1;
      if (v.cand_slot) v.cand_slot[i] = slot == kNoSlot ? 0xFFFFFFFFu : (uint32_t)slot;
    };
    if (kInsertPrefetch) {
      for_listed_ahead<false>(v, false, insert_one);
    } else {
      for_listed(v, [&](uint64_t i) {
        bool sent;
        const uint64_t g = list_at(v, i, &sent, false);
        insert_one(i, g, sent, 0u);
      });
    }
    return;
  }
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t g = v.p_begin + (uint64_t)blockIdx.x * kBlock + threadIdx.x; g < v.p_end; g += stride) {
    if (!((__ldg(v.ctemp + (g >> 5)) >> (g & 31)) & 1u)) continue;
    OccT<KW> oc;
    if (!read_occurrence<KW>(v, g, &oc)) continue;
    if (insert_occurrence<KW, TS>(v, cap, oc, g) == kNoSlot) v.hdr->overflow = 1;
  }
}

// Algorithm 1, probe loop, second pass: a candidate is a junction iff its
// k-mer is a sentinel or has more than one distinct in- or out-base. Sets
// the junction's bit of C_final (cleared before the first round). A listed
// candidate reads its mask from the slot the insert loop kept (or looks its
// k-mer up when no slots were kept).
template <int KW, int TS>
__global__ void __launch_bounds__(kBlock) pass2_classify_kernel(RunView v) {
  if (v.o_fused && ordered_round(v)) return;  // the fused records took this round's pass 2
  const uint64_t cap = *(volatile unsigned long long*)&v.hdr->table_slots;
  unsigned long long found = 0;
  auto mark = [&](uint64_t g, int mk) {
    if (mk < 0) v.hdr->overflow = 1;
    if (mk < 0 || is_junction_mask(mk)) {
      atomicOr(v.cfinal + (g >> 5), 1u << (g & 31));
      ++found;
    }
  };
  if (*(volatile unsigned int*)&v.hdr->round_listed) {
    auto classify_one = [&](uint64_t i, uint64_t g, bool sent, uint32_t slot) {
      if (v.cand_slot) {
        mark(g, slot == 0xFFFFFFFFu ? -1 : table_mask<TS>(v, slot));
      } else {
        OccT<KW> oc;
        read_listed<KW>(v, g, sent, &oc);
        mark(g, find_occurrence<KW, TS>(v, cap, oc));
      }
    };
    if (kClassifyPrefetch && v.cand_slot) {
      for_listed_ahead<true>(v, true, classify_one);
    } else if (kClassifyPrefetch) {
      for_listed_ahead<false>(v, true, classify_one);
    } else {
      for_listed(v, [&](uint64_t i) {
        bool sent;
        const uint64_t g = list_at(v, i, &sent, true);
        classify_one(i, g, sent, v.cand_slot ? __ldcs(v.cand_slot + i) : 0u);
      });
    }
  } else {
    const uint64_t stride = (uint64_t)gridDim.x * kBlock;
    for (uint64_t g = v.p_begin + (uint64_t)blockIdx.x * kBlock + threadIdx.x; g < v.p_end; g += stride) {
      if (!((__ldg(v.ctemp + (g >> 5)) >> (g & 31)) & 1u)) continue;
      OccT<KW> oc;
      if (!read_occurrence<KW>(v, g, &oc)) continue;
      mark(g, find_occurrence<KW, TS>(v, cap, oc));
    }
  }
  block_add(found, &v.hdr->pass2_kept);
}

// Partition counters (section "Multiple Rounds"): a Bloom pre-pass over all
// k-mers; counter f(k-mer) grows when the k-mer was not yet in the filter. On
// large inputs only a hash-chosen sample of the k-mers is counted (bits of H
// that neither the bin nor the filter block uses): every bin's count then
// shrinks by the same factor in expectation, which keeps the cut's balance
// while the random filter accesses drop by that factor.
template <int KW, int HB>
__global__ void __launch_bounds__(kBlock) partition_count_kernel(RunView v) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock * kR;
  for (uint64_t p0 = ((uint64_t)blockIdx.x * kBlock + threadIdx.x) * kR; p0 < v.m; p0 += stride) {
    if ((uint32_t)(p0 >> 16) & v.part_chunks) continue;  // a sample of the 64K-position chunks
    walk<KW, kR>(v, p0, [&](int, uint64_t, bool valid, const auto& oc) {
      if (!valid || ((uint32_t)(oc.H >> 16) & v.part_sample)) return;
      const uint64_t G = second_hash(oc.H);
      const uint64_t m = item_bits<HB>(G, 17u, v.hashes);
      unsigned long long* w = filter_word(v, oc.H, G);
      if ((__ldcg(w) & m) == m) return;
      const unsigned long long old = atomicOr(w, (unsigned long long)m);
      if ((old & m) != m) atomicAdd(v.bins + ((uint32_t)oc.H & v.qmask), 1u);
    });
  }
}

// Greedy class cut over the q counters: class r takes a maximal run of bins
// whose sum stays within (sum of all counters) / rounds, at least one bin,
// leaving one bin for every later class; the last class takes the rest.
__global__ void __launch_bounds__(1024) partition_cut_kernel(RunView v, int rounds, uint64_t* prefix) {
  const uint32_t q = v.qmask + 1u;
  __shared__ unsigned long long carry_s;
  __shared__ unsigned long long wsum[32];
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint32_t base = 0; base < q; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    unsigned long long x = (i < q) ? v.bins[i] : 0ull, inc = x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      before += (w < wid) ? wsum[w] : 0ull;
      all += wsum[w];
    }
    const unsigned long long c0 = carry_s;
    if (i < q) prefix[i] = c0 + before + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = c0 + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = carry_s;
    prefix[q] = total;
    const unsigned long long L = (unsigned long long)rounds;
    uint32_t j = 0;
    v.cuts[0] = 0;
    for (int r = 0; r < rounds - 1; ++r) {
      const uint32_t start = j;
      const uint32_t limit = q - (uint32_t)(rounds - 1 - r);
      // largest e in [start+1, limit] with (prefix[e] - prefix[start]) * L <= total
      uint32_t lo = start + 1, hi = limit, best = start + 1;
      while (lo <= hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if ((prefix[mid] - prefix[start]) * L <= total) {
          best = mid;
          lo = mid + 1;
        } else {
          hi = mid - 1;
        }
      }
      j = best;
      v.cuts[r + 1] = j;
    }
    v.cuts[rounds] = q;
  }
}

// Emit (single pass): tiles of kEmitTileWords bitmap words are claimed in
// order from a ticket; each publishes its junction count, looks back over its
// predecessors for the exclusive prefix (decoupled look-back, Merrill &
// Garland 2016), publishes its inclusive prefix and writes the position of
// every junction within its string, in ascending order (C_final of
// Algorithm 3). Tiles are claimed in order, so every wait is on a block that
// is already running; a wait that exceeds kSpinLimit polls sets the timeout
// flag and gives up (the result is then reported as invalid).
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

__global__ void __launch_bounds__(kBlock) emit_kernel(RunView v) {
  __shared__ unsigned long long tile_s, prefix_s, total_s;
  __shared__ uint32_t before_s[kEmitTileWords];  // junctions of the tile before each of its words
  __shared__ uint32_t warp_s[kBlock / 32];
  __shared__ uint16_t stage_s[kBlock / 32][32 * 32];  // one batch's junctions: bit offsets within the tile
  __shared__ uint64_t t_lo_s, t_hi_s;
  volatile unsigned long long* status =
      reinterpret_cast<volatile unsigned long long*>(v.tile_prefix);  // n_tiles entries, zeroed per run
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) tile_s = atomicAdd(&v.hdr->emit_ticket, 1ull);
    __syncthreads();
    const uint64_t tile = tile_s;
    if (tile >= v.n_tiles) break;
    // warp w takes the tile's words [256 w, 256 w + 256) in kEmitWordsPerThread
    // batches of 32 consecutive words, one word per lane
    const uint64_t tile_base = tile * kEmitTileWords;
    const uint32_t wbase = (uint32_t)wid * 32 * kEmitWordsPerThread;
    uint32_t words[kEmitWordsPerThread];
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < kEmitWordsPerThread; ++q) {
      const uint64_t w = tile_base + wbase + 32 * q + lane;
      words[q] = w < v.bitmap_words ? __ldcg(v.cfinal + w) : 0u;
      c += __popc(words[q]);
    }
    c = warp_sum(c);
    if (lane == 0) warp_s[wid] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kBlock / 32; ++w) {
        const uint32_t x = warp_s[w];
        warp_s[w] = tot;
        tot += x;
      }
      total_s = tot;
      unsigned long long prefix = 0;
      if (tile == 0) {
        status[0] = kFlagPrefix | tot;
      } else {
        status[tile] = kFlagAgg | tot;
        uint64_t j = tile - 1;
        uint32_t spins = 0;
        for (;;) {
          const unsigned long long st = status[j];
          if (st & kFlagPrefix) {
            prefix += st & kValMask;
            break;
          }
          if (st & kFlagAgg) {
            prefix += st & kValMask;
            --j;  // tile 0 only ever holds a prefix, so j stays >= 0
            continue;
          }
          if (++spins > kSpinLimit) {
            v.hdr->timeout = 1;
            break;
          }
          __nanosleep(32);
        }
        status[tile] = kFlagPrefix | (prefix + tot);
      }
      prefix_s = prefix;
    }
    __syncthreads();
    // batch by batch: every lane expands its word into the warp's stage at its
    // exclusive prefix, then the warp writes the batch with consecutive lanes
    // on consecutive entries
    uint32_t at = warp_s[wid];  // junctions of the tile before this batch
    uint16_t* stage = stage_s[wid];
    Bounds bd{1, 0};
#pragma unroll
    for (int q = 0; q < kEmitWordsPerThread; ++q) {
      const uint32_t n = __popc(words[q]);
      uint32_t inc = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t word_at = wbase + 32 * q + lane;  // the word's index within the tile
      before_s[word_at] = at + inc - n;
      uint32_t bits = words[q], i = inc - n;
      while (bits) {
        const uint32_t b = __ffs(bits) - 1;
        bits &= bits - 1;
        stage[i++] = (uint16_t)(word_at * 32 + b);  // below 2^16: a tile is 65536 positions
      }
      const uint32_t batch = __shfl_sync(0xffffffffu, inc, 31);
      __syncwarp();
      const uint64_t o0 = prefix_s + at;
      for (uint32_t e = lane; e < batch; e += 32) {
        const uint64_t g = tile_base * 32 + stage[e];
        if (g < bd.start || g >= bd.end) bd = seq_bounds(v, g);
        if (o0 + e < v.out_capacity) v.out_positions[o0 + e] = g - bd.start;
      }
      __syncwarp();
      at += batch;
    }
    // out_offsets[t] (junctions before string t) for the strings that start in
    // this tile; the last tile also takes t = n_seqs (start m: the total)
    if (threadIdx.x == 0) {
      const uint64_t g_lo = tile_base * 32;
      const uint64_t g_hi = tile + 1 == v.n_tiles ? ~0ull : (tile_base + kEmitTileWords) * 32;
      auto lower = [&](uint64_t g) {  // first t in [0, n_seqs + 1) with offsets[t] >= g
        uint64_t lo = 0, hi = (uint64_t)v.n_seqs + 1;
        while (lo < hi) {
          const uint64_t mid = (lo + hi) >> 1;
          if (__ldg(v.offsets + mid) < g) lo = mid + 1; else hi = mid;
        }
        return lo;
      };
      t_lo_s = lower(g_lo);
      t_hi_s = lower(g_hi);
    }
    __syncthreads();
    for (uint64_t t = t_lo_s + threadIdx.x; t < t_hi_s; t += kBlock) {
      const uint64_t g = __ldg(v.offsets + t), w = g >> 5, j = w - tile_base;
      unsigned long long cnt = prefix_s + (j < (uint64_t)kEmitTileWords ? before_s[j] : total_s);
      if ((g & 31) && w < v.bitmap_words) cnt += __popc(__ldcg(v.cfinal + w) & ((1u << (g & 31)) - 1u));
      v.out_offsets[t] = cnt;
      if (t == v.n_seqs && cnt > v.out_capacity) v.hdr->out_overflow = 1;
    }
    __syncthreads();
  }
}

// offsets[t] = junctions in strings before t (one block per string); the
// last entry is the total, checked against the output's capacity. Only runs
// without input use it: otherwise the emit kernel writes the offsets.
__global__ void __launch_bounds__(kBlock) emit_offsets_kernel(RunView v) {
  const uint64_t t = blockIdx.x;
  const uint64_t g = (t == v.n_seqs) ? v.m : __ldg(v.offsets + t);
  const uint64_t w = g >> 5;
  const uint64_t tile = w / kEmitTileWords;
  unsigned long long cnt = 0;
  for (uint64_t x = tile * kEmitTileWords + threadIdx.x; x < w; x += kBlock) cnt += __popc(__ldcg(v.cfinal + x));
  __shared__ unsigned long long part[kBlock / 32];
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    cnt = 0;
    for (int i = 0; i < kBlock / 32; ++i) cnt += part[i];
    if (tile > 0) cnt += __ldcg(reinterpret_cast<const unsigned long long*>(v.tile_prefix) + (tile - 1)) & kValMask;
    if (g & 31) cnt += __popc(__ldcg(v.cfinal + w) & ((1u << (g & 31)) - 1u));
    v.out_offsets[t] = cnt;
    if (t == v.n_seqs && cnt > v.out_capacity) v.hdr->out_overflow = 1;
  }
}

// ---------------------------------------------------------------------------
// Compacted-graph edges (section "Reduction to the Problem of Finding
// Junction Positions"): consecutive junction positions of a string.
// ---------------------------------------------------------------------------

struct EdgeOut {  // layout of twopaco_edge
  unsigned long long from_hi, from_lo, to_hi, to_lo, start, length;
  unsigned int from_rc, to_rc;
};

// With N splitting no edge crosses an N. Every piece of at least k bases
// holds a junction (its first k-mer is a sentinel), so a string with j
// junctions spread over r such pieces has j - r edges: one fewer per piece.
// run_rank[j] = pieces of at least k bases among runs[0 .. j) (one block).
__global__ void __launch_bounds__(1024) runs_rank_kernel(const DevHeader* hdr) {
  __shared__ unsigned int wsum[32];
  __shared__ unsigned int carry_s;
  if (!hdr->nmask) return;  // the run did not split at N
  const uint64_t n = hdr->n_runs;
  const uint64_t* runs = hdr->runs;
  const uint32_t* nmask = hdr->nmask;
  uint32_t* rank = hdr->run_rank;
  const uint64_t k = (uint64_t)hdr->k;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t base = 0; base < n; base += 1024) {
    const uint64_t j = base + threadIdx.x;
    unsigned int x = 0;
    if (j < n) {
      const uint64_t a = runs[j], b = runs[j + 1];
      x = (!((nmask[a >> 5] >> (a & 31)) & 1u) && b - a >= k) ? 1u : 0u;
    }
    unsigned int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned int before = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      before += (w < wid) ? wsum[w] : 0u;
      all += wsum[w];
    }
    const unsigned int c0 = carry_s;
    if (j < n) rank[j] = c0 + before + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = c0 + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) rank[n] = carry_s;
}

// First j in [0, n] with runs[j] >= g (runs[n] = m).
__device__ __forceinline__ uint64_t runs_lower_bound(const uint64_t* runs, uint64_t n, uint64_t g) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (runs[mid] < g) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Pieces of at least k bases in string t (N splitting).
__device__ __forceinline__ uint64_t long_pieces(const DevHeader* hdr, const uint64_t* offsets, uint64_t t) {
  const uint64_t n = hdr->n_runs;
  const uint64_t lo = runs_lower_bound(hdr->runs, n, offsets[t]);
  const uint64_t hi = runs_lower_bound(hdr->runs, n, offsets[t + 1]);
  return (uint64_t)hdr->run_rank[hi] - hdr->run_rank[lo];
}

// edge_offsets[t] = sum over strings before t of their edges: junctions - 1
// (none for a string without junctions), or junctions - pieces with N splitting.
__global__ void __launch_bounds__(1024) edge_offsets_kernel(const DevHeader* hdr, const uint64_t* offsets,
                                                            const uint64_t* out_off, uint64_t n_seqs,
                                                            uint64_t* edge_off, uint64_t capacity) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const bool split = hdr->nmask != nullptr;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t base = 0; base < n_seqs; base += 1024) {
    const uint64_t t = base + threadIdx.x;
    unsigned long long x = 0;
    if (t < n_seqs) {
      const unsigned long long j = out_off[t + 1] - out_off[t];
      if (split) x = j - long_pieces(hdr, offsets, t);
      else x = j ? j - 1 : 0;
    }
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      before += (w < wid) ? wsum[w] : 0ull;
      all += wsum[w];
    }
    const unsigned long long c0 = carry_s;
    if (t < n_seqs) edge_off[t] = c0 + before + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = c0 + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    edge_off[n_seqs] = carry_s;
    if (carry_s > capacity) const_cast<DevHeader*>(hdr)->overflow = 1;
  }
}

// The normalized k-mer at g (for k > 63 its 128 least significant bits, the
// last 64 bases) and whether the string reads its reverse complement.
template <int KW>
__device__ __forceinline__ void edge_vertex(const uint32_t* packed, uint64_t g, int k, int both,
                                            unsigned long long* hi, unsigned long long* lo,
                                            unsigned int* rc) {
  const KeyT<KW> f = load_kmer<KW>(packed, g, k);
  const KeyT<KW> r = both ? revcomp<KW>(f, k) : f;
  const bool use_r = both && key_less(r, f);
  const KeyT<KW>& x = use_r ? r : f;
  if constexpr (KW == 4) {
    *hi = x.w[2];
    *lo = x.w[3];
  } else {
    *hi = x.hi;
    *lo = x.lo;
  }
  *rc = use_r ? 1u : 0u;
}

// One thread per junction: the edge from it to the next junction of its
// string (with N splitting: of its piece; the last junction of a piece has
// none, and the edges of later pieces move down by one per earlier piece).
__global__ void __launch_bounds__(kBlock) edges_kernel(const DevHeader* hdr, const uint64_t* offsets,
                                                      uint64_t n_seqs, const uint64_t* out_off,
                                                      const uint64_t* out_pos, const uint64_t* edge_off,
                                                      EdgeOut* edges, uint64_t capacity) {
  const uint32_t* packed = hdr->packed;
  const int k = hdr->k, both = hdr->both;
  const bool split = hdr->nmask != nullptr;
  const uint64_t total = out_off[n_seqs];
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < total; i += stride) {
    uint64_t lo = 0, hi = n_seqs;  // largest t with out_off[t] <= i
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (__ldg(out_off + mid) <= i) lo = mid; else hi = mid;
    }
    const uint64_t t = lo;
    const uint64_t a = i - out_off[t];
    if (a + 1 >= out_off[t + 1] - out_off[t]) continue;  // the string's last junction
    const uint64_t p = out_pos[i], q = out_pos[i + 1], g0 = offsets[t];
    uint64_t e = edge_off[t] + a;
    if (split) {
      const uint64_t n = hdr->n_runs;
      const uint64_t jr = runs_lower_bound(hdr->runs, n, g0 + p + 1) - 1;  // the piece holding p
      if (hdr->runs[jr + 1] < g0 + q + (uint64_t)k) continue;            // q lies in a later piece
      const uint64_t first = runs_lower_bound(hdr->runs, n, g0);
      e -= (uint64_t)hdr->run_rank[jr] - hdr->run_rank[first];
    }
    if (e >= capacity) continue;
    EdgeOut o;
    if (k <= 31) {
      edge_vertex<1>(packed, g0 + p, k, both, &o.from_hi, &o.from_lo, &o.from_rc);
      edge_vertex<1>(packed, g0 + q, k, both, &o.to_hi, &o.to_lo, &o.to_rc);
    } else if (k <= 63) {
      edge_vertex<2>(packed, g0 + p, k, both, &o.from_hi, &o.from_lo, &o.from_rc);
      edge_vertex<2>(packed, g0 + q, k, both, &o.to_hi, &o.to_lo, &o.to_rc);
    } else {
      edge_vertex<4>(packed, g0 + p, k, both, &o.from_hi, &o.from_lo, &o.from_rc);
      edge_vertex<4>(packed, g0 + q, k, both, &o.to_hi, &o.to_lo, &o.to_rc);
    }
    o.start = p;
    o.length = q - p;
    edges[e] = o;
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Grid of at most (SMs x resident blocks per SM) blocks for work_items threads.
template <typename K>
unsigned grid_for(K kernel, int block, uint64_t work_items, int cap_per_sm = 0, size_t dyn_smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, dyn_smem);
  if (cap_per_sm > 0 && per_sm > cap_per_sm) per_sm = cap_per_sm;  // a chosen launch shape
  if (per_sm < 1) per_sm = 1;
  const uint64_t full = (uint64_t)sm_count() * per_sm;
  const uint64_t need = (work_items + block - 1) / block;
  return (unsigned)(need < full ? (need ? need : 1) : full);
}

int done(int n) {
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  count_launches(n);
  return n;
}

}  // namespace

#ifndef TWOPACO_WIDE_ONLY
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n); }
unsigned long long launches_so_far() { return g_launches.load(); }

int launch_init(const RunView& v, cudaStream_t s) {
  return cudaMemsetAsync(v.hdr, 0, sizeof(DevHeader), s) == cudaSuccess ? 0 : -1;
}

int launch_digest(DevHeader* hdr_dev, const uint32_t* packed, uint64_t words, const uint64_t* offsets,
                  uint64_t n_seqs, const uint32_t* nmask, uint64_t nmask_words, cudaStream_t s) {
  if (cudaMemsetAsync(&hdr_dev->input_digest, 0, sizeof(unsigned long long), s) != cudaSuccess) return -1;
  digest_kernel<<<grid_for(digest_kernel, kBlock, words), kBlock, 0, s>>>(hdr_dev, packed, words, offsets,
                                                                         n_seqs + 1, nmask, nmask_words);
  return done(1);
}

int launch_pack(const RunView& v, cudaStream_t s) {
  if (launch_pack_chunk(v, 0, v.packed_words, true, s) < 0) return -1;
  return launch_pack_finish(v, s);
}

int launch_pack_chunk(const RunView& v, uint64_t w_begin, uint64_t w_end, bool first, cudaStream_t s) {
  Timed t("pack", s);
  pack_kernel<<<grid_for(pack_kernel, kBlock, (w_end - w_begin + 3) / 4), kBlock, 0, s>>>(v, w_begin, w_end,
                                                                                          first ? 1 : 0);
  return done(1);
}

int launch_pack_finish(const RunView& v, cudaStream_t s) {
  if (!v.nmask || v.m == 0) return 0;
  {
    Timed t("runs", s);
    runs_mark_kernel<<<grid_for(runs_mark_kernel, kBlock, v.bitmap_words), kBlock, 0, s>>>(v);
    runs_starts_kernel<<<grid_for(runs_starts_kernel, kBlock, v.n_seqs), kBlock, 0, s>>>(v);
    const unsigned gc = grid_for(runs_count_kernel, kBlock, v.n_chunks * kBlock);
    runs_count_kernel<<<gc, kBlock, 0, s>>>(v);
    runs_scan_kernel<<<1, 1024, 0, s>>>(v);
    runs_write_kernel<<<grid_for(runs_write_kernel, kBlock, v.n_chunks * kBlock), kBlock, 0, s>>>(v);
  }
  return done(5);
}

#endif  // TWOPACO_WIDE_ONLY

// Run f with the filter's bits per item as a compile-time constant.
template <typename F>
void with_hashes(int h, F&& f) {
  switch (h) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    default: f(std::integral_constant<int, 8>{}); break;
  }
}

#ifndef TWOPACO_WIDE_ONLY
int launch_partition(const RunView& v, int rounds, cudaStream_t s) {
  if (v.m == 0) return 0;
  // the filter is clear (pack kernel); the pre-pass uses it, round 0 clears it again
  if (cudaMemsetAsync(v.bins, 0, (uint64_t)(v.qmask + 1u) * 4, s) != cudaSuccess) return -1;
  const uint64_t threads = (v.m + kR - 1) / kR;
  {
    Timed t("partition_count", s);
    if (v.k > 63) {
      if (launch_partition_count_wide(v, s) < 0) return -1;
    } else {
      with_hashes(v.hashes, [&](auto hb) {
        constexpr int HB = decltype(hb)::value;
        if (v.k <= 31)
          partition_count_kernel<1, HB><<<grid_for(partition_count_kernel<1, HB>, kBlock, threads), kBlock, 0, s>>>(v);
        else
          partition_count_kernel<2, HB><<<grid_for(partition_count_kernel<2, HB>, kBlock, threads), kBlock, 0, s>>>(v);
      });
    }
  }
  uint64_t* prefix = reinterpret_cast<uint64_t*>(v.bins + (v.qmask + 1u));
  {
    Timed t("partition_cut", s);
    partition_cut_kernel<<<1, 1024, 0, s>>>(v, rounds, prefix);
  }
  return done(2);
}
#endif  // TWOPACO_WIDE_ONLY

template <int KW, bool RD, int HB, int TS>
int round_impl(const RunView& v, int round, cudaStream_t s, const Ranges* ranges) {
  // the pack kernel cleared the filter and the LC bitmap for round 0; the
  // partition pre-pass (rounds > 1) uses the filter before round 0
  if (RD && cudaMemsetAsync(v.filter, 0, v.filter_words64 * 8, s) != cudaSuccess) return -1;
  if (round > 0 && cudaMemsetAsync(v.lc_bits, 0, (1ull << v.lc_log2) / 8, s) != cudaSuccess) return -1;
  constexpr bool kDescOk = HB <= 6;
  const bool cm = RD && v.cmap != nullptr;  // rounds visit only their class's positions
  const bool desc = !cm && kDescOk && v.use_desc;
  // every loop over all positions at once, or once per string (ranges)
  const Ranges whole{{v.p_begin, v.p_end}};
  const Ranges& rs = ranges ? *ranges : whole;
  auto part = [&](const std::pair<uint64_t, uint64_t>& r) {
    RunView x = v;
    x.p_begin = r.first;
    x.p_end = r.second;
    return x;
  };
  int launched = 0;
  // filters beyond L2: the region-ordered first pass (class-map rounds), or
  // region buckets for the inserts alone, chunk by chunk
  constexpr bool kBktOk = HB <= 6;  // a record carries the bit bases of up to 6 bits per item
  constexpr int HBO = kBktOk ? HB : 1;
  const bool bkt = kBktOk && v.n_regions > 0;
  const bool ord = kBktOk && cm && v.o_regions > 0 && !ranges;
  const bool fused = ord && v.o_fused;
  if (ord) {
    {
      Timed t("ord_scatter", s);
      const uint64_t chunks = (v.o_tiles + kOrdScanTiles - 1) / kOrdScanTiles;
      ord_room_sum_kernel<<<(unsigned)chunks, kBlock, 0, s>>>(v, round);
      ord_room_prefix_kernel<<<v.o_regions, kBlock, 0, s>>>(v, chunks);
      ord_room_scan_kernel<<<(unsigned)chunks, kBlock, 0, s>>>(v, round);
      ord_setup_kernel<<<1, kBlock, 0, s>>>(v, round);
      const uint64_t tiles = (v.p_end - v.p_begin + kOrdTile - 1) / kOrdTile;
      auto kern = ord_scatter_kernel<KW, HBO, false>;
      if constexpr (KW == 1)
        if (fused) kern = ord_scatter_kernel<KW, HBO, true>;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOrdStageBytes) !=
          cudaSuccess)
        return -1;
      kern<<<grid_for(kern, kBlock, tiles * kBlock, v.blocks_per_sm, kOrdStageBytes), kBlock, kOrdStageBytes, s>>>(
          v, round);
    }
    {
      Timed t("ord_or", s);
      auto kern = fused ? ord_or_kernel<HBO, true> : ord_or_kernel<HBO, false>;
      kern<<<grid_for(kern, kBlock, ~0ull >> 1), kBlock, 0, s>>>(v);
    }
    launched += 6;
  }
  {
    for (const auto& r : rs) {
      const uint64_t step = bkt ? v.bucket_chunk : r.second - r.first;
      for (uint64_t c0 = r.first; c0 < r.second; c0 += step) {
        const RunView x = part({c0, std::min(r.second, c0 + step)});
        const uint64_t threads = (x.p_end - x.p_begin + kInsertR - 1) / kInsertR;
        {
        Timed t("pass1_insert", s);
        if (bkt && cudaMemsetAsync(v.bucket_fill, 0, ((uint64_t)v.n_regions * v.n_sub + 1) * kFillStride * 4,
                                   s) != cudaSuccess)
          return -1;
        if (cm && bkt)
          pass1_insert_cm_kernel<KW, HB, kBktOk><<<grid_for(pass1_insert_cm_kernel<KW, HB, kBktOk>, kBlock, threads, v.blocks_per_sm),
                                                   kBlock, 0, s>>>(x, round);
        else if (cm)
          pass1_insert_cm_kernel<KW, HB><<<grid_for(pass1_insert_cm_kernel<KW, HB>, kBlock, threads, v.blocks_per_sm), kBlock, 0,
                                           s>>>(x, round);
        else if (desc && bkt)
          pass1_insert_kernel<KW, RD, HB, kDescOk, kBktOk>
              <<<grid_for(pass1_insert_kernel<KW, RD, HB, kDescOk, kBktOk>, kBlock, threads, v.blocks_per_sm), kBlock, 0, s>>>(x, round);
        else if (desc)
          pass1_insert_kernel<KW, RD, HB, kDescOk><<<grid_for(pass1_insert_kernel<KW, RD, HB, kDescOk>, kBlock,
                                                              threads),
                                                     kBlock, 0, s>>>(x, round);
        else if (bkt)
          pass1_insert_kernel<KW, RD, HB, false, kBktOk>
              <<<grid_for(pass1_insert_kernel<KW, RD, HB, false, kBktOk>, kBlock, threads, v.blocks_per_sm), kBlock, 0, s>>>(x, round);
        else
          pass1_insert_kernel<KW, RD, HB, false><<<grid_for(pass1_insert_kernel<KW, RD, HB, false>, kBlock, threads, v.blocks_per_sm),
                                                   kBlock, 0, s>>>(x, round);
        }
        ++launched;
        if (bkt) {
          Timed ta("filter_apply", s);
          filter_apply_kernel<kBktOk ? HB : 1><<<grid_for(filter_apply_kernel<kBktOk ? HB : 1>, kBlock, ~0ull >> 1),
                                                 kBlock, 0, s>>>(v);
          ++launched;
        }
      }
    }
  }
  RunView pv = v;
  for (const auto& r : rs) {
    pv = part(r);
    const uint64_t threads = (r.second - r.first + kProbeR - 1) / kProbeR;
    // one candidate-list segment per probe warp
    unsigned grid = cm     ? grid_for(pass1_probe_cm_kernel<KW, HB>, kBlock, (r.second - r.first + 15) / 16, v.blocks_per_sm)
                    : desc ? grid_for(pass1_probe_desc_kernel<kDescOk ? HB : 1>, kBlock, threads, v.blocks_per_sm)
                           : grid_for(pass1_probe_kernel<KW, RD, HB>, kBlock, threads, v.blocks_per_sm);
    if (grid * (kBlock / 32) > kMaxSegments) grid = kMaxSegments / (kBlock / 32);
    pv.n_segments = grid * (kBlock / 32);
    // the list region holds cand_cap 8-byte records, or twice as many 32-bit
    // ones; launched per string there is no list (pass 2 walks C_temp)
    pv.seg_cap = ranges ? 0 : (v.narrow ? 2 * v.cand_cap : v.cand_cap) / pv.n_segments;
    if (ord) {  // the gather's warps own the list segments, as the probe's would
      if (fused && cudaMemsetAsync(v.table, 0xFF, (uint64_t)v.o_tcap * v.o_regions * 8, s) != cudaSuccess)
        return -1;  // every fused table slot empty (all ones)
      {
        Timed t("ord_probe", s);
        auto kern = fused ? ord_probe_kernel<HBO, true> : ord_probe_kernel<HBO, false>;
        kern<<<grid_for(kern, kBlock, ~0ull >> 1), kBlock, 0, s>>>(v);
      }
      if (fused) {
        Timed t("ord_classify", s);
        ord_classify_kernel<<<grid_for(ord_classify_kernel, kBlock, ~0ull >> 1), kBlock, 0, s>>>(v);
        ++launched;
      }
      {
        Timed t("ord_gather", s);
        ord_gather_kernel<<<grid, kBlock, 0, s>>>(pv, round);
      }
      launched += 2;
    }
    Timed t("pass1_probe", s);
    if (cm) pass1_probe_cm_kernel<KW, HB><<<grid, kBlock, 0, s>>>(pv, round);
    else if (desc) pass1_probe_desc_kernel<kDescOk ? HB : 1><<<grid, kBlock, 0, s>>>(pv, round);
    else pass1_probe_kernel<KW, RD, HB><<<grid, kBlock, 0, s>>>(pv, round);
    ++launched;
  }
  if (v.partial) return done(launched);  // the partially compacted graph: no second pass
  {
    Timed t("table_setup", s);
    table_setup_kernel<<<grid_for(table_setup_kernel, kBlock, (1ull << v.lc_log2) / 32), kBlock, 0, s>>>(pv);
  }
  {
    Timed t("table_clear", s);
    table_clear_kernel<TS><<<grid_for(table_clear_kernel<TS>, kBlock, v.table_max_slots), kBlock, 0, s>>>(pv);
  }
  launched += 2;
  // pass 2: one resident wave; the warps share out the list's segment parts
  const unsigned g2 = grid_for(pass2_insert_kernel<KW, TS>, kBlock, ~0ull >> 1, v.blocks_per_sm);
  const unsigned g3 = grid_for(pass2_classify_kernel<KW, TS>, kBlock, ~0ull >> 1, v.blocks_per_sm);
  {
    Timed t("pass2_insert", s);
    for (const auto& r : rs) {
      RunView x = part(r);
      x.n_segments = pv.n_segments;
      x.seg_cap = pv.seg_cap;
      pass2_insert_kernel<KW, TS><<<g2, kBlock, 0, s>>>(x);
      ++launched;
    }
  }
  {
    Timed t("pass2_classify", s);
    for (const auto& r : rs) {
      RunView x = part(r);
      x.n_segments = pv.n_segments;
      x.seg_cap = pv.seg_cap;
      pass2_classify_kernel<KW, TS><<<g3, kBlock, 0, s>>>(x);
      ++launched;
    }
  }
  return done(launched);
}

#ifndef TWOPACO_WIDE_ONLY
int launch_round(const RunView& v, int round, int rounds, cudaStream_t s, const Ranges* ranges) {
  if (v.m == 0) return 0;
  if (v.k > 63) return launch_round_wide(v, round, rounds, s, ranges);
  int rc = 0;
  with_hashes(v.hashes, [&](auto hb) {
    constexpr int HB = decltype(hb)::value;
    const int ts = table_slot_kind(v.k);
    if (ts == 0)
      rc = rounds > 1 ? round_impl<1, true, HB, 0>(v, round, s, ranges) : round_impl<1, false, HB, 0>(v, round, s, ranges);
    else if (ts == 1)
      rc = rounds > 1 ? round_impl<1, true, HB, 1>(v, round, s, ranges) : round_impl<1, false, HB, 1>(v, round, s, ranges);
    else
      rc = rounds > 1 ? round_impl<2, true, HB, 2>(v, round, s, ranges) : round_impl<2, false, HB, 2>(v, round, s, ranges);
  });
  return rc;
}

int launch_class_map(const RunView& v, cudaStream_t s) {
  if (!v.cmap || v.m == 0) return 0;
  if (v.k > 63) return launch_class_map_wide(v, s) < 0 ? -1 : done(1);
  Timed t("class_map", s);
  const uint64_t threads = (v.m + kInsertR - 1) / kInsertR;
  if (v.o_regions) {
    const unsigned grid = v.k <= 31 ? grid_for(class_map_ord_kernel<1>, kBlock, v.o_tiles * kBlock)
                                    : grid_for(class_map_ord_kernel<2>, kBlock, v.o_tiles * kBlock);
    if (v.k <= 31) class_map_ord_kernel<1><<<grid, kBlock, 0, s>>>(v);
    else class_map_ord_kernel<2><<<grid, kBlock, 0, s>>>(v);
    // every tile's first member number, per round
    const uint64_t chunks = (v.o_tiles + kOrdScanTiles - 1) / kOrdScanTiles;
    ord_tile_sum_kernel<<<(unsigned)(chunks * v.rounds), kBlock, 0, s>>>(v, chunks);
    ord_tile_scan_kernel<<<(unsigned)(chunks * v.rounds), kBlock, 0, s>>>(v, chunks);
    return done(3);
  }
  if (v.k <= 31) class_map_kernel<1><<<grid_for(class_map_kernel<1>, kBlock, threads), kBlock, 0, s>>>(v);
  else class_map_kernel<2><<<grid_for(class_map_kernel<2>, kBlock, threads), kBlock, 0, s>>>(v);
  return done(1);
}

int launch_emit(const RunView& v, cudaStream_t s, bool again) {
  // again: a second emit of the same run (into a larger output): its tile
  // tickets, tile status and output flag start over
  if (again && (cudaMemsetAsync(v.tile_prefix, 0, (v.n_tiles + 1) * 8, s) != cudaSuccess ||
                cudaMemsetAsync(&v.hdr->emit_ticket, 0, sizeof(unsigned long long), s) != cudaSuccess ||
                cudaMemsetAsync(&v.hdr->out_overflow, 0, sizeof(unsigned int), s) != cudaSuccess))
    return -1;
  if (v.n_tiles) {  // tile status cleared by the pack kernel; writes the offsets too
    Timed t("emit", s);
    emit_kernel<<<grid_for(emit_kernel, kBlock, v.n_tiles * kBlock), kBlock, 0, s>>>(v);
  } else {  // no input: every offset is 0
    Timed t("emit_offsets", s);
    emit_offsets_kernel<<<(unsigned)(v.n_seqs + 1), kBlock, 0, s>>>(v);
  }
  return done(1);
}

int launch_edges(const DevHeader* hdr_dev, const uint64_t* d_offsets, uint64_t n_seqs,
                 const uint64_t* d_out_offsets, const uint64_t* d_out_positions,
                 uint64_t* d_edge_offsets, void* d_edges, uint64_t edge_capacity, cudaStream_t s) {
  // the piece ranks, when the run split its strings at N (the kernel reads the
  // header and returns at once otherwise)
  {
    Timed t("edge_offsets", s);
    runs_rank_kernel<<<1, 1024, 0, s>>>(hdr_dev);
    edge_offsets_kernel<<<1, 1024, 0, s>>>(hdr_dev, d_offsets, d_out_offsets, n_seqs, d_edge_offsets,
                                           edge_capacity);
  }
  {
    Timed t("edges", s);
    edges_kernel<<<grid_for(edges_kernel, kBlock, 1ull << 30), kBlock, 0, s>>>(
        hdr_dev, d_offsets, n_seqs, d_out_offsets, d_out_positions, d_edge_offsets,
        static_cast<EdgeOut*>(d_edges), edge_capacity);
  }
  return done(3);
}

#else
// k > 63: four-word k-mers, reference slots, the bits per item a run-time value.
int launch_round_wide(const RunView& v, int round, int rounds, cudaStream_t s, const Ranges* ranges) {
  return rounds > 1 ? round_impl<4, true, 0, 3>(v, round, s, ranges) : round_impl<4, false, 0, 3>(v, round, s, ranges);
}

int launch_partition_count_wide(const RunView& v, cudaStream_t s) {
  const uint64_t threads = (v.m + kR - 1) / kR;
  partition_count_kernel<4, 0><<<grid_for(partition_count_kernel<4, 0>, kBlock, threads), kBlock, 0, s>>>(v);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_class_map_wide(const RunView& v, cudaStream_t s) {
  Timed t("class_map", s);
  const uint64_t threads = (v.m + kInsertR - 1) / kInsertR;
  class_map_kernel<4><<<grid_for(class_map_kernel<4>, kBlock, threads), kBlock, 0, s>>>(v);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
#endif  // TWOPACO_WIDE_ONLY

}  // namespace twopaco

#ifndef TWOPACO_WIDE_ONLY

extern "C" unsigned long long twopaco_kernel_launches(void) {
  return twopaco::g_launches.load();
}

extern "C" int twopaco_profile_enable(int on) {
  using namespace twopaco;
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto& r : g_prof) {
    g_event_pool.push_back(r.start);
    g_event_pool.push_back(r.stop);
  }
  g_prof.clear();
  g_prof_on = on != 0;
  return 0;
}

extern "C" int twopaco_profile_kernels(const char** names, unsigned long long* launches,
                                       double* total_ms, int capacity) {
  using namespace twopaco;
  std::lock_guard<std::mutex> g(g_prof_mu);
  std::vector<std::string> seen;
  std::vector<unsigned long long> cnt;
  std::vector<double> ms;
  std::vector<const char*> ptr;
  for (auto& r : g_prof) {
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return -5;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) return -5;
    size_t i = 0;
    while (i < seen.size() && seen[i] != r.name) ++i;
    if (i == seen.size()) {
      seen.push_back(r.name);
      ptr.push_back(r.name);
      cnt.push_back(0);
      ms.push_back(0.0);
    }
    cnt[i] += 1;
    ms[i] += t;
  }
  const int n = (int)seen.size();
  for (int i = 0; i < n && i < capacity; ++i) {
    if (names) names[i] = ptr[i];
    if (launches) launches[i] = cnt[i];
    if (total_ms) total_ms[i] = ms[i];
  }
  return n;
}

#endif  // TWOPACO_WIDE_ONLY
