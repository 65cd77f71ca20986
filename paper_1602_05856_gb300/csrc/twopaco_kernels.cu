// CUDA kernels of the junction-detection library (sm_103a).
//
// One run = pack, then per round (Algorithm 3, section "Multiple Rounds")
// the two passes of Algorithm 2 (Filter-Junctions-Two-Pass), each an
// instance of Algorithm 1 (Filter-Junctions): an insert loop and a probe
// loop over every position, separated by a kernel boundary (the barrier of
// section "Parallelization Scheme"); then one emit of the junction
// positions. Every kernel walks positions with one thread per position, so a
// warp covers 32 consecutive positions and its ballot is one bitmap word.
//
// Encoding: A,C,G,T = 0,1,2,3, 16 bases per 32-bit word, first base in the
// two most significant bits. A k-mer is the integer with its first base most
// significant, so integer order is lexicographic order (the normalized form
// of a k-mer is min(k-mer, reverse complement)), and complement is 3 - x.
#include "twopaco_internal.h"

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

namespace twopaco {

constexpr int TWOPACO_ECUDA_INTERNAL = -5;

namespace {

std::atomic<unsigned long long> g_launches{0};

// Optional per-kernel timing: CUDA events recorded on the launch stream
// right before and after every kernel.
struct ProfRecord {
  const char* name;
  cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_prof;
std::vector<cudaEvent_t> g_event_pool;

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
  Timed(const char* name, cudaStream_t st) : s(st) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on) return;
    rec.name = name;
    rec.start = take_event();
    rec.stop = take_event();
    cudaEventRecord(rec.start, s);
  }
  ~Timed() {
    if (!rec.name) return;
    cudaEventRecord(rec.stop, s);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back(rec);
  }
};

// ---------------------------------------------------------------------------
// k-mer words
// ---------------------------------------------------------------------------

struct Key {
  uint64_t hi, lo;  // value = hi * 2^64 + lo; hi == 0 for k <= 31
};

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
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

// Reverse the order of the 32 two-bit groups of x.
__device__ __forceinline__ uint64_t rev_pairs(uint64_t x) {
  const uint64_t b = __brevll(x);
  return ((b >> 1) & 0x5555555555555555ull) | ((b & 0x5555555555555555ull) << 1);
}

__device__ __forceinline__ uint32_t base_at(const uint32_t* __restrict__ packed, uint64_t g) {
  return (__ldg(packed + (g >> 4)) >> (30u - 2u * (uint32_t)(g & 15))) & 3u;
}

// The k-mer starting at base g and the base right after it. KW = 1 for
// k <= 31 (one 64-bit word), 2 for 32 <= k <= 63.
template <int KW>
__device__ __forceinline__ Key load_kmer(const uint32_t* __restrict__ packed, uint64_t g, int k,
                                         uint32_t* succ) {
  const uint32_t* p = packed + (g >> 4);
  const uint32_t o2 = 2u * (uint32_t)(g & 15);
  const uint32_t w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2);
  uint64_t a = ((uint64_t)w0 << 32) | w1;  // bases 16w .. 16w+31
  if (o2) a = (a << o2) | (w2 >> (32u - o2));  // bases g .. g+31
  Key v;
  if (KW == 1) {
    v.hi = 0;
    v.lo = a >> (64 - 2 * k);
    *succ = (uint32_t)(a >> (62 - 2 * k)) & 3u;
  } else {
    const uint32_t w3 = __ldg(p + 3), w4 = __ldg(p + 4);
    uint64_t b = ((uint64_t)w2 << 32) | w3;
    if (o2) b = (b << o2) | (w4 >> (32u - o2));  // bases g+32 .. g+63
    const int sh = 128 - 2 * k;                  // 2 .. 64
    if (sh == 64) {
      v.hi = 0;
      v.lo = a;
    } else {
      v.hi = a >> sh;
      v.lo = (b >> sh) | (a << (64 - sh));
    }
    *succ = (uint32_t)(b >> (62 - 2 * (k - 32))) & 3u;
  }
  return v;
}

// Reverse complement of a k-mer.
template <int KW>
__device__ __forceinline__ Key revcomp(const Key& v, int k) {
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

template <int KW>
__device__ __forceinline__ uint64_t key_hash(const Key& v) {
  return KW == 1 ? mix64(v.lo) : mix64(v.lo ^ mix64(v.hi));
}

__device__ __forceinline__ uint64_t second_hash(uint64_t H) { return mix64(H ^ 0x9e3779b97f4a7c15ull); }

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

// One k-mer occurrence, read in the orientation of its normalized form.
struct Occ {
  Key key;         // normalized k-mer
  uint64_t H;      // key_hash(key)
  uint32_t items;  // filter items this occurrence inserts (bit j = item j)
  uint32_t tbits;  // pass-2 bits: in-bases 0-3, out-bases 4-7, sentinel 8
  bool sentinel;   // first or last k-mer of its string
};

template <int KW>
__device__ __forceinline__ bool read_occurrence(const RunView& v, uint64_t g, Occ* oc) {
  const Bounds b = seq_bounds(v, g);
  if (g + (uint64_t)v.k > b.end) return false;  // no k-mer starts here
  uint32_t succ;
  const Key f = load_kmer<KW>(v.packed, g, v.k, &succ);
  const bool has_pred = g > b.start, has_succ = g + (uint64_t)v.k < b.end;
  const uint32_t pred = has_pred ? base_at(v.packed, g - 1) : 0u;
  const Key r = v.both ? revcomp<KW>(f, v.k) : f;
  const bool use_f = !v.both || !key_less(r, f);  // f is the normalized form
  const bool use_r = v.both && !key_less(f, r);   // r is (palindromes: both)
  oc->key = use_f ? f : r;
  oc->H = key_hash<KW>(oc->key);
  oc->sentinel = !has_pred || !has_succ;
  if (oc->sentinel) {
    oc->items = 1u << 16;
    oc->tbits = 1u << 8;
  } else {
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
    oc->items = items;
    oc->tbits = tb;
  }
  return true;
}

__device__ __forceinline__ bool in_round(const RunView& v, uint64_t H, int round) {
  const uint32_t bin = (uint32_t)H & v.qmask;
  return bin >= __ldg(v.cuts + round) && bin < __ldg(v.cuts + round + 1);
}

// ---------------------------------------------------------------------------
// Split-block filter: a block is one 32-byte sector of eight 32-bit words.
// A k-mer picks a block (top bits of H), an even first word o and, for each
// of its h words, a bit base; item j sets bit (base + j) & 31 of each word.
// All 17 items of one k-mer therefore sit in one sector: one load answers
// every probe of the k-mer, and an insert is at most ceil(h/2) 64-bit ORs.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t salt(int u) {
  // First 32 fractional bits of the cube roots of 2, 3, 5, 7, 11, 13, 17, 19,
  // made odd.
  constexpr uint32_t s[8] = {0x428a2f99u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u,
                             0x3956c25bu, 0x59f111f1u, 0x923f82a5u, 0xab1c5ed5u};
  return s[u];
}

struct Spot {
  unsigned long long* blk;  // the block's four 64-bit words
  uint32_t o2;              // first logical 64-bit pair (word o = 2 * o2)
  uint32_t base[8];
};

__device__ __forceinline__ Spot filter_spot(const RunView& v, uint64_t H) {
  Spot s;
  const uint64_t G = second_hash(H);
  const uint64_t block = v.lg_blocks ? (H >> (64 - v.lg_blocks)) : 0ull;
  s.blk = v.filter + block * 4;
  s.o2 = (uint32_t)(G >> 62);
  const uint32_t g32 = (uint32_t)G;
#pragma unroll
  for (int u = 0; u < 8; ++u) s.base[u] = (g32 * salt(u)) >> 27;
  return s;
}

// Bits of item j in logical 64-bit pair U (logical words 2U and 2U+1).
__device__ __forceinline__ uint64_t item_bits(const Spot& s, int U, uint32_t j, int h) {
  uint64_t m = 0;
  if (2 * U < h) m |= 1ull << ((s.base[2 * U] + j) & 31u);
  if (2 * U + 1 < h) m |= (1ull << ((s.base[2 * U + 1] + j) & 31u)) << 32;
  return m;
}

__device__ __forceinline__ uint64_t pick4(const uint64_t P[4], uint32_t i) {
  const uint64_t x = (i & 1) ? P[1] : P[0];
  const uint64_t y = (i & 1) ? P[3] : P[2];
  return (i & 2) ? y : x;
}

__device__ __forceinline__ void load_block(const unsigned long long* blk, uint64_t P[4]) {
  const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2*>(blk));
  const ulonglong2 b = __ldcg(reinterpret_cast<const ulonglong2*>(blk) + 1);
  P[0] = a.x;
  P[1] = a.y;
  P[2] = b.x;
  P[3] = b.y;
}

// Bit j of the result: item j is present (all of its h bits are set).
__device__ __forceinline__ uint32_t present_items(const Spot& s, const uint64_t P[4], int h) {
  uint32_t pres = 0x1FFFFu;
#pragma unroll
  for (int U = 0; U < 4; ++U) {
    if (2 * U < h) {
      const uint64_t L = pick4(P, (s.o2 + U) & 3u);
      const uint32_t lo = (uint32_t)L, hi = (uint32_t)(L >> 32);
      pres &= __funnelshift_r(lo, lo, s.base[2 * U]);
      if (2 * U + 1 < h) pres &= __funnelshift_r(hi, hi, s.base[2 * U + 1]);
    }
  }
  return pres & 0x1FFFFu;
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

// Insert (key, bits); false if every slot was tried (the table is full).
template <int KW>
__device__ __forceinline__ bool table_insert(const RunView& v, uint64_t cap, const Key& key,
                                             uint64_t G, uint32_t bits) {
  const uint64_t mask = cap - 1;
  uint64_t i = G & mask;
  for (uint64_t probe = 0; probe < cap; ++probe, i = (i + 1) & mask) {
    unsigned int* mword;
    if (KW == 1) {
      Slot1* s = static_cast<Slot1*>(v.table) + i;
      unsigned long long cur = __ldcg(&s->key);
      if (cur == kEmpty) {
        cur = atomicCAS(&s->key, kEmpty, (unsigned long long)key.lo);
        if (cur == kEmpty) cur = key.lo;
      }
      if (cur != key.lo) continue;
      mword = &s->mask;
    } else {
      Slot2* s = static_cast<Slot2*>(v.table) + i;
      uint64_t ol, oh;
      cas128(&s->w0, kEmpty, kEmpty, key.lo, key.hi, &ol, &oh);
      const bool mine = (ol == kEmpty && oh == kEmpty) || (ol == key.lo && oh == key.hi);
      if (!mine) continue;
      mword = &s->mask;
    }
    if ((__ldcg(mword) & bits) != bits) atomicOr(mword, bits);
    return true;
  }
  return false;
}

// Mask of key, or -1 if absent.
template <int KW>
__device__ __forceinline__ int table_find(const RunView& v, uint64_t cap, const Key& key, uint64_t G) {
  const uint64_t mask = cap - 1;
  uint64_t i = G & mask;
  for (uint64_t probe = 0; probe < cap; ++probe, i = (i + 1) & mask) {
    if (KW == 1) {
      const Slot1* s = static_cast<const Slot1*>(v.table) + i;
      const unsigned long long cur = __ldcg(&s->key);
      if (cur == key.lo) return (int)__ldcg(&s->mask);
      if (cur == kEmpty) return -1;
    } else {
      const Slot2* s = static_cast<const Slot2*>(v.table) + i;
      const ulonglong2 w = __ldcg(reinterpret_cast<const ulonglong2*>(&s->w0));
      if (w.x == key.lo && w.y == key.hi) return (int)__ldcg(&s->mask);
      if (w.x == kEmpty && w.y == kEmpty) return -1;
    }
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Block reductions (blockDim.x == kBlock)
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Exclusive scan of x over the block; *total receives the block sum.
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

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

__global__ void init_kernel(RunView v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevHeader* h = v.hdr;
    h->bad_index = ~0ull;
    h->positions = 0;
    h->pass1_kept = 0;
    h->pass2_kept = 0;
    h->round_kept = 0;
    h->table_slots = 0;
    h->table_max = 0;
    h->overflow = 0;
    h->timeout = 0;
    h->ctemp = v.ctemp;
    h->cfinal = v.cfinal;
    h->bins = v.bins;
    h->cuts = v.cuts;
    h->bitmap_words = v.bitmap_words;
    h->q = (unsigned long long)v.qmask + 1ull;
    h->rounds = (unsigned long long)v.rounds;
    if (v.cuts) {  // one class holding every bin until the partition step runs
      v.cuts[0] = 0;
      v.cuts[1] = v.qmask + 1u;
    }
  }
}

// Four ASCII bytes -> four 2-bit codes (first byte in bits 7-6); *bad gets
// 0xFF in every byte that is not one of ACGTacgt.
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t* bad) {
  const uint32_t low = x | 0x20202020u;
  const uint32_t ok = __vcmpeq4(low, 0x61616161u) | __vcmpeq4(low, 0x63636363u) |
                      __vcmpeq4(low, 0x67676767u) | __vcmpeq4(low, 0x74747474u);
  *bad = ~ok;
  // a=0x61 c=0x63 g=0x67 t=0x74: bits 2-1 are 00 01 11 10; fold to 0 1 2 3
  const uint32_t t = (low >> 1) & 0x03030303u;
  const uint32_t c = t ^ ((t >> 1) & 0x01010101u);
  return ((c & 3u) << 6) | (((c >> 8) & 3u) << 4) | (((c >> 16) & 3u) << 2) | ((c >> 24) & 3u);
}

// Section 8(a) step a0: ASCII -> 2-bit words, 16 bytes (one 128-bit load) per thread.
__global__ void __launch_bounds__(kBlock) pack_kernel(RunView v) {
  const bool vec = (reinterpret_cast<uintptr_t>(v.bases) & 15) == 0;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t w = (uint64_t)blockIdx.x * kBlock + threadIdx.x; w < v.packed_words; w += stride) {
    const uint64_t g = w * 16;
    uint32_t out = 0;
    uint64_t bad_at = ~0ull;
    if (vec && g + 16 <= v.m) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(v.bases + g));
      const uint32_t part[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t bad;
        out |= pack4(part[c], &bad) << (24 - 8 * c);
        if (bad && bad_at == ~0ull) bad_at = g + 4 * c + (__ffs(bad) - 1) / 8;
      }
    } else if (g < v.m) {
      for (int i = 0; i < 16 && g + i < v.m; ++i) {
        const uint32_t c = v.bases[g + i];
        uint32_t bad;
        const uint32_t code = pack4(c | 0x61616100u, &bad) >> 6;  // pad bytes are 'a'
        if ((bad & 0xFFu) && bad_at == ~0ull) bad_at = g + i;
        out |= code << (30 - 2 * i);
      }
    }
    v.packed[w] = out;
    if (bad_at != ~0ull) atomicMin(&v.hdr->bad_index, (unsigned long long)bad_at);
  }
}

// Algorithm 1, insert loop, first pass: every active position records its
// item(s) in the filter; a 64-bit OR is skipped when its bits are already set.
template <int KW, bool ROUNDS>
__global__ void __launch_bounds__(kBlock) pass1_insert_kernel(RunView v, int round) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t g = (uint64_t)blockIdx.x * kBlock + threadIdx.x; g < v.m; g += stride) {
    Occ oc;
    if (!read_occurrence<KW>(v, g, &oc)) continue;
    if (ROUNDS && !in_round(v, oc.H, round)) continue;
    const Spot s = filter_spot(v, oc.H);
    uint64_t P[4];
    load_block(s.blk, P);
    const uint32_t j1 = __ffs(oc.items) - 1, j2 = 31 - __clz(oc.items);
#pragma unroll
    for (int U = 0; U < 4; ++U) {
      if (2 * U < v.hashes) {
        const uint64_t m = item_bits(s, U, j1, v.hashes) | item_bits(s, U, j2, v.hashes);
        const uint32_t phys = (s.o2 + U) & 3u;
        if ((pick4(P, phys) & m) != m) atomicOr(s.blk + phys, (unsigned long long)m);
      }
    }
  }
}

// Algorithm 1, probe loop, first pass: a position stays a candidate iff it is
// a sentinel position, its k-mer's sentinel item is present, or at least two
// of its 16 (predecessor, successor) items are present -- i.e. the filter
// does not show exactly one in-edge and one out-edge. Writes C_temp.
template <int KW, bool ROUNDS>
__global__ void __launch_bounds__(kBlock) pass1_probe_kernel(RunView v, int round) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  const int lane = threadIdx.x & 31;
  unsigned long long kept = 0, valid_n = 0;
  for (uint64_t g0 = (uint64_t)blockIdx.x * kBlock; g0 < v.m; g0 += stride) {
    const uint64_t g = g0 + threadIdx.x;
    bool keep = false, valid = false;
    Occ oc;
    if (g < v.m && read_occurrence<KW>(v, g, &oc)) {
      valid = true;
      if (!ROUNDS || in_round(v, oc.H, round)) {
        if (oc.sentinel) {
          keep = true;
        } else {
          const Spot s = filter_spot(v, oc.H);
          uint64_t P[4];
          load_block(s.blk, P);
          const uint32_t pres = present_items(s, P, v.hashes);
          keep = (pres >> 16) || __popc(pres & 0xFFFFu) >= 2;
        }
      }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    const uint32_t vb = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) {
      const uint64_t w = g >> 5;
      if (w < v.bitmap_words) v.ctemp[w] = bal;
      kept += __popc(bal);
      valid_n += __popc(vb);
    }
  }
  __shared__ unsigned long long red[2][kBlock / 32];
  if (lane == 0) {
    red[0][threadIdx.x >> 5] = kept;
    red[1][threadIdx.x >> 5] = valid_n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    if (a) {
      atomicAdd(&v.hdr->pass1_kept, a);
      atomicAdd(&v.hdr->round_kept, a);
    }
    if (round == 0 && b) atomicAdd(&v.hdr->positions, b);
  }
}

// Size the pass-2 table of this round from the number of candidates:
// the next power of two >= 2 x candidates (at least 1024), capped by the
// workspace.
__global__ void table_setup_kernel(RunView v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long kept = v.hdr->round_kept;
    unsigned long long want = 2ull * kept;
    if (want < 1024ull) want = 1024ull;
    unsigned long long cap = 1ull;
    while (cap < want) cap <<= 1;
    if (cap > v.table_max_slots) cap = v.table_max_slots;
    v.hdr->table_slots = cap;
    if (cap > v.hdr->table_max) v.hdr->table_max = cap;
    v.hdr->round_kept = 0;
  }
}

template <int KW>
__global__ void __launch_bounds__(kBlock) table_clear_kernel(RunView v) {
  const uint64_t cap = *(volatile unsigned long long*)&v.hdr->table_slots;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < cap; i += stride) {
    if (KW == 1) {
      Slot1* s = static_cast<Slot1*>(v.table) + i;
      *reinterpret_cast<ulonglong2*>(s) = make_ulonglong2(kEmpty, 0ull);
    } else {
      Slot2* s = static_cast<Slot2*>(v.table) + i;
      reinterpret_cast<ulonglong2*>(s)[0] = make_ulonglong2(kEmpty, kEmpty);
      reinterpret_cast<ulonglong2*>(s)[1] = make_ulonglong2(0ull, 0ull);
    }
  }
}

// Algorithm 1, insert loop, second pass: every candidate ORs its in/out bases
// (or the sentinel bit) into the exact table entry of its k-mer.
template <int KW>
__global__ void __launch_bounds__(kBlock) pass2_insert_kernel(RunView v) {
  const uint64_t cap = *(volatile unsigned long long*)&v.hdr->table_slots;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t g = (uint64_t)blockIdx.x * kBlock + threadIdx.x; g < v.m; g += stride) {
    if (!((__ldg(v.ctemp + (g >> 5)) >> (g & 31)) & 1u)) continue;
    Occ oc;
    if (!read_occurrence<KW>(v, g, &oc)) continue;
    if (!table_insert<KW>(v, cap, oc.key, second_hash(oc.H), oc.tbits)) v.hdr->overflow = 1;
  }
}

// Algorithm 1, probe loop, second pass: a candidate is a junction iff its
// k-mer is a sentinel or has more than one distinct in- or out-base.
template <int KW>
__global__ void __launch_bounds__(kBlock) pass2_classify_kernel(RunView v, int round) {
  const uint64_t cap = *(volatile unsigned long long*)&v.hdr->table_slots;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  const int lane = threadIdx.x & 31;
  unsigned long long found = 0;
  for (uint64_t g0 = (uint64_t)blockIdx.x * kBlock; g0 < v.m; g0 += stride) {
    const uint64_t g = g0 + threadIdx.x;
    const uint64_t w = g >> 5;
    const uint32_t cw = (w < v.bitmap_words) ? __ldg(v.ctemp + w) : 0u;
    bool junction = false;
    if (cw && ((cw >> lane) & 1u)) {
      Occ oc;
      if (read_occurrence<KW>(v, g, &oc)) {
        const int mk = table_find<KW>(v, cap, oc.key, second_hash(oc.H));
        if (mk < 0) {
          v.hdr->overflow = 1;
          junction = true;
        } else {
          junction = ((mk >> 8) & 1) || __popc(mk & 15) > 1 || __popc((mk >> 4) & 15) > 1;
        }
      }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, junction);
    if (lane == 0 && w < v.bitmap_words) {
      v.cfinal[w] = (round == 0) ? bal : (v.cfinal[w] | bal);
      found += __popc(bal);
    }
  }
  if (lane == 0 && found) atomicAdd(&v.hdr->pass2_kept, found);
}

// Partition counters (section "Multiple Rounds"): a Bloom pre-pass over all
// k-mers; counter f(k-mer) grows when the k-mer was not yet in the filter.
template <int KW>
__global__ void __launch_bounds__(kBlock) partition_count_kernel(RunView v) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t g = (uint64_t)blockIdx.x * kBlock + threadIdx.x; g < v.m; g += stride) {
    Occ oc;
    if (!read_occurrence<KW>(v, g, &oc)) continue;
    const Spot s = filter_spot(v, oc.H);
    const uint64_t m = item_bits(s, 0, 17u, v.hashes);
    const uint32_t phys = s.o2 & 3u;
    if ((__ldcg(s.blk + phys) & m) == m) continue;
    const unsigned long long old = atomicOr(s.blk + phys, (unsigned long long)m);
    if ((old & m) != m) atomicAdd(v.bins + ((uint32_t)oc.H & v.qmask), 1u);
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

// Emit, step 1: junctions per tile of kEmitTileWords bitmap words.
__global__ void __launch_bounds__(kBlock) emit_count_kernel(RunView v) {
  for (uint64_t tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
    const uint64_t w = tile * kEmitTileWords + threadIdx.x;
    uint32_t c = (w < v.bitmap_words) ? __popc(v.cfinal[w]) : 0u;
    uint32_t tot;
    block_exclusive_scan(c, &tot);
    if (threadIdx.x == 0) v.tile_count[tile] = tot;
  }
}

// Emit, step 2: exclusive prefix over tiles (one block); flags a short output.
__global__ void __launch_bounds__(1024) emit_scan_kernel(RunView v) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t base = 0; base < v.n_tiles; base += 1024) {
    const uint64_t i = base + threadIdx.x;
    const unsigned long long x = (i < v.n_tiles) ? v.tile_count[i] : 0ull;
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
    if (i < v.n_tiles) v.tile_prefix[i] = c0 + before + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = c0 + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    v.tile_prefix[v.n_tiles] = carry_s;
    if (carry_s > v.out_capacity) v.hdr->overflow = 1;
  }
}

// Emit, step 3: every junction bit becomes its position within its string,
// in ascending order (C_final of Algorithm 3).
__global__ void __launch_bounds__(kBlock) emit_write_kernel(RunView v) {
  for (uint64_t tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
    const uint64_t w = tile * kEmitTileWords + threadIdx.x;
    uint32_t bits = (w < v.bitmap_words) ? v.cfinal[w] : 0u;
    uint32_t tot;
    const uint32_t excl = block_exclusive_scan(__popc(bits), &tot);
    uint64_t at = v.tile_prefix[tile] + excl;
    while (bits) {
      const uint32_t b = __ffs(bits) - 1;
      bits &= bits - 1;
      const uint64_t g = w * 32 + b;
      const Bounds bd = seq_bounds(v, g);
      if (at < v.out_capacity) v.out_positions[at] = g - bd.start;
      ++at;
    }
  }
}

// Emit, step 4: offsets[t] = junctions in strings before t.
__global__ void __launch_bounds__(kBlock) emit_offsets_kernel(RunView v) {
  const uint64_t t = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (t > v.n_seqs) return;
  const uint64_t g = (t == v.n_seqs) ? v.m : __ldg(v.offsets + t);
  const uint64_t w = g >> 5;
  const uint64_t tile = w / kEmitTileWords;
  uint64_t cnt = v.tile_prefix[tile < v.n_tiles ? tile : v.n_tiles];
  for (uint64_t x = tile * kEmitTileWords; x < w; ++x) cnt += __popc(v.cfinal[x]);
  if (g & 31) cnt += __popc(v.cfinal[w] & ((1u << (g & 31)) - 1u));
  v.out_offsets[t] = cnt;
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

template <typename K>
unsigned grid_for(K kernel, int block, uint64_t work_items) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
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

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n); }

int launch_init(const RunView& v, cudaStream_t s) {
  { Timed t("init", s); init_kernel<<<1, 32, 0, s>>>(v); }
  return done(1);
}

int launch_pack(const RunView& v, cudaStream_t s) {
  if (v.packed_words == 0) return 0;
  { Timed t("pack", s); pack_kernel<<<grid_for(pack_kernel, kBlock, v.packed_words), kBlock, 0, s>>>(v); }
  return done(1);
}

int launch_partition(const RunView& v, int rounds, cudaStream_t s) {
  if (v.m == 0) return 0;
  if (cudaMemsetAsync(v.filter, 0, v.filter_words64 * 8, s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(v.bins, 0, (uint64_t)(v.qmask + 1u) * 4, s) != cudaSuccess) return -1;
  {
    Timed t("partition_count", s);
    if (v.k <= 31)
      partition_count_kernel<1><<<grid_for(partition_count_kernel<1>, kBlock, v.m), kBlock, 0, s>>>(v);
    else
      partition_count_kernel<2><<<grid_for(partition_count_kernel<2>, kBlock, v.m), kBlock, 0, s>>>(v);
  }
  uint64_t* prefix = reinterpret_cast<uint64_t*>(v.bins + (v.qmask + 1u));
  {
    Timed t("partition_cut", s);
    partition_cut_kernel<<<1, 1024, 0, s>>>(v, rounds, prefix);
  }
  return done(2);
}

template <int KW>
int round_impl(const RunView& v, int round, bool rounds_on, cudaStream_t s) {
  if (cudaMemsetAsync(v.filter, 0, v.filter_words64 * 8, s) != cudaSuccess) return -1;
  const unsigned gm = grid_for(pass1_probe_kernel<KW, true>, kBlock, v.m);
  {
    Timed t("pass1_insert", s);
    if (rounds_on) pass1_insert_kernel<KW, true><<<gm, kBlock, 0, s>>>(v, round);
    else pass1_insert_kernel<KW, false><<<gm, kBlock, 0, s>>>(v, round);
  }
  {
    Timed t("pass1_probe", s);
    if (rounds_on) pass1_probe_kernel<KW, true><<<gm, kBlock, 0, s>>>(v, round);
    else pass1_probe_kernel<KW, false><<<gm, kBlock, 0, s>>>(v, round);
  }
  {
    Timed t("table_setup", s);
    table_setup_kernel<<<1, 32, 0, s>>>(v);
  }
  {
    Timed t("table_clear", s);
    table_clear_kernel<KW><<<grid_for(table_clear_kernel<KW>, kBlock, v.table_max_slots), kBlock, 0, s>>>(v);
  }
  {
    Timed t("pass2_insert", s);
    pass2_insert_kernel<KW><<<gm, kBlock, 0, s>>>(v);
  }
  {
    Timed t("pass2_classify", s);
    pass2_classify_kernel<KW><<<gm, kBlock, 0, s>>>(v, round);
  }
  return done(6);
}

int launch_round(const RunView& v, int round, int rounds, cudaStream_t s) {
  if (v.m == 0) return 0;
  const bool on = rounds > 1;
  return v.k <= 31 ? round_impl<1>(v, round, on, s) : round_impl<2>(v, round, on, s);
}

int launch_emit(const RunView& v, cudaStream_t s) {
  int n = 0;
  if (v.n_tiles) {
    Timed t("emit_count", s);
    emit_count_kernel<<<grid_for(emit_count_kernel, kBlock, v.n_tiles * kBlock), kBlock, 0, s>>>(v);
    n++;
  }
  {
    Timed t("emit_scan", s);
    emit_scan_kernel<<<1, 1024, 0, s>>>(v);
    n++;
  }
  if (v.n_tiles) {
    Timed t("emit_write", s);
    emit_write_kernel<<<grid_for(emit_write_kernel, kBlock, v.n_tiles * kBlock), kBlock, 0, s>>>(v);
    n++;
  }
  {
    Timed t("emit_offsets", s);
    emit_offsets_kernel<<<(unsigned)((v.n_seqs + 1 + kBlock - 1) / kBlock), kBlock, 0, s>>>(v);
    n++;
  }
  return done(n);
}

}  // namespace twopaco

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
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return TWOPACO_ECUDA_INTERNAL;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) return TWOPACO_ECUDA_INTERNAL;
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
