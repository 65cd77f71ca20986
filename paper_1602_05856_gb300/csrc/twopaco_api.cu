// C-ABI layer of the junction-detection library: argument checks, workspace
// layout, the launch sequence of one run, and the host-to-host build.
#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "twopaco.h"
#include "twopaco_checksum.h"
#include "twopaco_internal.h"

namespace twopaco {
namespace {

constexpr uint64_t kAlign = 256;
constexpr uint64_t kStreamChunkMin = 64 << 10;  // bytes per staging half, at least

uint64_t align_up(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int log2_exact(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

twopaco_options resolve(const twopaco_options* opt) {
  twopaco_options o;
  twopaco_default_options(&o);
  if (opt) o = *opt;
  return o;
}

int validate(uint64_t n_seqs, int k, uint64_t filter_bits, int rounds, const twopaco_options& o) {
  if (k < 1 || k > 127) return TWOPACO_EINVAL;
  if (filter_bits < 256 || !is_pow2(filter_bits) || filter_bits > (1ull << 40)) return TWOPACO_EINVAL;
  if (rounds < 1) return TWOPACO_EINVAL;
  if (o.hashes < 1 || o.hashes > 8) return TWOPACO_EINVAL;
  if (o.both_strands != 0 && o.both_strands != 1) return TWOPACO_EINVAL;
  if (!is_pow2(o.partition_bins) || o.partition_bins < (uint32_t)rounds) return TWOPACO_EINVAL;
  if (rounds > 1 && o.partition_bins < 2) return TWOPACO_EINVAL;
  if (n_seqs >= (1ull << 32)) return TWOPACO_EINVAL;
  if (o.split_at_n != 0 && o.split_at_n != 1) return TWOPACO_EINVAL;
  if (o.wide_layout < 0 || o.wide_layout > 2) return TWOPACO_EINVAL;
  if (o.run_capacity >= (1ull << 32)) return TWOPACO_EINVAL;  // piece ranks are 32-bit
  if (o.partial != 0 && o.partial != 1) return TWOPACO_EINVAL;
  if (o.per_string_launches != 0 && o.per_string_launches != 1) return TWOPACO_EINVAL;
  if (o.bucket_inserts < 0 || o.bucket_inserts > 2) return TWOPACO_EINVAL;
  if (o.launch_blocks_per_sm < 0 || o.launch_blocks_per_sm > 32) return TWOPACO_EINVAL;
  if (o.ordered_first_pass < 0 || o.ordered_first_pass > 2) return TWOPACO_EINVAL;
  return TWOPACO_OK;
}

// A failed call of another library (an allocation, say) leaves its error for
// cudaPeekAtLastError, which the launch helpers read after their launches:
// clear it when a call of this library starts, so that only this call's
// launches are judged.
void clear_stale_error() { (void)cudaGetLastError(); }

int validate_size(uint64_t total_bases) {
  return total_bases >= (1ull << 48) ? TWOPACO_EINVAL : TWOPACO_OK;  // positions fit 48 bits
}

struct Layout {
  uint64_t header, packed, filter, ctemp, cfinal, tile_count, tile_prefix, bins, cuts, table;
  uint64_t cands, lc, segs, desc, cslot, nmask, bounds, chunks, runs, rank, cmap, bfill, brecs;
  int narrow, use_desc, use_slot, split, use_cmap;
  uint32_t n_regions, n_sub;
  int lg_region_words;
  uint32_t o_regions;  // region-ordered first pass (0: off)
  int o_fused;         // ... with pass 2 on its records
  uint32_t o_tcap;     // fused: table slots per region
  int o_lg_region_words;
  uint64_t o_rec_cap, o_tiles;
  uint64_t rplane, othist, owcount, ocsum, ocpre, obtot, ostart, ofill, orecs, odec, ometa, otcount, otbase, otsum,
      operm;
  uint64_t bucket_cap, bucket_chunk;
  uint64_t n_chunks, run_cap;
  uint64_t total;
  uint64_t packed_words, bitmap_words, n_tiles, table_slots, cand_cap;
  int lc_log2;
};

uint64_t auto_table_slots(uint64_t m, int rounds) {
  uint64_t per_round = (m + (uint64_t)rounds - 1) / (uint64_t)rounds;
  uint64_t want = 2 * per_round;
  if (want < 1024) want = 1024;
  return next_pow2(want);
}

uint64_t auto_run_capacity(uint64_t m, uint64_t n_seqs) {
  const uint64_t want = n_seqs + 1 + m / 64;
  return want < (1ull << 32) ? want : (1ull << 32) - 1;  // piece ranks are 32-bit
}

Layout layout(uint64_t m, uint64_t n_seqs, int k, uint64_t filter_bits, int rounds,
              const twopaco_options& o) {
  Layout L{};
  L.packed_words = (m + 15) / 16 + kPackPadWords;
  L.bitmap_words = (m + 31) / 32;
  L.n_tiles = (L.bitmap_words + kEmitTileWords - 1) / kEmitTileWords;
  L.table_slots = o.table_slots ? next_pow2(o.table_slots) : auto_table_slots(m, rounds);
  if (o.partial) L.table_slots = 0;  // no second pass: no table, list or kept slots
  // 32-bit candidate records (31-bit positions and a sentinel flag) below 2^31 bases
  L.narrow = (m < (1ull << 31) && o.wide_layout == 0) ? 1 : 0;
  uint64_t at = 0;
  L.header = at;
  at += align_up(sizeof(DevHeader));
  L.packed = at;
  at += align_up(L.packed_words * 4);
  L.filter = at;
  at += align_up(filter_bits / 8);
  L.ctemp = at;
  at += align_up((L.bitmap_words + 8) * 4);
  L.cfinal = at;
  at += align_up((L.bitmap_words + 8) * 4);
  L.tile_count = at;
  at += align_up((L.n_tiles + 1) * 4);
  L.tile_prefix = at;
  at += align_up((L.n_tiles + 1) * 8);
  L.bins = at;
  if (rounds > 1) at += align_up((uint64_t)o.partition_bins * 4 + ((uint64_t)o.partition_bins + 1) * 8);
  L.cuts = at;
  at += align_up(((uint64_t)rounds + 1) * 4);
  L.table = at;
  at += align_up(L.table_slots * table_slot_bytes(k));
  // candidate list: half the positions of a round in 8-byte units by default
  // (every position of the round, as 32-bit records, under 2^31 bases); a
  // longer round falls back to walking C_temp
  const uint64_t per_round = (m + (uint64_t)rounds - 1) / (uint64_t)rounds;
  L.cand_cap = o.candidate_records ? o.candidate_records
                                   : (per_round / 2 > (1u << 16) ? per_round / 2 : (1u << 16));
  if (o.partial) L.cand_cap = 0;
  // region-ordered first pass: class-map rounds (k <= 63, h <= 6, one launch
  // per loop) with at most kOrdMaxRegions regions of at most 2^22 words and
  // at most kOrdMaxHist (round, region) counters; automatically for filters of
  // 1 GiB and more (far beyond L2), or for any filter when asked
  L.o_regions = 0;
  {
    const uint64_t fwords = filter_bits / 64;
    const uint64_t rw = std::max<uint64_t>(1, std::min<uint64_t>(1ull << kRegionWordsLog2, fwords / 64));
    const uint64_t R = fwords / rw;
    const bool want = o.ordered_first_pass == 1 || (o.ordered_first_pass == 0 && filter_bits / 8 >= (1ull << 30));
    if (want && rounds > 1 && rounds <= kMaxMapRounds && k <= 63 && o.hashes <= 6 && !o.per_string_launches &&
        m > 0 && R <= kOrdMaxRegions && R * (uint64_t)rounds <= kOrdMaxHist) {
      L.o_regions = (uint32_t)R;
      L.o_lg_region_words = log2_exact(rw);
      // records for a round's positions and a quarter more (classes are cut
      // to hold about m / rounds distinct k-mers each; repeats make their
      // positions vary more), plus each bucket's rounding to 32; a round whose
      // records do not fit takes the direct kernels
      L.o_rec_cap = per_round + per_round / 4 + 32ull * R + 4096;
      L.o_tiles = (m + kOrdTile - 1) / kOrdTile;
      // pass 2 on the records too (one-word table slots, k <= 27): the table
      // reserve split into one part per region, at least 1024 slots each
      const uint64_t tcap = L.table_slots / R;
      if (k <= 27 && !o.partial && tcap >= 1024 && tcap < (1ull << 32)) {
        L.o_fused = 1;
        L.o_tcap = (uint32_t)tcap;
      }
    }
  }
  L.cands = at;
  // with the ordered first pass the list shares the records' room: the gather
  // writes the list after the probe read the last record
  if (!L.o_regions) at += align_up(L.cand_cap * cand_record_bytes(k));
  // the table slot of every listed candidate (32-bit slot indices), kept by
  // the second-pass insert for its probe loop; one per record of the list
  // (twice as many 32-bit records under 2^31 bases)
  // (slot 0xFFFFFFFF stands for "no slot", so the table stays below 2^32 slots)
  L.use_slot = (L.table_slots < (1ull << 32) && o.wide_layout < 2) ? 1 : 0;
  L.cslot = at;
  if (L.use_slot) at += align_up(L.cand_cap * (L.narrow ? 2 : 1) * 4);
  // linear-counting bitmap: 2^lc_log2 >= the list's capacity, at least 2^16
  // bits and at most 2^28 (32 MiB, which stays in L2 while the probe sets its
  // bits at random; linear counting stays exact to a small fraction of a
  // percent up to about 7 distinct candidates per bit)
  L.lc_log2 = 16;
  while ((1ull << L.lc_log2) < L.cand_cap && L.lc_log2 < 28) ++L.lc_log2;
  L.lc = at;
  at += align_up((1ull << L.lc_log2) / 8);
  L.segs = at;
  at += align_up((uint64_t)kMaxSegments * 4);
  // probe descriptors: one 64-bit word per position (filter word index, 30 bits
  // of bit bases, flags) when they fit -- under 2^31 bases, h <= 6, b <= 2^37
  // class map: one byte per position for 2 .. kMaxMapRounds rounds (then the
  // rounds need no descriptors: each visits only its class's positions)
  L.use_cmap = (rounds > 1 && rounds <= kMaxMapRounds) ? 1 : 0;
  L.cmap = at;
  if (L.use_cmap) at += align_up(m + 64);
  L.use_desc = (L.narrow && o.hashes <= 6 && filter_bits <= (1ull << 37) && !L.use_cmap) ? 1 : 0;
  L.desc = at;
  if (L.use_desc) at += align_up((m + 16) * 8);
  // region buckets for the first-pass inserts: filters beyond L2 (over 64 MiB),
  // or any filter when asked; regions of up to 2^22 words (32 MiB), at most
  // kMaxRegions of them; records carry up to 6 bits per item
  const uint64_t fwords = filter_bits / 64;
  const bool want_bkt = o.bucket_inserts == 1 || (o.bucket_inserts == 0 && filter_bits / 8 > (64ull << 20));
  uint64_t region_words = std::min<uint64_t>(1ull << kRegionWordsLog2, fwords / 4);
  L.n_regions = 0;
  // automatically only where it measured faster: when a chunk's records put at
  // least 16 ORs on every 32-byte filter sector on average (on a 24 Gbp input
  // with a 2^36-bit filter, about 7 per sector, the cold misses of every region
  // cost more than the direct ORs; on 310 Mbp with 2^30 bits, 77 per sector, the
  // buckets win)
  const uint64_t per_chunk = std::min<uint64_t>(per_round, 1ull << 31) * 4 / 5;
  const bool dense = per_chunk >= 16 * (filter_bits / 256);
  if (want_bkt && (o.bucket_inserts == 1 || dense) && o.hashes <= 6 && m > 0 && region_words >= 1 &&
      fwords / region_words <= kMaxRegions) {
    L.n_regions = (uint32_t)(fwords / region_words);
    L.n_sub = 1;
    while (L.n_regions * L.n_sub < kMinBuckets) L.n_sub *= 2;
    L.lg_region_words = log2_exact(region_words);
    // records for a round's positions and a quarter more (at most 2^31 of them),
    // shared out evenly over the buckets; a chunk of positions fills about 80%
    const uint64_t buckets = (uint64_t)L.n_regions * L.n_sub;
    uint64_t recs = std::min<uint64_t>(per_round + per_round / 4 + 4096ull * buckets, 1ull << 31);
    L.bucket_cap = recs / buckets;
    const uint64_t chunk = L.bucket_cap * buckets / 5 * 4 * (uint64_t)rounds;
    L.bucket_chunk = std::max<uint64_t>(kRangeTile, chunk / kRangeTile * kRangeTile);
  }
  if (L.o_regions) L.n_regions = 0;  // the ordered first pass applies the inserts by region itself
  L.bfill = at;
  if (L.n_regions) at += align_up(((uint64_t)L.n_regions * L.n_sub + 1) * 128);
  L.brecs = at;
  if (L.n_regions) at += align_up(L.bucket_cap * L.n_regions * L.n_sub * 8);
  L.rplane = L.othist = L.owcount = L.ocsum = L.ocpre = L.obtot = L.ostart = L.ofill = L.orecs = L.odec = L.ometa = at;
  L.otcount = L.otbase = L.otsum = L.operm = at;
  if (L.o_regions) {
    const uint64_t R = L.o_regions;
    L.rplane = at;
    at += align_up(m + 64);
    const uint64_t chunks = (L.o_tiles + kOrdScanTiles - 1) / kOrdScanTiles;
    L.othist = at;
    at += align_up(L.o_tiles * rounds * R * 2);
    L.owcount = at;
    at += align_up((uint64_t)rounds * L.o_tiles * 8 * 2);
    L.ocsum = at;
    at += align_up(chunks * R * 4);
    L.ocpre = at;
    at += align_up(chunks * R * 8);
    L.obtot = at;
    at += align_up(R * 8);
    L.ostart = at;
    at += align_up((R + 1) * 8);
    L.ofill = at;
    at += align_up(R * kOrdFillStride * 4);
    L.orecs = at;
    L.cands = at;
    at += align_up(std::max<uint64_t>(L.o_rec_cap * 8, L.cand_cap * cand_record_bytes(k)));
    L.odec = at;
    at += align_up((L.o_rec_cap + 31) / 32 * 4 * (L.o_fused ? 2 : 1));
    L.ometa = at;
    at += align_up(L.o_tiles * R * 4);
    L.otcount = at;
    at += align_up((uint64_t)rounds * L.o_tiles * 4);
    L.otbase = at;
    at += align_up((uint64_t)rounds * L.o_tiles * 8);
    L.otsum = at;
    at += align_up((uint64_t)rounds * ((L.o_tiles + kOrdScanTiles - 1) / kOrdScanTiles) * 8);
    L.operm = at;
    at += align_up(L.o_rec_cap * 2);
  }
  // N splitting: N mask and boundary bitmap (one bit per base), per-chunk
  // boundary counts, the sorted boundaries and their ranks
  L.split = o.split_at_n;
  L.n_chunks = (L.bitmap_words + kRunChunkWords - 1) / kRunChunkWords;
  L.run_cap = o.run_capacity ? o.run_capacity : auto_run_capacity(m, n_seqs);
  L.nmask = L.bounds = L.chunks = L.runs = L.rank = at;
  if (L.split) {
    // the pack kernel writes one N-mask word per two packed words, pad included
    at += align_up((L.packed_words + 3) / 2 * 4);
    L.bounds = at;
    at += align_up((L.bitmap_words + 8) * 4);
    L.chunks = at;
    at += align_up((L.n_chunks + 1) * 8);
    L.runs = at;
    at += align_up((L.run_cap + 1) * 8);
    L.rank = at;
    at += align_up((L.run_cap + 1) * 4);
  }
  L.total = at;
  return L;
}

RunView make_view(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs, uint64_t m,
                  int k, uint64_t filter_bits, int rounds, const twopaco_options& o,
                  const Layout& L, void* ws, uint64_t* d_out_offsets, uint64_t* d_out_positions,
                  uint64_t out_capacity) {
  char* base = static_cast<char*>(ws);
  RunView v{};
  v.bases = d_bases;
  v.offsets = d_offsets;
  v.n_seqs = (uint32_t)n_seqs;
  v.m = m;
  v.k = k;
  v.both = o.both_strands;
  v.hashes = o.hashes;
  v.rounds = rounds;
  v.partial = o.partial;
  v.lg_blocks = log2_exact(filter_bits / 256);
  v.qmask = o.partition_bins - 1u;
  // the pre-pass counts every k-mer up to 2^29 bases, then a 2^-s sample with
  // s = floor(log2(m / 2^28)), at most 2^-8 (2^-6 at 24 Gbp)
  int sample_log2 = 0;
  while (sample_log2 < 8 && (m >> (28 + sample_log2 + 1)) > 0) ++sample_log2;
  v.part_sample = (1u << sample_log2) - 1u;
  // from 2^33 bases the pre-pass also walks only every fourth chunk of 65536
  // positions: the walk, not the counting, is its cost, and the cut needs
  // the bins' proportions only
  v.part_chunks = m >= (1ull << 33) ? 3u : 0u;
  v.hdr = reinterpret_cast<DevHeader*>(base + L.header);
  v.packed = reinterpret_cast<uint32_t*>(base + L.packed);
  v.packed_words = L.packed_words;
  v.filter = reinterpret_cast<unsigned long long*>(base + L.filter);
  v.filter_words64 = filter_bits / 64;
  v.ctemp = reinterpret_cast<uint32_t*>(base + L.ctemp);
  v.cfinal = reinterpret_cast<uint32_t*>(base + L.cfinal);
  v.bitmap_words = L.bitmap_words;
  v.p_begin = 0;
  v.p_end = m;
  v.blocks_per_sm = o.launch_blocks_per_sm;
  v.table = base + L.table;
  v.table_max_slots = L.table_slots;
  v.cands = reinterpret_cast<uint64_t*>(base + L.cands);
  v.narrow = L.narrow;
  v.use_desc = L.use_desc;
  v.cand_slot = L.use_slot ? reinterpret_cast<uint32_t*>(base + L.cslot) : nullptr;
  v.desc = reinterpret_cast<uint64_t*>(base + L.desc);
  if (L.split) {
    v.nmask = reinterpret_cast<uint32_t*>(base + L.nmask);
    v.bound_bits = reinterpret_cast<uint32_t*>(base + L.bounds);
    v.chunk_counts = reinterpret_cast<uint64_t*>(base + L.chunks);
    v.n_chunks = L.n_chunks;
    v.runs = reinterpret_cast<uint64_t*>(base + L.runs);
    v.run_rank = reinterpret_cast<uint32_t*>(base + L.rank);
    v.run_cap = L.run_cap;
  }
  v.cand_cap = L.cand_cap;
  v.lc_bits = reinterpret_cast<uint32_t*>(base + L.lc);
  v.lc_log2 = L.lc_log2;
  v.seg_count = reinterpret_cast<uint32_t*>(base + L.segs);
  v.bins = rounds > 1 ? reinterpret_cast<uint32_t*>(base + L.bins) : nullptr;
  v.cuts = reinterpret_cast<uint32_t*>(base + L.cuts);
  v.cmap = L.use_cmap ? reinterpret_cast<uint8_t*>(base + L.cmap) : nullptr;
  v.n_regions = L.n_regions;
  if (L.n_regions) {
    v.lg_region_words = L.lg_region_words;
    v.n_sub = L.n_sub;
    v.bucket_fill = reinterpret_cast<uint32_t*>(base + L.bfill);
    v.bucket_recs = reinterpret_cast<uint64_t*>(base + L.brecs);
    v.bucket_cap = L.bucket_cap;
    v.bucket_chunk = L.bucket_chunk;
  }
  v.o_regions = L.o_regions;
  if (L.o_regions) {
    v.o_lg_region_words = L.o_lg_region_words;
    v.rplane = reinterpret_cast<uint8_t*>(base + L.rplane);
    v.o_thist = reinterpret_cast<uint16_t*>(base + L.othist);
    v.o_wcount = reinterpret_cast<uint16_t*>(base + L.owcount);
    v.o_csum = reinterpret_cast<uint32_t*>(base + L.ocsum);
    v.o_cpre = reinterpret_cast<unsigned long long*>(base + L.ocpre);
    v.o_btot = reinterpret_cast<unsigned long long*>(base + L.obtot);
    v.o_start = reinterpret_cast<uint64_t*>(base + L.ostart);
    v.o_fill = reinterpret_cast<uint32_t*>(base + L.ofill);
    v.o_recs = reinterpret_cast<uint64_t*>(base + L.orecs);
    v.o_rec_cap = L.o_rec_cap;
    v.o_dec = reinterpret_cast<uint32_t*>(base + L.odec);
    v.o_meta = reinterpret_cast<uint32_t*>(base + L.ometa);
    v.o_tiles = L.o_tiles;
    v.o_tcount = reinterpret_cast<uint32_t*>(base + L.otcount);
    v.o_tbase = reinterpret_cast<unsigned long long*>(base + L.otbase);
    v.o_tsum = reinterpret_cast<unsigned long long*>(base + L.otsum);
    v.o_perm = reinterpret_cast<uint16_t*>(base + L.operm);
    v.o_fused = L.o_fused;
    v.o_tcap = L.o_tcap;
    // large rounds count distinct candidates on an eighth of the k-mers
    v.lc_sample_log2 = L.o_rec_cap >= (1ull << 26) ? 3 : 0;
  }
  v.tile_count = reinterpret_cast<uint32_t*>(base + L.tile_count);
  v.tile_prefix = reinterpret_cast<uint64_t*>(base + L.tile_prefix);
  v.n_tiles = L.n_tiles;
  v.out_offsets = d_out_offsets;
  v.out_positions = d_out_positions;
  v.out_capacity = out_capacity;
  return v;
}

// Boundaries of the N-free pieces and N runs of host strings: one per
// non-empty string plus one per change between N and a base inside a string.
uint64_t count_run_boundaries(const char* const* seqs, const uint64_t* lengths, uint64_t n) {
  uint64_t r = 0;
  for (uint64_t t = 0; t < n; ++t) {
    if (!lengths[t]) continue;
    ++r;
    bool prev_n = (seqs[t][0] | 0x20) == 'n';
    for (uint64_t i = 1; i < lengths[t]; ++i) {
      const bool is_n = (seqs[t][i] | 0x20) == 'n';
      r += is_n != prev_n;
      prev_n = is_n;
    }
  }
  return r;
}

// Host builds know their input: with N splitting the boundary list gets at
// least the exact count, so that only the table or the output can run short.
void raise_run_capacity(twopaco_options* o, const char* const* seqs, const uint64_t* lengths, uint64_t n) {
  if (!o->split_at_n) return;
  const uint64_t need = count_run_boundaries(seqs, lengths, n) + 1;
  if (o->run_capacity < need) o->run_capacity = need;
}

int cuda_code(cudaError_t e) {
  if (e == cudaSuccess) return TWOPACO_OK;
  if (e == cudaErrorMemoryAllocation) return TWOPACO_ENOMEM;
  return TWOPACO_ECUDA;
}

}  // namespace
}  // namespace twopaco

using namespace twopaco;

extern "C" {

void twopaco_default_options(twopaco_options* opt) {
  if (!opt) return;
  opt->hashes = 4;
  opt->both_strands = 1;
  opt->partition_bins = 65536;
  opt->table_slots = 0;
  opt->candidate_records = 0;
  opt->cuda_stream = nullptr;
  opt->split_at_n = 0;
  opt->run_capacity = 0;
  opt->wide_layout = 0;
  opt->partial = 0;
  opt->per_string_launches = 0;
  opt->bucket_inserts = 0;
  opt->launch_blocks_per_sm = 0;
  opt->ordered_first_pass = 0;
}

const char* twopaco_strerror(int code) {
  switch (code) {
    case TWOPACO_OK: return "ok";
    case TWOPACO_EINVAL: return "invalid argument";
    case TWOPACO_EBADBASE: return "input byte is not one of ACGTacgt (or Nn with split_at_n)";
    case TWOPACO_ENOMEM: return "out of memory";
    case TWOPACO_ETIMEOUT: return "a bounded device wait gave up";
    case TWOPACO_ECUDA: return "CUDA error";
    case TWOPACO_EOVERFLOW: return "pass-2 table, output buffer or run boundary list too small";
    case TWOPACO_ESCRATCH: return "run needs more than the no-alloc scratch buffer holds";
    default: return "unknown error";
  }
}

int twopaco_workspace_size(uint64_t total_bases, uint64_t n_seqs, int k, uint64_t filter_bits,
                           int rounds, const twopaco_options* opt, uint64_t* bytes) {
  const twopaco_options o = resolve(opt);
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (!bytes || validate_size(total_bases)) return TWOPACO_EINVAL;
  *bytes = layout(total_bases, n_seqs, k, filter_bits, rounds, o).total;
  return TWOPACO_OK;
}

}  // extern "C"

namespace twopaco {
namespace {

// The checks every device-resident call makes before launching anything, and
// the run's view of the workspace.
int device_run_view(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                    uint64_t total_bases, int k, uint64_t filter_bits, int rounds, const twopaco_options& o,
                    void* d_workspace, uint64_t workspace_bytes, uint64_t* d_out_offsets,
                    uint64_t* d_out_positions, uint64_t out_capacity, bool need_output, RunView* v) {
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (validate_size(total_bases)) return TWOPACO_EINVAL;
  if (total_bases > 0 && (n_seqs == 0 || !d_bases || !d_offsets)) return TWOPACO_EINVAL;
  if (n_seqs > 0 && !d_offsets) return TWOPACO_EINVAL;
  if (need_output && (!d_out_offsets || (out_capacity && !d_out_positions))) return TWOPACO_EINVAL;
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)) return TWOPACO_EINVAL;
  const Layout L = layout(total_bases, n_seqs, k, filter_bits, rounds, o);
  if (workspace_bytes < L.total) return TWOPACO_EINVAL;
  *v = make_view(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, o, L, d_workspace,
                 d_out_offsets, d_out_positions, out_capacity);
  return TWOPACO_OK;
}

// The position ranges of per-string launches: tiles of kRangeTile positions,
// each launched with the string that holds its first position (so that every
// position is visited exactly once), one range per string that owns a tile.
// Reads the offsets back from the device (synchronises the stream).
int string_ranges(const uint64_t* d_offsets, uint64_t n_seqs, uint64_t m, cudaStream_t s,
                  std::vector<std::pair<uint64_t, uint64_t>>* out) {
  std::vector<uint64_t> off(n_seqs + 1);
  cudaError_t e = cudaMemcpyAsync(off.data(), d_offsets, (n_seqs + 1) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_code(e);
  out->clear();
  for (uint64_t t = 0; t < n_seqs; ++t) {
    const uint64_t a = (off[t] + kRangeTile - 1) / kRangeTile * kRangeTile;  // first tile starting in t
    const uint64_t b = std::min(m, (off[t + 1] + kRangeTile - 1) / kRangeTile * kRangeTile);
    if (a < b) out->push_back({a, b});
  }
  return TWOPACO_OK;
}

}  // namespace
}  // namespace twopaco

extern "C" {

int twopaco_run_rounds(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                       uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                       const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                       int round_begin, int round_end, uint64_t* d_out_offsets,
                       uint64_t* d_out_positions, uint64_t out_capacity) {
  clear_stale_error();
  const twopaco_options o = resolve(opt);
  RunView v;
  int rc = device_run_view(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, o, d_workspace,
                           workspace_bytes, d_out_offsets, d_out_positions, out_capacity, true, &v);
  if (rc) return rc;
  if (round_begin < 0 || round_end > rounds || round_begin > round_end) return TWOPACO_EINVAL;
  if (round_begin == round_end && round_end != rounds) return TWOPACO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);
  if (round_begin == 0) {  // a new run: pack, and the class cut of Algorithm 3
    if (launch_init(v, s) < 0) return TWOPACO_ECUDA;
    if (launch_pack(v, s) < 0) return TWOPACO_ECUDA;
    if (rounds > 1 && launch_partition(v, rounds, s) < 0) return TWOPACO_ECUDA;
    if (launch_class_map(v, s) < 0) return TWOPACO_ECUDA;
  }
  std::vector<std::pair<uint64_t, uint64_t>> ranges;
  if (o.per_string_launches && round_begin < round_end) {
    rc = string_ranges(d_offsets, n_seqs, total_bases, s, &ranges);
    if (rc) return rc;
  }
  for (int r = round_begin; r < round_end; ++r)
    if (launch_round(v, r, rounds, s, o.per_string_launches ? &ranges : nullptr) < 0) return TWOPACO_ECUDA;
  if (round_end == rounds && launch_emit(v, s, round_begin == rounds) < 0) return TWOPACO_ECUDA;
  return TWOPACO_OK;
}

int twopaco_run_streamed(const uint8_t* h_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                         uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                         const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                         void* d_staging, uint64_t staging_bytes, uint64_t* d_out_offsets,
                         uint64_t* d_out_positions, uint64_t out_capacity) {
  clear_stale_error();
  const twopaco_options o = resolve(opt);
  RunView v;
  int rc = device_run_view(h_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, o, d_workspace,
                           workspace_bytes, d_out_offsets, d_out_positions, out_capacity, true, &v);
  if (rc) return rc;
  if (!d_staging || (reinterpret_cast<uintptr_t>(d_staging) % kAlign)) return TWOPACO_EINVAL;
  // two staging halves of a multiple of 256 bytes each (so that every chunk
  // starts on a packed word that is a multiple of 4, and 16-byte aligned)
  const uint64_t chunk = staging_bytes / 2 / kAlign * kAlign;
  if (chunk < kStreamChunkMin) return TWOPACO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);
  cudaStream_t cs = nullptr;
  cudaEvent_t start = nullptr, copied[2] = {nullptr, nullptr}, packed[2] = {nullptr, nullptr};
  auto finish = [&](int code) {
    for (cudaEvent_t e : {start, copied[0], copied[1], packed[0], packed[1]})
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);  // its work completes first; the release is deferred
    return code;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&start, &copied[0], &copied[1], &packed[0], &packed[1]})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return finish(cuda_code(e));
  // the copies start once earlier work on the stream (which may still read the
  // staging buffer) is done
  if ((e = cudaEventRecord(start, s)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, start, 0)) != cudaSuccess)
    return finish(cuda_code(e));
  if (launch_init(v, s) < 0) return finish(TWOPACO_ECUDA);
  char* stage = static_cast<char*>(d_staging);
  const uint64_t n_chunks = total_bases ? (total_bases + chunk - 1) / chunk : 0;
  if (n_chunks == 0 && launch_pack_chunk(v, 0, v.packed_words, true, s) < 0) return finish(TWOPACO_ECUDA);
  for (uint64_t c = 0; c < n_chunks; ++c) {
    const int b = (int)(c & 1);
    const uint64_t g0 = c * chunk, len = std::min(chunk, total_bases - g0);
    char* buf = stage + b * chunk;
    // reuse a half only after the pack of the chunk it held two chunks ago
    if (c >= 2 && (e = cudaStreamWaitEvent(cs, packed[b], 0)) != cudaSuccess) return finish(cuda_code(e));
    if ((e = cudaMemcpyAsync(buf, h_bases + g0, len, cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
        (e = cudaEventRecord(copied[b], cs)) != cudaSuccess || (e = cudaStreamWaitEvent(s, copied[b], 0)) != cudaSuccess)
      return finish(cuda_code(e));
    RunView cv = v;
    cv.bases = reinterpret_cast<const uint8_t*>(buf) - g0;  // bytes [g0, g0 + len) at buf
    const uint64_t w_begin = g0 / 16;
    const uint64_t w_end = c + 1 == n_chunks ? v.packed_words : (g0 + len) / 16;  // the last takes the pad
    if (launch_pack_chunk(cv, w_begin, w_end, c == 0, s) < 0) return finish(TWOPACO_ECUDA);
    if ((e = cudaEventRecord(packed[b], s)) != cudaSuccess) return finish(cuda_code(e));
  }
  if (launch_pack_finish(v, s) < 0) return finish(TWOPACO_ECUDA);
  if (rounds > 1 && launch_partition(v, rounds, s) < 0) return finish(TWOPACO_ECUDA);
  if (launch_class_map(v, s) < 0) return finish(TWOPACO_ECUDA);
  for (int r = 0; r < rounds; ++r)
    if (launch_round(v, r, rounds, s) < 0) return finish(TWOPACO_ECUDA);
  if (launch_emit(v, s) < 0) return finish(TWOPACO_ECUDA);
  return finish(TWOPACO_OK);
}

int twopaco_shard_begin(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                        uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                        const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                        int compute_cut) {
  clear_stale_error();
  const twopaco_options o = resolve(opt);
  RunView v;
  int rc = device_run_view(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, o, d_workspace,
                           workspace_bytes, nullptr, nullptr, 0, false, &v);
  if (rc) return rc;
  if (compute_cut != 0 && compute_cut != 1) return TWOPACO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);
  if (launch_init(v, s) < 0 || launch_pack(v, s) < 0) return TWOPACO_ECUDA;
  if (compute_cut && rounds > 1 && launch_partition(v, rounds, s) < 0) return TWOPACO_ECUDA;
  return TWOPACO_OK;
}

int twopaco_shard_rounds(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                         uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                         const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                         int shard, int n_shards, const uint32_t* d_class_cut) {
  clear_stale_error();
  const twopaco_options o = resolve(opt);
  RunView v;
  int rc = device_run_view(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, o, d_workspace,
                           workspace_bytes, nullptr, nullptr, 0, false, &v);
  if (rc) return rc;
  if (n_shards < 1 || shard < 0 || shard >= n_shards) return TWOPACO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);
  if (d_class_cut && rounds > 1 &&
      cudaMemcpyAsync(v.cuts, d_class_cut, 4 * ((uint64_t)rounds + 1), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return TWOPACO_ECUDA;
  v.count_round = shard;  // every shard counts the positions in its first round
  if (shard < rounds && launch_class_map(v, s) < 0) return TWOPACO_ECUDA;
  for (int r = shard; r < rounds; r += n_shards)
    if (launch_round(v, r, rounds, s) < 0) return TWOPACO_ECUDA;
  return TWOPACO_OK;
}

int twopaco_state_device(uint64_t total_bases, uint64_t n_seqs, int k, uint64_t filter_bits, int rounds,
                         const twopaco_options* opt, void* d_workspace, int which, void** d_ptr,
                         uint64_t* bytes) {
  const twopaco_options o = resolve(opt);
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (validate_size(total_bases) || !d_workspace || !d_ptr || !bytes) return TWOPACO_EINVAL;
  const Layout L = layout(total_bases, n_seqs, k, filter_bits, rounds, o);
  char* base = static_cast<char*>(d_workspace);
  switch (which) {
    case TWOPACO_STATE_CANDIDATES: *d_ptr = base + L.ctemp; *bytes = L.bitmap_words * 4; break;
    case TWOPACO_STATE_JUNCTIONS: *d_ptr = base + L.cfinal; *bytes = L.bitmap_words * 4; break;
    case TWOPACO_STATE_BINS:
      *d_ptr = rounds > 1 ? base + L.bins : nullptr;
      *bytes = rounds > 1 ? (uint64_t)o.partition_bins * 4 : 0;
      break;
    case TWOPACO_STATE_CUTS: *d_ptr = base + L.cuts; *bytes = ((uint64_t)rounds + 1) * 4; break;
    default: return TWOPACO_EINVAL;
  }
  return TWOPACO_OK;
}

int twopaco_run_device(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                       uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                       const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                       uint64_t* d_out_offsets, uint64_t* d_out_positions, uint64_t out_capacity) {
  return twopaco_run_rounds(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, opt,
                            d_workspace, workspace_bytes, 0, rounds < 1 ? 1 : rounds, d_out_offsets,
                            d_out_positions, out_capacity);
}

int twopaco_edges_device(const void* d_workspace, const uint64_t* d_offsets, uint64_t n_seqs,
                         const uint64_t* d_out_offsets, const uint64_t* d_out_positions,
                         uint64_t* d_edge_offsets, twopaco_edge* d_edges, uint64_t edge_capacity,
                         void* cuda_stream) {
  clear_stale_error();
  static_assert(sizeof(twopaco_edge) == 56, "twopaco_edge layout");
  if (!d_workspace || !d_out_offsets || !d_edge_offsets || (n_seqs && !d_offsets)) return TWOPACO_EINVAL;
  if (edge_capacity && !d_edges) return TWOPACO_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_workspace) % kAlign)) return TWOPACO_EINVAL;
  if (n_seqs >= (1ull << 32)) return TWOPACO_EINVAL;
  const int rc = launch_edges(static_cast<const DevHeader*>(d_workspace), d_offsets, n_seqs, d_out_offsets,
                              d_out_positions, d_edge_offsets, d_edges, edge_capacity,
                              static_cast<cudaStream_t>(cuda_stream));
  return rc < 0 ? TWOPACO_ECUDA : TWOPACO_OK;
}

}  // extern "C"

namespace twopaco {
namespace {

// The counters and failure flags of a run, from a copy of its header.
int stats_from_header(const DevHeader& h, twopaco_stats* stats) {
  stats->positions = h.positions;
  stats->pass1_marks = h.pass1_kept;
  stats->pass2_marks = h.pass2_kept;
  stats->table_slots = h.table_max;
  stats->bad_base_index = h.bad_inv ? ~h.bad_inv : ~0ull;
  stats->overflow = h.overflow | h.out_overflow;
  stats->timeout = h.timeout;
  stats->ordered_rounds = h.ord_rounds;
  stats->pad = 0;
  if (h.bad_inv) return TWOPACO_EBADBASE;
  if (h.timeout) return TWOPACO_ETIMEOUT;
  if (h.overflow || h.out_overflow) return TWOPACO_EOVERFLOW;
  return TWOPACO_OK;
}

// Output room a host build starts with: every k-mer position up to 2^27 of
// them (1 GiB), else an eighth of them; a run whose junctions do not fit
// writes its exact count, and the output is then written again into a buffer
// of that size (twopaco_run_rounds(..., rounds, rounds, ...)).
uint64_t first_output_capacity(uint64_t positions) {
  constexpr uint64_t kAll = 1ull << 27;
  const uint64_t c = positions <= kAll ? positions : std::max(kAll, positions / 8);
  return c ? c : 1;
}

}  // namespace
}  // namespace twopaco

extern "C" {

int twopaco_read_stats(const void* d_workspace, void* cuda_stream, twopaco_stats* stats) {
  if (!d_workspace || !stats) return TWOPACO_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_code(e);
  DevHeader h;
  e = cudaMemcpy(&h, d_workspace, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_code(e);
  return stats_from_header(h, stats);
}

int twopaco_read_state(const void* d_workspace, int which, void* host_dst, uint64_t bytes,
                       void* cuda_stream) {
  if (!d_workspace || (!host_dst && bytes)) return TWOPACO_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_code(e);
  DevHeader h;
  e = cudaMemcpy(&h, d_workspace, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_code(e);
  const void* src = nullptr;
  uint64_t avail = 0;
  switch (which) {
    case TWOPACO_STATE_CANDIDATES: src = h.ctemp; avail = h.bitmap_words * 4; break;
    case TWOPACO_STATE_JUNCTIONS: src = h.cfinal; avail = h.bitmap_words * 4; break;
    case TWOPACO_STATE_BINS: src = h.bins; avail = h.bins ? h.q * 4 : 0; break;
    case TWOPACO_STATE_CUTS: src = h.cuts; avail = (h.rounds + 1) * 4; break;
    default: return TWOPACO_EINVAL;
  }
  if (bytes > avail) return TWOPACO_EINVAL;
  if (!bytes) return TWOPACO_OK;
  return cuda_code(cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost));
}

// ---------------------------------------------------------------------------
// Checkpoints: the state between rounds (C_final, the class cut, counters)
// ---------------------------------------------------------------------------

}  // extern "C"

namespace twopaco {
namespace {

static_assert(offsetof(DevHeader, pass2_kept) == offsetof(DevHeader, positions) + 16,
              "positions, pass1_kept, pass2_kept are restored as one block");

struct CheckpointHead {
  char magic[8];  // "TPCKPT01"
  uint32_t version;
  int32_t k, rounds, hashes, both, split, next_round, lg_blocks, partial, reserved;
  uint64_t m, n_seqs, q, bitmap_words, input_digest;
  uint64_t positions, pass1_kept, pass2_kept, table_max;
  uint64_t checksum;  // checkpoint_checksum: this head (with this field 0) and the payload
};
static_assert(sizeof(CheckpointHead) == 128, "no padding: every byte of the head is checksummed");
constexpr char kCheckpointMagic[8] = {'T', 'P', 'C', 'K', 'P', 'T', '0', '1'};
constexpr uint32_t kCheckpointVersion = 3;

// Checksum of a whole checkpoint: the head with its checksum field zeroed,
// then the payload, so that a change to any field that steers the resume
// (next_round, the counters, the digest) is refused like a payload change.
uint64_t checkpoint_checksum(const CheckpointHead& head, const char* payload, uint64_t n) {
  CheckpointHead z = head;
  z.checksum = 0;
  return checksum_mix(payload_checksum(&z, sizeof(z)) + 0x9e3779b97f4a7c15ull) ^ payload_checksum(payload, n);
}

uint64_t checkpoint_bytes(uint64_t m, int rounds, uint64_t q) {
  const uint64_t words = (m + 31) / 32;
  return sizeof(CheckpointHead) + 4 * ((uint64_t)rounds + 1) + (rounds > 1 ? 4 * q : 0) + 4 * words;
}

}  // namespace
}  // namespace twopaco

extern "C" {

int twopaco_checkpoint_bytes(uint64_t total_bases, uint64_t n_seqs, int k, uint64_t filter_bits,
                             int rounds, const twopaco_options* opt, uint64_t* bytes) {
  const twopaco_options o = resolve(opt);
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (!bytes || validate_size(total_bases)) return TWOPACO_EINVAL;
  *bytes = checkpoint_bytes(total_bases, rounds, o.partition_bins);
  return TWOPACO_OK;
}

int twopaco_checkpoint_save(void* d_workspace, int next_round, void* host_dst, uint64_t bytes,
                            void* cuda_stream) {
  if (!d_workspace || !host_dst || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)) return TWOPACO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_code(e);
  DevHeader* hd = static_cast<DevHeader*>(d_workspace);
  DevHeader h;
  if ((e = cudaMemcpy(&h, hd, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_code(e);
  if (h.bad_inv) return TWOPACO_EBADBASE;
  if (h.timeout) return TWOPACO_ETIMEOUT;
  if (h.overflow) return TWOPACO_EOVERFLOW;
  if (!h.packed || next_round < 1 || (uint64_t)next_round > h.rounds) return TWOPACO_EINVAL;
  const int rounds = (int)h.rounds;
  if (bytes < checkpoint_bytes(h.m, rounds, h.q)) return TWOPACO_EINVAL;
  if (launch_digest(hd, h.packed, h.packed_words, h.offsets, h.n_seqs, h.nmask, h.bitmap_words, s) < 0)
    return TWOPACO_ECUDA;
  unsigned long long digest = 0;
  if ((e = cudaMemcpyAsync(&digest, &hd->input_digest, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_code(e);
  CheckpointHead c{};
  std::memcpy(c.magic, kCheckpointMagic, 8);
  c.version = kCheckpointVersion;
  c.k = h.k;
  c.rounds = rounds;
  c.hashes = h.hashes;
  c.both = h.both;
  c.split = h.nmask ? 1 : 0;
  c.next_round = next_round;
  c.lg_blocks = h.lg_blocks;
  c.partial = h.partial;
  c.m = h.m;
  c.n_seqs = h.n_seqs;
  c.q = h.q;
  c.bitmap_words = h.bitmap_words;
  c.input_digest = digest;
  c.positions = h.positions;
  c.pass1_kept = h.pass1_kept;
  c.pass2_kept = h.pass2_kept;
  c.table_max = h.table_max;
  char* out = static_cast<char*>(host_dst);
  out += sizeof(c);
  if ((e = cudaMemcpy(out, h.cuts, 4 * ((uint64_t)rounds + 1), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_code(e);
  out += 4 * ((uint64_t)rounds + 1);
  if (rounds > 1) {
    if ((e = cudaMemcpy(out, h.bins, 4 * h.q, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_code(e);
    out += 4 * h.q;
  }
  if (h.bitmap_words && (e = cudaMemcpy(out, h.cfinal, 4 * h.bitmap_words, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_code(e);
  // the head last, with the checksum of itself and the payload just written
  c.checksum = checkpoint_checksum(c, static_cast<const char*>(host_dst) + sizeof(c),
                                   checkpoint_bytes(h.m, rounds, h.q) - sizeof(c));
  std::memcpy(host_dst, &c, sizeof(c));
  return TWOPACO_OK;
}

int twopaco_checkpoint_load(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                            uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                            const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                            const void* host_src, uint64_t bytes, int* next_round) {
  clear_stale_error();
  const twopaco_options o = resolve(opt);
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (validate_size(total_bases) || !host_src || !next_round) return TWOPACO_EINVAL;
  if (total_bases > 0 && (n_seqs == 0 || !d_bases || !d_offsets)) return TWOPACO_EINVAL;
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)) return TWOPACO_EINVAL;
  const Layout L = layout(total_bases, n_seqs, k, filter_bits, rounds, o);
  if (workspace_bytes < L.total) return TWOPACO_EINVAL;
  if (bytes < sizeof(CheckpointHead)) return TWOPACO_EINVAL;
  CheckpointHead c;
  std::memcpy(&c, host_src, sizeof(c));
  const uint64_t q = o.partition_bins;
  if (std::memcmp(c.magic, kCheckpointMagic, 8) || c.version != kCheckpointVersion || c.k != k || c.rounds != rounds ||
      c.hashes != o.hashes || c.both != o.both_strands || c.split != o.split_at_n || c.partial != o.partial ||
      c.lg_blocks != log2_exact(filter_bits / 256) || c.m != total_bases || c.n_seqs != n_seqs ||
      c.q != q || c.bitmap_words != L.bitmap_words || c.next_round < 1 || c.next_round > rounds ||
      bytes < checkpoint_bytes(total_bases, rounds, q))
    return TWOPACO_EINVAL;
  // a head or payload changed since it was saved is refused
  const char* payload = static_cast<const char*>(host_src) + sizeof(c);
  if (checkpoint_checksum(c, payload, checkpoint_bytes(total_bases, rounds, q) - sizeof(c)) != c.checksum)
    return TWOPACO_EINVAL;
  // a class cut must cover the q bins in rounds non-empty, ascending ranges
  // (written only for rounds > 1 and a non-empty input)
  if (rounds > 1 && total_bases > 0) {
    std::vector<uint32_t> cuts((size_t)rounds + 1);
    std::memcpy(cuts.data(), payload, 4 * cuts.size());
    if (cuts[0] != 0 || cuts[rounds] != q) return TWOPACO_EINVAL;
    for (int r = 0; r < rounds; ++r)
      if (cuts[r] >= cuts[r + 1]) return TWOPACO_EINVAL;
  }
  // the input, packed again, must be the one the checkpoint was taken on
  const RunView v = make_view(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, o, L,
                              d_workspace, nullptr, nullptr, 0);
  cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);
  DevHeader* hd = v.hdr;
  if (launch_init(v, s) < 0 || launch_pack(v, s) < 0) return TWOPACO_ECUDA;
  if (launch_digest(hd, v.packed, v.packed_words, v.offsets, n_seqs, v.nmask, v.bitmap_words, s) < 0)
    return TWOPACO_ECUDA;
  unsigned long long digest = 0, bad = 0;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&digest, &hd->input_digest, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&bad, &hd->bad_inv, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_code(e);
  if (bad) return TWOPACO_EBADBASE;
  if (digest != c.input_digest) return TWOPACO_EINVAL;
  const char* in = payload;
  if ((e = cudaMemcpyAsync(v.cuts, in, 4 * ((uint64_t)rounds + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_code(e);
  in += 4 * ((uint64_t)rounds + 1);
  if (rounds > 1) {
    if ((e = cudaMemcpyAsync(v.bins, in, 4 * q, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_code(e);
    in += 4 * q;
  }
  if (v.bitmap_words &&
      (e = cudaMemcpyAsync(v.cfinal, in, 4 * v.bitmap_words, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_code(e);
  if (launch_class_map(v, s) < 0) return TWOPACO_ECUDA;  // the remaining rounds' classes, from the restored cut
  const unsigned long long counters[3] = {c.positions, c.pass1_kept, c.pass2_kept};
  if ((e = cudaMemcpyAsync(&hd->positions, counters, sizeof(counters), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&hd->table_max, &c.table_max, 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_code(e);
  *next_round = c.next_round;
  return TWOPACO_OK;
}

int twopaco_selftest_bounded_wait(void* cuda_stream) {
  clear_stale_error();
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* word = nullptr;
  unsigned int* status = nullptr;
  cudaError_t e = cudaMalloc(&word, 16);
  if (e != cudaSuccess) return cuda_code(e);
  status = reinterpret_cast<unsigned int*>(word + 1);
  unsigned int got = 0;
  if ((e = cudaMemsetAsync(word, 0, 16, s)) == cudaSuccess) {
    if (launch_bounded_wait(word, status, s) < 0) e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&got, status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(word);
  if (e != cudaSuccess) return cuda_code(e);
  return got == 1 ? TWOPACO_ETIMEOUT : (got == 2 ? TWOPACO_OK : TWOPACO_ECUDA);
}

void twopaco_result_free(twopaco_result* res) {
  if (!res) return;
  std::free(res->offsets);
  std::free(res->positions);
  std::free(res);
}

int twopaco_build(const char* const* seqs, const uint64_t* lengths, uint64_t n_seqs, int k,
                  uint64_t filter_bits, int rounds, twopaco_result** out) {
  return twopaco_build_ex(seqs, lengths, n_seqs, k, filter_bits, rounds, nullptr, out);
}

int twopaco_build_ex(const char* const* seqs, const uint64_t* lengths, uint64_t n_seqs, int k,
                     uint64_t filter_bits, int rounds, const twopaco_options* opt,
                     twopaco_result** out) {
  if (!out) return TWOPACO_EINVAL;
  *out = nullptr;
  twopaco_options o = resolve(opt);
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (n_seqs && (!seqs || !lengths)) return TWOPACO_EINVAL;
  std::vector<uint64_t> offsets(n_seqs + 1, 0);
  uint64_t positions = 0;
  for (uint64_t t = 0; t < n_seqs; ++t) {
    if (lengths[t] && !seqs[t]) return TWOPACO_EINVAL;
    offsets[t + 1] = offsets[t] + lengths[t];
    if (lengths[t] >= (uint64_t)k) positions += lengths[t] - (uint64_t)k + 1;
  }
  const uint64_t m = offsets[n_seqs];
  if (validate_size(m)) return TWOPACO_EINVAL;
  raise_run_capacity(&o, seqs, lengths, n_seqs);
  cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);

  uint8_t* d_bases = nullptr;
  uint64_t* d_off = nullptr;
  uint64_t* d_out_off = nullptr;
  uint64_t* d_pos = nullptr;
  void* d_ws = nullptr;
  twopaco_result* res = nullptr;
  twopaco_stats st{};
  auto fail = [&](int code) {
    cudaStreamSynchronize(s);
    cudaFree(d_bases);
    cudaFree(d_off);
    cudaFree(d_out_off);
    cudaFree(d_pos);
    cudaFree(d_ws);
    if (res) twopaco_result_free(res);
    return code;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&d_bases, m ? m : 1)) != cudaSuccess) return fail(cuda_code(e));
  if ((e = cudaMalloc(&d_off, (n_seqs + 1) * 8)) != cudaSuccess) return fail(cuda_code(e));
  if ((e = cudaMalloc(&d_out_off, (n_seqs + 1) * 8)) != cudaSuccess) return fail(cuda_code(e));
  uint64_t out_cap = first_output_capacity(positions);
  if ((e = cudaMalloc(&d_pos, out_cap * 8)) != cudaSuccess) return fail(cuda_code(e));
  for (uint64_t t = 0; t < n_seqs; ++t) {
    if (!lengths[t]) continue;
    e = cudaMemcpyAsync(d_bases + offsets[t], seqs[t], lengths[t], cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(cuda_code(e));
  }
  e = cudaMemcpyAsync(d_off, offsets.data(), (n_seqs + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(cuda_code(e));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_code(e));

  for (int attempt = 0;; ++attempt) {
    uint64_t ws = 0;
    if ((rc = twopaco_workspace_size(m, n_seqs, k, filter_bits, rounds, &o, &ws))) return fail(rc);
    if ((e = cudaMalloc(&d_ws, ws)) != cudaSuccess) return fail(cuda_code(e));
    rc = twopaco_run_device(d_bases, d_off, n_seqs, m, k, filter_bits, rounds, &o, d_ws, ws,
                            d_out_off, d_pos, out_cap);
    if (rc) return fail(rc);
    rc = twopaco_read_stats(d_ws, o.cuda_stream, &st);
    if (rc == TWOPACO_EOVERFLOW) {
      DevHeader h;
      if ((e = cudaMemcpy(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(cuda_code(e));
      if (!h.overflow && h.out_overflow) {
        // only the output was too small: it holds the exact count; write it again
        uint64_t total = 0;
        if ((e = cudaMemcpy(&total, d_out_off + n_seqs, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
          return fail(cuda_code(e));
        cudaFree(d_pos);
        d_pos = nullptr;
        out_cap = total ? total : 1;
        if ((e = cudaMalloc(&d_pos, out_cap * 8)) != cudaSuccess) return fail(cuda_code(e));
        rc = twopaco_run_rounds(d_bases, d_off, n_seqs, m, k, filter_bits, rounds, &o, d_ws, ws, rounds,
                                rounds, d_out_off, d_pos, out_cap);
        if (rc) return fail(rc);
        rc = twopaco_read_stats(d_ws, o.cuda_stream, &st);
      }
    }
    if (rc != TWOPACO_EOVERFLOW || attempt >= 4) break;
    // The table was too small for this input: grow it and run again.
    const Layout L = layout(m, n_seqs, k, filter_bits, rounds, o);
    o.table_slots = L.table_slots * 4;
    cudaFree(d_ws);
    d_ws = nullptr;
  }
  if (rc) return fail(rc);

  res = static_cast<twopaco_result*>(std::calloc(1, sizeof(twopaco_result)));
  if (!res) return fail(TWOPACO_ENOMEM);
  res->n_seqs = n_seqs;
  res->stats = st;
  res->offsets = static_cast<uint64_t*>(std::malloc((n_seqs + 1) * 8));
  res->positions = static_cast<uint64_t*>(std::malloc((st.pass2_marks ? st.pass2_marks : 1) * 8));
  if (!res->offsets || !res->positions) return fail(TWOPACO_ENOMEM);
  if ((e = cudaMemcpy(res->offsets, d_out_off, (n_seqs + 1) * 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(cuda_code(e));
  if (st.pass2_marks &&
      (e = cudaMemcpy(res->positions, d_pos, st.pass2_marks * 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(cuda_code(e));
  twopaco_result* done = res;
  res = nullptr;
  fail(TWOPACO_OK);
  *out = done;
  return TWOPACO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Captured runs
// ---------------------------------------------------------------------------

struct twopaco_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;  // library kernels in one replay
};

extern "C" {

int twopaco_plan_create(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                        uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                        const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                        uint64_t* d_out_offsets, uint64_t* d_out_positions, uint64_t out_capacity,
                        twopaco_plan** plan) {
  clear_stale_error();
  if (!plan) return TWOPACO_EINVAL;
  *plan = nullptr;
  twopaco_options o = resolve(opt);
  if (o.per_string_launches) return TWOPACO_EINVAL;  // they read the offsets back: no capture
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_code(e);
  o.cuda_stream = cs;
  twopaco_plan* p = new (std::nothrow) twopaco_plan();
  if (!p) {
    cudaStreamDestroy(cs);
    return TWOPACO_ENOMEM;
  }
  const unsigned long long before = launches_so_far();
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? TWOPACO_OK : cuda_code(e);
  if (rc == TWOPACO_OK) {
    rc = twopaco_run_device(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, &o,
                            d_workspace, workspace_bytes, d_out_offsets, d_out_positions, out_capacity);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);  // always end the capture, even after an error
    if (rc == TWOPACO_OK && e != cudaSuccess) rc = cuda_code(e);
    p->graph = g;
  }
  // the captured launches did not run: take them back out of the count
  p->kernels = launches_so_far() - before;
  count_launches(-(int)p->kernels);
  if (rc == TWOPACO_OK) {
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) rc = cuda_code(e);
  }
  cudaStreamDestroy(cs);
  if (rc != TWOPACO_OK) {
    twopaco_plan_destroy(p);
    return rc;
  }
  *plan = p;
  return TWOPACO_OK;
}

int twopaco_plan_launch(twopaco_plan* p, void* cuda_stream) {
  if (!p || !p->exec) return TWOPACO_EINVAL;
  cudaError_t e = cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_code(e);
  count_launches((int)p->kernels);
  return TWOPACO_OK;
}

void twopaco_plan_destroy(twopaco_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  delete p;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Reusable context
// ---------------------------------------------------------------------------

struct twopaco_context {
  int device = 0;
  cudaStream_t stream = nullptr;  // copies and kernels (spreading the copies over more streams
                                  // measured slower: one already fills the host link)
  twopaco::DevHeader* h_hdr = nullptr;  // pinned: the last run's header
  uint8_t* d_bases = nullptr;
  uint64_t cap_bases = 0;
  uint64_t* d_off = nullptr;
  uint64_t cap_d_off = 0;
  uint64_t* d_out_off = nullptr;
  uint64_t cap_d_out_off = 0;
  uint64_t* d_pos = nullptr;
  uint64_t cap_pos = 0;
  void* d_ws = nullptr;
  uint64_t cap_ws = 0;
  uint64_t* h_off = nullptr;      // pinned: input offsets
  uint64_t cap_h_off = 0;
  uint64_t* h_out_off = nullptr;  // pinned: result offsets
  uint64_t cap_h_out_off = 0;
  uint64_t* h_pos = nullptr;      // pinned: result positions
  uint64_t cap_hpos = 0;
  // the last build, for twopaco_edges_ctx
  uint64_t last_n = 0, last_junctions = 0;
  bool have_last = false;
  uint64_t* d_edge_off = nullptr;
  uint64_t cap_d_edge_off = 0;
  twopaco_edge* d_edges = nullptr;
  uint64_t cap_d_edges = 0;
  uint64_t* h_edge_off = nullptr;
  uint64_t cap_h_edge_off = 0;
  twopaco_edge* h_edges = nullptr;
  uint64_t cap_h_edges = 0;
};

namespace {

// Grow a device buffer to at least `need` bytes (contents are not kept).
template <typename T>
cudaError_t grow_device(T** p, uint64_t* cap, uint64_t need) {
  if (*cap >= need && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), need ? need : 1);
  if (e == cudaSuccess) *cap = need;
  return e;
}

template <typename T>
cudaError_t grow_pinned(T** p, uint64_t* cap, uint64_t need) {
  if (*cap >= need && *p) return cudaSuccess;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(p), need ? need : 1);
  if (e == cudaSuccess) *cap = need;
  return e;
}

}  // namespace

extern "C" {

int twopaco_context_create(twopaco_context** ctx) {
  if (!ctx) return TWOPACO_EINVAL;
  *ctx = nullptr;
  twopaco_context* c = new (std::nothrow) twopaco_context();
  if (!c) return TWOPACO_ENOMEM;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_hdr, sizeof(twopaco::DevHeader));
  if (e != cudaSuccess) {
    twopaco_context_destroy(c);
    return cuda_code(e);
  }
  *ctx = c;
  return TWOPACO_OK;
}

void twopaco_context_destroy(twopaco_context* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_bases);
  cudaFree(c->d_off);
  cudaFree(c->d_out_off);
  cudaFree(c->d_pos);
  cudaFree(c->d_ws);
  cudaFreeHost(c->h_off);
  cudaFreeHost(c->h_out_off);
  cudaFreeHost(c->h_pos);
  cudaFree(c->d_edge_off);
  cudaFree(c->d_edges);
  cudaFreeHost(c->h_edge_off);
  cudaFreeHost(c->h_edges);
  cudaFreeHost(c->h_hdr);
  if (c->stream) cudaStreamDestroy(c->stream);
  cudaSetDevice(prev);
  delete c;
}

int twopaco_build_ctx(twopaco_context* c, const char* const* seqs, const uint64_t* lengths,
                      uint64_t n_seqs, int k, uint64_t filter_bits, int rounds,
                      const twopaco_options* opt, twopaco_result* out) {
  clear_stale_error();
  if (!c || !out) return TWOPACO_EINVAL;
  twopaco_options o = resolve(opt);
  int rc = validate(n_seqs, k, filter_bits, rounds, o);
  if (rc) return rc;
  if (n_seqs && (!seqs || !lengths)) return TWOPACO_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  o.cuda_stream = c->stream;
  auto finish = [&](int code) {
    if (prev != c->device) cudaSetDevice(prev);
    return code;
  };
  cudaError_t e;
  const uint64_t off_bytes = (n_seqs + 1) * 8;
  if ((e = grow_pinned(&c->h_off, &c->cap_h_off, off_bytes)) != cudaSuccess ||
      (e = grow_pinned(&c->h_out_off, &c->cap_h_out_off, off_bytes)) != cudaSuccess ||
      (e = grow_device(&c->d_off, &c->cap_d_off, off_bytes)) != cudaSuccess ||
      (e = grow_device(&c->d_out_off, &c->cap_d_out_off, off_bytes)) != cudaSuccess)
    return finish(cuda_code(e));
  uint64_t positions = 0;
  c->h_off[0] = 0;
  for (uint64_t t = 0; t < n_seqs; ++t) {
    if (lengths[t] && !seqs[t]) return finish(TWOPACO_EINVAL);
    c->h_off[t + 1] = c->h_off[t] + lengths[t];
    if (lengths[t] >= (uint64_t)k) positions += lengths[t] - (uint64_t)k + 1;
  }
  const uint64_t m = c->h_off[n_seqs];
  if (validate_size(m)) return finish(TWOPACO_EINVAL);
  raise_run_capacity(&o, seqs, lengths, n_seqs);
  if ((e = grow_device(&c->d_bases, &c->cap_bases, m)) != cudaSuccess) return finish(cuda_code(e));
  if ((e = grow_device(&c->d_pos, &c->cap_pos, first_output_capacity(positions) * 8)) != cudaSuccess)
    return finish(cuda_code(e));
  for (uint64_t t = 0; t < n_seqs; ++t) {
    if (!lengths[t]) continue;
    e = cudaMemcpyAsync(c->d_bases + c->h_off[t], seqs[t], lengths[t], cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return finish(cuda_code(e));
  }
  e = cudaMemcpyAsync(c->d_off, c->h_off, (n_seqs + 1) * 8, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return finish(cuda_code(e));
  twopaco_stats st{};
  for (int attempt = 0;; ++attempt) {
    uint64_t ws = 0;
    if ((rc = twopaco_workspace_size(m, n_seqs, k, filter_bits, rounds, &o, &ws))) return finish(rc);
    if ((e = grow_device(reinterpret_cast<char**>(&c->d_ws), &c->cap_ws, ws)) != cudaSuccess)
      return finish(cuda_code(e));
    rc = twopaco_run_device(c->d_bases, c->d_off, n_seqs, m, k, filter_bits, rounds, &o, c->d_ws, ws,
                            c->d_out_off, c->d_pos, c->cap_pos / 8);
    if (rc) return finish(rc);
    e = cudaMemcpyAsync(c->h_out_off, c->d_out_off, (n_seqs + 1) * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->h_hdr, c->d_ws, sizeof(DevHeader), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return finish(cuda_code(e));
    rc = stats_from_header(*c->h_hdr, &st);
    if (rc == TWOPACO_EOVERFLOW && !c->h_hdr->overflow && c->h_hdr->out_overflow) {
      // only the output was too small: it holds the exact count; write it again
      const uint64_t total = c->h_out_off[n_seqs];
      if ((e = grow_device(&c->d_pos, &c->cap_pos, (total ? total : 1) * 8)) != cudaSuccess)
        return finish(cuda_code(e));
      rc = twopaco_run_rounds(c->d_bases, c->d_off, n_seqs, m, k, filter_bits, rounds, &o, c->d_ws, ws,
                              rounds, rounds, c->d_out_off, c->d_pos, c->cap_pos / 8);
      if (rc) return finish(rc);
      e = cudaMemcpyAsync(c->h_hdr, c->d_ws, sizeof(DevHeader), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return finish(cuda_code(e));
      rc = stats_from_header(*c->h_hdr, &st);
    }
    if (rc != TWOPACO_EOVERFLOW || attempt >= 4) break;
    o.table_slots = layout(m, n_seqs, k, filter_bits, rounds, o).table_slots * 4;
  }
  if (rc) return finish(rc);
  const uint64_t total = c->h_out_off[n_seqs];
  if ((e = grow_pinned(&c->h_pos, &c->cap_hpos, (total ? total : 1) * 8)) != cudaSuccess)
    return finish(cuda_code(e));
  if (total) {
    e = cudaMemcpyAsync(c->h_pos, c->d_pos, total * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return finish(cuda_code(e));
  }
  out->n_seqs = n_seqs;
  out->offsets = c->h_out_off;
  out->positions = c->h_pos;
  out->stats = st;
  c->last_n = n_seqs;
  c->last_junctions = total;
  c->have_last = true;
  return finish(TWOPACO_OK);
}

int twopaco_edges_ctx(twopaco_context* c, twopaco_edge_list* out) {
  clear_stale_error();
  if (!c || !out || !c->have_last) return TWOPACO_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  auto finish = [&](int code) {
    if (prev != c->device) cudaSetDevice(prev);
    return code;
  };
  const uint64_t n = c->last_n, cap = c->last_junctions ? c->last_junctions : 1;
  cudaError_t e;
  if ((e = grow_device(&c->d_edge_off, &c->cap_d_edge_off, (n + 1) * 8)) != cudaSuccess ||
      (e = grow_device(&c->d_edges, &c->cap_d_edges, cap * sizeof(twopaco_edge))) != cudaSuccess ||
      (e = grow_pinned(&c->h_edge_off, &c->cap_h_edge_off, (n + 1) * 8)) != cudaSuccess ||
      (e = grow_pinned(&c->h_edges, &c->cap_h_edges, cap * sizeof(twopaco_edge))) != cudaSuccess)
    return finish(cuda_code(e));
  int rc = twopaco_edges_device(c->d_ws, c->d_off, n, c->d_out_off, c->d_pos, c->d_edge_off, c->d_edges,
                                cap, c->stream);
  if (rc) return finish(rc);
  e = cudaMemcpyAsync(c->h_edge_off, c->d_edge_off, (n + 1) * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return finish(cuda_code(e));
  const uint64_t ne = c->h_edge_off[n];
  if (ne > cap) return finish(TWOPACO_EOVERFLOW);
  if (ne) {
    e = cudaMemcpyAsync(c->h_edges, c->d_edges, ne * sizeof(twopaco_edge), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return finish(cuda_code(e));
  }
  out->n_seqs = n;
  out->offsets = c->h_edge_off;
  out->edges = c->h_edges;
  return finish(TWOPACO_OK);
}

}  // extern "C"
