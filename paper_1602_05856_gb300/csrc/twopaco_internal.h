// Internal declarations shared by the kernels and the C-ABI layer of the
// junction-detection library. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

namespace twopaco {

// Counters and failure flags kept at the start of the workspace.
struct DevHeader {
  unsigned long long bad_inv;      // ~(smallest invalid byte index), 0 if none
  unsigned long long positions;    // k-mer positions in the input
  unsigned long long pass1_kept;   // candidates after pass 1, all rounds
  unsigned long long pass2_kept;   // junction positions
  unsigned long long round_kept;   // candidates after pass 1, current round
  unsigned long long table_slots;  // pass-2 table capacity of the current round
  unsigned long long table_max;    // largest capacity used by any round
  unsigned long long lc_set;       // linear-counting bits set this round
  unsigned int cand_overflow;      // a warp's list segment ran out of room this round
  unsigned int round_listed;       // pass 2 of this round reads the list (else C_temp)
  unsigned int lc_blocks_done;     // blocks of lc_count finished this round
  unsigned int list_parts;         // pass-2 parts per list segment this round
  unsigned long long emit_ticket;  // next emit tile to claim
  unsigned int overflow;           // the pass-2 table or a boundary list out of room
  unsigned int timeout;            // a bounded wait gave up
  // where the last run left its bitmaps and partition state (for inspection)
  uint32_t* ctemp;
  uint32_t* cfinal;
  uint32_t* bins;
  uint32_t* cuts;
  unsigned long long bitmap_words;
  unsigned long long q;
  unsigned long long rounds;
  // what a later edge computation needs from the run
  const uint32_t* packed;
  unsigned long long m;
  int k;
  int both;
  // N splitting (null / 0 without it): the N mask, the sorted boundaries of
  // the N-free pieces and N runs, and (after an edge computation) their ranks
  const uint32_t* nmask;
  const uint64_t* runs;
  uint32_t* run_rank;
  unsigned long long n_runs;
  unsigned long long run_cap;
  // what a checkpoint records about the run (and the input it digests)
  const uint64_t* offsets;
  unsigned long long n_seqs;
  int hashes;
  int lg_blocks;
  int partial;
  unsigned long long packed_words;
  unsigned long long input_digest;  // written by launch_digest
  unsigned int out_overflow;        // the output positions did not fit (the offsets are exact)
  unsigned int ord_ok;              // region-ordered first pass: this round's records fit
  unsigned int ord_ticket[3];       // region-ordered first pass: apply, probe and classify work items
  unsigned int ord_rounds;          // rounds the region-ordered kernels took
};

// Device view of one run: every buffer lives inside the workspace except the
// caller's input and output arrays.
struct RunView {
  const uint8_t* bases;     // caller's ASCII, m bytes
  const uint64_t* offsets;  // caller's n + 1 string offsets
  uint32_t n_seqs;
  uint64_t m;               // total bases
  int k;
  int both;                 // comprehensive graph
  int hashes;               // bits per filter item
  int rounds;               // classes of Algorithm 3
  int partial;              // omit pass 2: C_final gathers every round's C_temp
  int count_round;          // the round whose probe counts the input's k-mer positions
  int blocks_per_sm;        // resident blocks per SM of the pass kernels' grids (0: all that fit)
  uint64_t p_begin, p_end;  // positions the first- and second-pass loops visit: all
                            // ([0, m)) or, launched per string, whole tiles of kRangeTile
  int lg_blocks;            // log2(filter_bits / 256)
  uint32_t qmask;           // partition_bins - 1
  uint32_t part_sample;     // the partition pre-pass counts the k-mers whose H has bits
                            // 16 .. 16 + log2(part_sample + 1) - 1 all zero (0: every k-mer)
  uint32_t part_chunks;     // ... and walks the chunks of 65536 positions whose index has these
                            // bits zero (0: every chunk)
  DevHeader* hdr;
  uint32_t* packed;         // 2-bit packed input, ceil(m/16) + pad words
  uint64_t packed_words;    // words written by the pack kernel (incl. pad)
  unsigned long long* filter;  // filter_bits / 64 words
  uint64_t filter_words64;
  uint32_t* ctemp;          // C_temp bitmap, one bit per base
  uint32_t* cfinal;         // C_final bitmap
  uint64_t bitmap_words;    // ceil(m/32)
  void* table;              // pass-2 slots
  uint64_t table_max_slots;
  uint64_t* cands;          // positions of the pass-1 survivors, for pass 2
  int narrow;               // m < 2^31: the list holds 32-bit records
  uint32_t* cand_slot;      // table slot of every listed candidate (null: look it up)
  // N splitting (nmask null without it): bit g of nmask = base g is N; the
  // boundary bitmap (string starts and N/base changes), its per-chunk counts,
  // and the sorted boundaries runs[0 .. n_runs] (runs[n_runs] = m)
  uint32_t* nmask;
  uint32_t* bound_bits;
  uint64_t* chunk_counts;
  uint64_t n_chunks;
  uint64_t* runs;
  uint32_t* run_rank;
  uint64_t run_cap;
  uint64_t* desc;           // per-position probe descriptors (use_desc), m + 16 entries
  // region-bucketed first-pass inserts (n_regions > 0): records of the ORs into
  // each filter region of 2^lg_region_words 64-bit words, applied region by region
  uint32_t n_regions;
  uint32_t n_sub;           // buckets per region (a power of two)
  int lg_region_words;
  uint32_t* bucket_fill;    // records appended per bucket, one counter per 128 bytes, then the apply ticket
  uint64_t* bucket_recs;    // n_regions * n_sub buckets of bucket_cap records
  uint64_t bucket_cap;
  uint64_t bucket_chunk;    // positions per scatter-and-apply chunk (a multiple of kRangeTile)
  // region-ordered first pass (o_regions > 0; class-map rounds): the class map
  // also records every position's filter region (rplane) and counts the
  // positions of every tile per (class, region) pair and per (class, warp
  // chunk); a round then writes one 8-byte record per position of its class
  // into the bucket of its region, applies the ORs and the probes bucket by
  // bucket, and gathers the decisions back in position order
  uint32_t o_regions;       // filter regions (buckets), at most kOrdMaxRegions
  int o_lg_region_words;    // log2 of the 64-bit words per region (at most 22)
  uint8_t* rplane;          // region of every position's k-mer, one byte per position
  uint16_t* o_thist;        // per tile, class and region: its positions (tile-major)
  uint16_t* o_wcount;       // per class, tile and warp chunk of kOrdTile / 8 positions: its positions
  uint32_t* o_csum;         // per chunk of kOrdScanTiles tiles and bucket: the round's members
  unsigned long long* o_cpre;  // per chunk and bucket: the round's members in the chunks before
  unsigned long long* o_btot;  // per bucket: the round's members
  uint64_t* o_start;        // o_regions + 1 bucket starts of the current round (multiples of 32)
  uint32_t* o_fill;         // records claimed per bucket, one counter per 128 bytes
  uint64_t* o_recs;         // o_rec_cap records
  uint64_t o_rec_cap;
  uint32_t* o_dec;          // one decision bit per record slot; fused: word pairs (candidates,
                            // junctions) per 32 slots
  uint32_t* o_meta;         // per tile and bucket: where the tile's records start in the bucket
  uint64_t o_tiles;         // tiles of kOrdTile positions: ceil(m / kOrdTile)
  uint32_t* o_tcount;       // positions of every class in every tile (rounds x o_tiles)
  unsigned long long* o_tbase;  // members of the round in the tiles before (rounds x o_tiles)
  unsigned long long* o_tsum;   // members of the round per scan chunk of tiles
  uint16_t* o_perm;         // per member of the round: its rank within its tile's room
  int o_fused;              // k <= 27, not partial: pass 2 runs on the records (fused records)
  uint32_t o_tcap;          // fused: table slots per bucket (region), the table is o_regions x o_tcap slots
  int use_desc;             // the insert leaves descriptors and the probe reads them
  uint64_t cand_cap;        // records the list can hold
  uint32_t* seg_count;      // candidates per list segment (one segment per probe warp)
  uint32_t n_segments;      // warps of the probe grid (set per launch)
  uint64_t seg_cap;         // records per segment (set per launch)
  uint32_t* lc_bits;        // linear-counting bitmap, 2^lc_log2 bits
  int lc_log2;
  int lc_sample_log2;       // region-ordered rounds count a 2^-lc_sample_log2 sample of the k-mers
  uint32_t* bins;           // partition counters (q), rounds > 1
  uint32_t* cuts;           // rounds + 1 class boundaries
  uint8_t* cmap;            // class map, one byte per position (null: rounds walk every position)
  uint32_t* tile_count;     // emit: junctions per tile
  uint64_t* tile_prefix;    // emit: exclusive prefix per tile
  uint64_t n_tiles;
  uint64_t* out_offsets;    // caller's n + 1
  uint64_t* out_positions;  // caller's capacity
  uint64_t out_capacity;
};

constexpr int kBlock = 256;             // threads per block of the position kernels
constexpr int kEmitWordsPerThread = 8;
constexpr int kEmitTileWords = kBlock * kEmitWordsPerThread;  // bitmap words per emit tile
constexpr uint64_t kPackPadWords = 16;  // zero words after the packed input (window reads of k <= 127 stay inside)
constexpr uint32_t kMaxSegments = 65536; // candidate-list segments (probe warps) at most
constexpr uint64_t kRunChunkWords = 1024;  // boundary-bitmap words per compaction chunk
constexpr int kMaxMapRounds = 64;          // rounds a class map can tell apart (6 class bits)
constexpr uint64_t kRangeTile = 4096;      // positions: the unit of per-string launch ranges
constexpr uint32_t kMaxRegions = 1024;     // filter regions of bucketed inserts, at most
constexpr uint32_t kMinBuckets = 256;      // buckets of bucketed inserts, at least (sub-buckets per region)
constexpr uint32_t kMaxBuckets = 1024;
constexpr int kRegionWordsLog2 = 22;       // 32 MiB regions (words of 8 bytes)
constexpr uint32_t kCmWindowPositions = 512;  // positions per class-map window (one warp's)
constexpr int kOrdTileWindows = 32;        // region-ordered first pass: windows per tile
constexpr uint64_t kOrdTile = (uint64_t)kOrdTileWindows * kCmWindowPositions;  // 16384 positions
constexpr uint32_t kOrdMaxRegions = 256;   // buckets (filter regions), at most
constexpr uint32_t kOrdMaxHist = 4096;     // rounds x regions, at most
constexpr uint32_t kOrdFillStride = 32;    // bucket fill counters 128 bytes apart
constexpr uint32_t kOrdScanTiles = 1024;   // tiles per block of the member-number scan

// Kernel launch helpers (twopaco_kernels.cu). Each returns the number of
// kernels it launched, or -1 after a launch error.
int launch_init(const RunView& v, cudaStream_t s);  // clears the header
int launch_pack(const RunView& v, cudaStream_t s);
// The pack in pieces: the packed words [w_begin, w_end) from v.bases (first:
// also the header and the first round's clears), then, once every word is
// packed, the piece boundaries of N splitting.
int launch_pack_chunk(const RunView& v, uint64_t w_begin, uint64_t w_end, bool first, cudaStream_t s);
int launch_pack_finish(const RunView& v, cudaStream_t s);
int launch_partition(const RunView& v, int rounds, cudaStream_t s);
// ranges: null, or the [begin, end) position ranges (multiples of kRangeTile but the
// last) of launches issued one per string for every loop of the round.
int launch_round(const RunView& v, int round, int rounds, cudaStream_t s,
                 const std::vector<std::pair<uint64_t, uint64_t>>* ranges = nullptr);
// The class map of a run with rounds > 1 (v.cmap), from the class cut in
// v.cuts; launches nothing without a class map.
int launch_class_map(const RunView& v, cudaStream_t s);
int launch_emit(const RunView& v, cudaStream_t s, bool again = false);
int launch_edges(const DevHeader* hdr_dev, const uint64_t* d_offsets, uint64_t n_seqs,
                 const uint64_t* d_out_offsets, const uint64_t* d_out_positions,
                 uint64_t* d_edge_offsets, void* d_edges, uint64_t edge_capacity, cudaStream_t s);

// Pass-2 slot layout for this k: 0 = one 64-bit word (key << 9 | mask, k <= 27),
// 1 = 16 bytes (k <= 31), 2 = 32 bytes (128-bit key).
// Pass-2 table slots: 0 = one word (key << 9 | mask, k <= 27); 1 = 16 B key +
// mask (k <= 31); 2 = 32 B 128-bit key + mask (k <= 63); 3 = 16 B reference
// to an occurrence + mask (k <= 127).
inline int table_slot_kind(int k) { return k <= 27 ? 0 : (k <= 31 ? 1 : (k <= 63 ? 2 : 3)); }
inline uint64_t table_slot_bytes(int k) {
  const int t = table_slot_kind(k);
  return t == 3 ? 16ull : (8ull << t);
}

// Bytes per candidate record (a global position).
inline uint64_t cand_record_bytes(int) { return 8; }

// The k > 63 halves of launch_round and of the partition pre-pass (compiled
// in twopaco_kernels_wide.cu).
int launch_round_wide(const RunView& v, int round, int rounds, cudaStream_t s,
                      const std::vector<std::pair<uint64_t, uint64_t>>* ranges);
int launch_partition_count_wide(const RunView& v, cudaStream_t s);
int launch_class_map_wide(const RunView& v, cudaStream_t s);

// Digest of a run's input into hdr->input_digest: an order-free sum over the
// packed words (the bases), the n_seqs + 1 string offsets (the boundaries,
// which decide the sentinels and where edges stop) and, with N splitting,
// the nmask_words words of the N mask (nmask null without it), each term
// mixed with its index and its kind, so that the same input always gives the
// same value and a change to any of the three changes it.
int launch_digest(DevHeader* hdr_dev, const uint32_t* packed, uint64_t words, const uint64_t* offsets,
                  uint64_t n_seqs, const uint32_t* nmask, uint64_t nmask_words, cudaStream_t s);

// One bounded wait on *word (which the caller leaves 0): *status = 1 when it
// gives up, 2 if it saw the word set.
int launch_bounded_wait(unsigned long long* word, unsigned int* status, cudaStream_t s);

// Process-wide count of kernels launched by the library.
void count_launches(int n);
unsigned long long launches_so_far();

}  // namespace twopaco
