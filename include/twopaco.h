/*
 * twopaco.h -- C ABI of the GB300 junction-detection library.
 *
 * The library finds J(S, k): every position of every input string whose
 * k-mer is a junction of the de Bruijn graph G(S, k) -- a bifurcation (more
 * than one distinct incoming or outgoing edge) or a sentinel (the first or
 * last k-mer of an input string) (Minkin, Pham & Medvedev, "TwoPaCo",
 * arXiv 1602.05856, section "Preliminaries"). By default the graph is the
 * comprehensive graph G(s) U G(s-bar) over both strands, with k-mers stored
 * in normalized form (paragraph after Algorithm 2). Junction positions
 * determine the compacted graph (Observation 1, section "Reduction to the
 * Problem of Finding Junction Positions").
 *
 * The work follows Algorithm 3 (TwoPaCo): the k-mers are split into
 * `rounds` classes (section "Multiple Rounds"), and every round runs
 * Algorithm 2 (Filter-Junctions-Two-Pass): Algorithm 1 (Filter-Junctions)
 * once with a Bloom filter of `filter_bits` bits, then once with an exact
 * hash table on the surviving candidates. Every step runs in CUDA kernels
 * on the current device; nothing falls back to the CPU.
 *
 * Conventions for every entry point:
 *   - Input bytes are A, C, G, T in either case; any other byte is an error
 *     (TWOPACO_EBADBASE). Strings are never joined: no k-mer spans two strings.
 *   - With options->split_at_n, N (either case) is also accepted and ends its
 *     string there: the paper does not say how N is handled, and this library
 *     reads it as splitting the string, so that the maximal N-free pieces are
 *     the strings of the definition -- no k-mer, edge or junction contains an
 *     N, and the first and last k-mers of every piece are sentinels. Positions
 *     stay 0-based offsets into the input string.
 *   - Positions are 0-based k-mer starts i in [0, |s| - k]; a string shorter
 *     than k has none.
 *   - Return value: TWOPACO_OK (0) or a negative TWOPACO_E* code.
 *   - k in [1, 127] (k-mers of up to 31 bases are held in one 64-bit word,
 *     up to 63 in two, up to 127 in four); filter_bits a power of two in
 *     [256, 2^40]; rounds >= 1; n_seqs < 2^32; total_bases < 2^48;
 *     options->hashes in [1, 8]; options->partition_bins a power of two
 *     >= rounds (and >= 2 when rounds > 1); options->both_strands and
 *     options->split_at_n, options->partial and options->per_string_launches 0 or 1;
 *     options->bucket_inserts 0, 1 or 2; options->launch_blocks_per_sm 0..32;
 *     options->ordered_first_pass 0, 1 or 2; options->wide_layout 0, 1 or 2;
 *     options->run_capacity < 2^32. Anything else is TWOPACO_EINVAL.
 *   - Calls on different workspaces may run concurrently from different host
 *     threads; calls that share a workspace must be serialised by the caller.
 */
#ifndef TWOPACO_H_
#define TWOPACO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TWOPACO_OK 0
#define TWOPACO_EINVAL (-1)    /* an argument is out of range */
#define TWOPACO_EBADBASE (-2)  /* an input byte is not one of ACGTacgt */
#define TWOPACO_ENOMEM (-3)    /* device or pinned-host allocation failed */
#define TWOPACO_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define TWOPACO_ECUDA (-5)     /* a CUDA runtime call failed */
#define TWOPACO_EOVERFLOW (-6) /* the pass-2 table, the output buffer or the piece
                                  boundary list (split_at_n) is too small */
#define TWOPACO_ESCRATCH (-7)  /* the run needs more than the no-alloc scratch buffer holds */

typedef struct twopaco_options {
  int hashes;              /* bits per filter item, 1..8 (paper default 4) */
  int both_strands;        /* 1: comprehensive graph (default); 0: single strand */
  uint32_t partition_bins; /* q of the rounds heuristic, power of two (65536) */
  uint64_t table_slots;    /* pass-2 table reserve in slots (rounded up to a power of two);
                              0 = automatic. A round sizes its table from an estimate of its
                              distinct candidates, within the reserve; pass 2 on ordered
                              records (ordered_first_pass) uses the whole reserve, one part
                              per filter region */
  uint64_t candidate_records; /* pass-2 candidate list size in 8-byte units; 0 =
                                 automatic (half a round's positions). It
                                 holds twice as many candidates when the input has
                                 fewer than 2^31 bases. A round with more candidates
                                 stays correct but slower. */
  void* cuda_stream;       /* cudaStream_t to launch on, borrowed; NULL = default */
  int split_at_n;          /* 1: an N ends its string (see above); 0 (default): N is
                              an invalid byte */
  uint64_t run_capacity;   /* split_at_n only: room for the boundaries of the
                              N-free pieces and N runs (one per string start and
                              one per N/base change inside a string); 0 =
                              automatic (n_seqs + 1 + total_bases / 64, at most
                              2^32 - 1). A device run with more boundaries
                              reports TWOPACO_EOVERFLOW; the host builds count them
                              and raise a smaller capacity to that count. At most
                              2^32 - 1, else TWOPACO_EINVAL. */
  int wide_layout;         /* 0 (default): the workspace layout follows the input
                              size. 1: the layout of inputs of 2^31 bases and more,
                              at any size: 64-bit candidate records and no probe
                              descriptors. 2: as 1, and pass 2 also keeps no table
                              slots (the layout of tables of 2^32 slots and more). Same
                              results; for testing those paths on small inputs. */
  int partial;             /* 1: the partially compacted graph (Discussion section:
                              the second pass of Algorithm 2 is omitted). The output
                              is every position that survives the first pass -- in
                              each round, C_temp of that round's class -- a candidate
                              set that holds every junction plus Bloom-filter false
                              positives, so that the edges between consecutive
                              output positions are non-branching paths, though not
                              all maximal. pass2_marks then counts the output
                              positions. 0 (default): the exact junctions. */
  int per_string_launches; /* 1: every first- and second-pass loop of a device run
                              is launched once per input string (over the tiles of
                              4096 positions that start in it) instead of once over
                              all strings, and pass 2 walks C_temp instead of a
                              candidate list: the same build and output, issued the
                              way a per-genome loop would issue it (a baseline for
                              the batched launch). The call reads the string offsets
                              back and synchronises the stream; twopaco_plan_create
                              refuses it. 0 (default): one launch per loop. */
  int bucket_inserts;      /* first-pass inserts through region buckets: each OR into the
                              filter becomes an 8-byte record in the bucket of its filter
                              region (32 MiB, or a quarter of a smaller filter), and the
                              records are then applied region by region while each region
                              sits in L2 -- a filter beyond L2 otherwise takes its random
                              ORs at DRAM's random-access rate. The workspace holds the
                              buckets (records for a round's positions and a quarter more,
                              at most 2^31); the positions go through in chunks that fill
                              them to about 80%, and a full bucket takes the OR directly.
                              Same results. 0 (default): for filters of more than 64 MiB
                              whose chunks put at least 16 ORs on every 32-byte filter
                              sector on average (sparser, the regions' cold misses cost
                              more than direct ORs); 1: for any filter; 2: never. Needs
                              hashes <= 6 and a filter of at most 2^38 bits (else the ORs
                              are direct). */
  int launch_blocks_per_sm; /* launch shape of the pass kernels (insert, probe, pass-2
                              insert and classify): at most this many resident blocks of
                              256 threads per SM in their grids, 1..32; 0 (default): as
                              many as fit. Same results (every loop strides over its
                              work); a latency-bound kernel can gain from fewer blocks
                              contending for L2. */
  int ordered_first_pass;  /* the first pass of a class-map run (rounds 2..64, k <= 63,
                              hashes <= 6) in filter-region order: every position of a
                              round's class becomes an 8-byte record in the bucket of its
                              k-mer's filter region (at most 32 MiB, which L2 holds); the
                              ORs and then the probes are applied bucket by bucket, and the
                              decisions are gathered back in position order. A filter
                              beyond L2 otherwise takes every OR and probe at DRAM's
                              random-access rate. For k <= 27 (and partial 0) pass 2 runs
                              on the same records: the table reserve (table_slots) is split
                              into one part per filter region, each candidate's edges are
                              inserted while its region is in L2, and a lookup per
                              candidate record decides the junctions -- no candidate list
                              and no table sizing per round; a part that fills up reports
                              TWOPACO_EOVERFLOW (twopaco_build and twopaco_build_ctx grow
                              the reserve and run again). The workspace holds a region byte
                              per position and records for a round's positions and a
                              quarter more (the candidate list shares their room); a round
                              with more positions takes the direct kernels. Same results.
                              0 (default): for filters of 1 GiB (2^33 bits) and more; 1:
                              for any filter; 2: never. Not with per_string_launches. */
} twopaco_options;

/* Counters of one run, in the spirit of Table 4 (marks after each pass). */
typedef struct twopaco_stats {
  uint64_t positions;      /* k-mer positions in the input */
  uint64_t pass1_marks;    /* candidates left after pass 1, summed over rounds */
  uint64_t pass2_marks;    /* junction positions (marks after pass 2) */
  uint64_t table_slots;    /* largest pass-2 table used in any round */
  uint64_t bad_base_index; /* first invalid byte, or UINT64_MAX if none */
  uint32_t overflow;       /* nonzero: the pass-2 table, the output or (split_at_n)
                              the piece boundary list ran out of room; when only the
                              output did, d_out_offsets holds the exact counts and
                              twopaco_run_rounds(..., rounds, rounds, ...) writes the
                              output again into a larger buffer */
  uint32_t timeout;        /* nonzero: a bounded device wait gave up */
  uint32_t ordered_rounds; /* rounds whose first pass ran in filter-region order
                              (options->ordered_first_pass) */
  uint32_t pad;
} twopaco_stats;

/* Result of twopaco_build: library-owned host memory. */
typedef struct twopaco_result {
  uint64_t n_seqs;
  uint64_t* offsets;   /* n_seqs + 1 entries: junctions of string t are      */
  uint64_t* positions; /* positions[offsets[t] .. offsets[t+1]), ascending   */
  twopaco_stats stats;
} twopaco_result;

/* Fill `opt` with the defaults listed in twopaco_options. */
void twopaco_default_options(twopaco_options* opt);

/* Static description of a return code; never NULL. */
const char* twopaco_strerror(int code);

/*
 * Host-to-host build (Algorithm 3 with Algorithm 2 in every round).
 *   seqs[t], lengths[t]  the n_seqs input strings (host memory, borrowed,
 *                        read before the call returns; seqs may be NULL
 *                        when n_seqs == 0)
 *   *out                 receives a result allocated by the library; free
 *                        it with twopaco_result_free. Left NULL on error.
 * Allocates device memory for the input and the workspace, copies the input
 * in, runs, copies the result out and frees everything before returning. If
 * the pass-2 table overflows it is grown and the run repeated; the output
 * buffer starts at every k-mer position up to 2^27 of them (else an eighth)
 * and, if the junctions do not fit, is reallocated at their exact count and
 * written again.
 */
int twopaco_build(const char* const* seqs, const uint64_t* lengths, uint64_t n_seqs, int k,
                  uint64_t filter_bits, int rounds, twopaco_result** out);

/* As twopaco_build, with options (NULL = defaults). */
int twopaco_build_ex(const char* const* seqs, const uint64_t* lengths, uint64_t n_seqs, int k,
                     uint64_t filter_bits, int rounds, const twopaco_options* opt,
                     twopaco_result** out);

/*
 * Diagnostic (no counterpart in the paper): launches one bounded device wait
 * of the kind the emit uses on a flag that nothing sets, on `cuda_stream`
 * (NULL = default), and synchronises. The wait gives up after its poll limit
 * (a fraction of a second) instead of hanging, so the call returns
 * TWOPACO_ETIMEOUT and the context stays usable; TWOPACO_ECUDA on a CUDA
 * error. Allocates 16 bytes of device memory for the flag and the status.
 */
int twopaco_selftest_bounded_wait(void* cuda_stream);

/* Release a result returned by twopaco_build*. NULL is ignored. */
void twopaco_result_free(twopaco_result* res);

/*
 * Device workspace size, in bytes, for a device-resident run of
 * `total_bases` bases in `n_seqs` strings. The workspace holds the 2-bit
 * packed input, the filter (filter_bits / 8 bytes), two position bitmaps,
 * the pass-2 table reserved for the worst case, the candidate list and the
 * slots it found, one 8-byte probe descriptor per base (under 2^31 bases,
 * hashes <= 6), the piece boundaries with split_at_n, and small counters.
 */
int twopaco_workspace_size(uint64_t total_bases, uint64_t n_seqs, int k, uint64_t filter_bits,
                           int rounds, const twopaco_options* opt, uint64_t* bytes);

/*
 * Device-resident run; all pointers are device memory owned by the caller.
 *   d_bases      total_bases bytes: the strings back to back
 *   d_offsets    n_seqs + 1 uint64: string t is d_bases[d_offsets[t] .. d_offsets[t+1]),
 *                d_offsets[0] == 0 and d_offsets[n_seqs] == total_bases
 *   d_workspace  at least twopaco_workspace_size(...) bytes, 256-byte aligned
 *   d_out_offsets    n_seqs + 1 uint64, written (as in twopaco_result)
 *   d_out_positions  out_capacity uint64, written; out_capacity >= the number
 *                    of k-mer positions can never overflow
 * Launches every kernel on options->cuda_stream and returns without
 * synchronising. Device-side failures (a bad byte, a full table or output,
 * a wait that gave up) are recorded in the workspace: read them with
 * twopaco_read_stats once the stream has reached this point. Host-side
 * argument errors are returned directly and launch nothing.
 */
int twopaco_run_device(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                       uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                       const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                       uint64_t* d_out_offsets, uint64_t* d_out_positions, uint64_t out_capacity);

/*
 * twopaco_run_device with the input bytes in host memory: they are streamed to
 * the device in chunks (section "Parallelization Scheme": a reader hands the
 * input over in pieces, so only a constant amount of it is resident), each
 * chunk copied into one half of a caller-owned device staging buffer on an
 * internal stream while the chunk before it is packed on options->cuda_stream;
 * then the run goes on as twopaco_run_device does from the packed input.
 *   h_bases        total_bases bytes in host memory, read until the stream has
 *                  passed the pack; page-locked memory lets the copies overlap
 *                  the packing (pageable memory works, without overlap)
 *   d_offsets      n_seqs + 1 uint64 in device memory, as for twopaco_run_device
 *   d_staging      staging_bytes of device memory, 256-byte aligned, owned by
 *                  the caller; each half (staging_bytes / 2 rounded down to a
 *                  multiple of 256) must be at least 64 KiB, else TWOPACO_EINVAL
 * The other arguments, the workspace (twopaco_workspace_size: the ASCII input
 * needs no room in it) and the results are those of twopaco_run_device.
 * Launches without synchronising.
 */
int twopaco_run_streamed(const uint8_t* h_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                         uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                         const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                         void* d_staging, uint64_t staging_bytes, uint64_t* d_out_offsets,
                         uint64_t* d_out_positions, uint64_t out_capacity);

/*
 * The rounds [round_begin, round_end) of a device-resident run (Algorithm 3
 * runs its rounds one after the other, each adding its junctions to
 * C_final), with the arguments of twopaco_run_device; 0 <= round_begin <
 * round_end <= rounds, or round_begin == round_end == rounds (only write the
 * output of a finished run, e.g. one restored from its last checkpoint),
 * else TWOPACO_EINVAL. round_begin == 0 starts the run
 * (packs the input and, for rounds > 1, cuts the k-mer classes); a later
 * round_begin continues the run the workspace holds -- from an earlier call
 * on the same workspace, or restored by twopaco_checkpoint_load. The call
 * with round_end == rounds also writes the output. twopaco_run_device is
 * twopaco_run_rounds(..., 0, rounds, ...). Launches without synchronising.
 */
int twopaco_run_rounds(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                       uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                       const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                       int round_begin, int round_end, uint64_t* d_out_offsets,
                       uint64_t* d_out_positions, uint64_t out_capacity);

/*
 * A run split over several devices by k-mer class (section "Multiple
 * Rounds": every position belongs to exactly one class, each round of
 * Algorithm 3 decides only the positions of its class, and C_final is the
 * union of the rounds' C'_i, which are disjoint). Shard `shard` of `n_shards`
 * (one per device, each with its own copy of the input and its own workspace)
 * runs the rounds r with r % n_shards == shard over the whole input; the
 * shards' C_final bitmaps are then merged -- a bitwise OR, which for these
 * disjoint bitmaps equals an integer sum of their 32-bit words, so one
 * all-reduce of the words does it -- and one of them writes the output.
 *
 * twopaco_shard_begin: pack the input into the workspace and clear C_final;
 *   with compute_cut = 1 (and rounds > 1) also count the partition bins and
 *   cut the classes (one shard, the leader, does this; the cut must be the
 *   same on every shard, and two separate cuts of one input may differ).
 *   compute_cut is 0 or 1, else TWOPACO_EINVAL. Launches without
 *   synchronising; no output arguments.
 *
 * twopaco_shard_rounds: after twopaco_shard_begin on this workspace, run the
 *   rounds shard, shard + n_shards, ... (< rounds), adding their junctions to
 *   the workspace's C_final. d_class_cut: device memory holding the rounds + 1
 *   uint32 class boundaries to use (the leader's, as read with
 *   twopaco_state_device / twopaco_read_state), copied into the workspace on
 *   options->cuda_stream before the first round; NULL keeps the cut the
 *   workspace holds (the leader's own, or none needed when rounds == 1).
 *   0 <= shard < n_shards, else TWOPACO_EINVAL. The counters of a shard
 *   cover its own rounds; positions counts every k-mer position. Launches
 *   without synchronising.
 *
 * After the merge into a workspace's C_final, twopaco_run_rounds(...,
 * rounds, rounds, ...) on that workspace writes the output.
 */
int twopaco_shard_begin(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                        uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                        const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                        int compute_cut);
int twopaco_shard_rounds(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                         uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                         const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                         int shard, int n_shards, const uint32_t* d_class_cut);

/*
 * Device address and size in bytes of one piece of a workspace's state
 * (which: TWOPACO_STATE_*, laid out as twopaco_read_state describes), for a
 * run with these parameters, so that a collective can read or write it in
 * place: C_final for the merge of shards, the class cut for its broadcast.
 * Host arithmetic only: no synchronisation, nothing launched. BINS of a
 * one-round run is NULL with size 0.
 */
int twopaco_state_device(uint64_t total_bases, uint64_t n_seqs, int k, uint64_t filter_bits, int rounds,
                         const twopaco_options* opt, void* d_workspace, int which, void** d_ptr,
                         uint64_t* bytes);

/*
 * Checkpoints between rounds (the paper has no counterpart; for runs long
 * enough that a failure should not restart every round). A checkpoint
 * holds what the finished rounds left: C_final (one bit per base), the class
 * cut and partition counters, the Table-4 counters, the run's parameters and
 * a digest of the packed input; host memory, owned by the caller, a plain
 * byte string that may be written to a file.
 *
 * twopaco_checkpoint_bytes: the size of a checkpoint of such a run.
 *
 * twopaco_checkpoint_save: after twopaco_run_rounds(..., round_end = r, ...)
 *   with 1 <= r <= rounds, copy the workspace's state into host_dst (bytes >=
 *   twopaco_checkpoint_bytes) with next_round = r; synchronises cuda_stream.
 *   The run's d_offsets must still hold the string offsets (they are part of
 *   the input digest). Returns the run's failure (TWOPACO_EBADBASE /
 *   EOVERFLOW / ETIMEOUT) instead of saving a failed state.
 *
 * twopaco_checkpoint_load: restore a checkpoint into a workspace (which may
 *   be a fresh one in another process), given the same input and
 *   parameters as the run it was taken from: the input is packed again and
 *   its digest compared. The digest covers the 2-bit packed bases, the
 *   n_seqs + 1 string offsets (so moved string boundaries differ) and, with
 *   split_at_n, the N mask (so a G changed to N or back differs: the packed
 *   code of N is G's). A checkpoint of another input, parameter set or
 *   format, or one whose head or payload changed after it was saved (each
 *   carries a checksum of its whole head -- next_round, counters, digest --
 *   and payload), is TWOPACO_EINVAL; nothing is launched before its head and
 *   payload check out. Synchronises options->cuda_stream; *next_round gets
 *   the round to continue with (twopaco_run_rounds(..., *next_round, rounds, ...)).
 */
int twopaco_checkpoint_bytes(uint64_t total_bases, uint64_t n_seqs, int k, uint64_t filter_bits,
                             int rounds, const twopaco_options* opt, uint64_t* bytes);
int twopaco_checkpoint_save(void* d_workspace, int next_round, void* host_dst, uint64_t bytes,
                            void* cuda_stream);
int twopaco_checkpoint_load(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                            uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                            const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                            const void* host_src, uint64_t bytes, int* next_round);

/*
 * A device-resident run captured as a CUDA graph. twopaco_plan_create takes
 * the arguments of twopaco_run_device (options->cuda_stream is ignored),
 * records that run's whole launch sequence -- pack, every round's two
 * passes, emit -- into a graph without executing it, and instantiates it.
 * twopaco_plan_launch replays it on cuda_stream with one launch; every
 * replay is a complete run on the same buffers, so the caller may rewrite the
 * input in place between replays (same sizes). Read the outcome with
 * twopaco_read_stats as after twopaco_run_device. Kernels launched by a
 * replay are counted by twopaco_kernel_launches; when profiling is enabled at
 * creation, every replay re-records the per-kernel events.
 */
typedef struct twopaco_plan twopaco_plan;
int twopaco_plan_create(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                        uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                        const twopaco_options* opt, void* d_workspace, uint64_t workspace_bytes,
                        uint64_t* d_out_offsets, uint64_t* d_out_positions, uint64_t out_capacity,
                        twopaco_plan** plan);
int twopaco_plan_launch(twopaco_plan* plan, void* cuda_stream);
void twopaco_plan_destroy(twopaco_plan* plan);

/*
 * Copy the counters of the last run on this workspace into *stats,
 * synchronising `cuda_stream` (NULL = default stream) first. Returns
 * TWOPACO_EBADBASE / TWOPACO_EOVERFLOW / TWOPACO_ETIMEOUT when the run
 * recorded that failure (stats is still filled), else TWOPACO_OK.
 */
int twopaco_read_stats(const void* d_workspace, void* cuda_stream, twopaco_stats* stats);

/*
 * One edge of the compacted de Bruijn graph: two consecutive junction
 * positions p < q of one string (section "Reduction to the Problem of Finding
 * Junction Positions"; Observation 1 makes these exactly the maximal
 * non-branching paths). The edge spells s[p .. q + k - 1]. With split_at_n,
 * p and q lie in one N-free piece (no edge crosses an N).
 */
typedef struct twopaco_edge {
  uint64_t from_hi, from_lo; /* normalized k-mer at p (value hi * 2^64 + lo, first base most
                                significant); for k > 63 its 128 least significant bits,
                                i.e. its last 64 bases */
  uint64_t to_hi, to_lo;     /* normalized k-mer at q */
  uint64_t start;            /* p, within its string */
  uint64_t length;           /* q - p */
  uint32_t from_rc, to_rc;   /* 1: the string reads the reverse complement of the stored k-mer */
} twopaco_edge;

/*
 * Edges of the last run on a workspace, computed on the device.
 *   d_workspace      the workspace of a finished twopaco_run_device call (it
 *                    still holds that run's packed input)
 *   d_offsets, n_seqs, d_out_offsets, d_out_positions   that call's input
 *                    offsets and output
 *   d_edge_offsets   n_seqs + 1 uint64, written: the edges of string t are
 *                    d_edges[d_edge_offsets[t] .. d_edge_offsets[t+1]), in
 *                    position order
 *   d_edges, edge_capacity   room for the edges (at most one per junction)
 * Launches on cuda_stream without synchronising; more edges than
 * edge_capacity set the overflow flag (twopaco_read_stats).
 */
int twopaco_edges_device(const void* d_workspace, const uint64_t* d_offsets, uint64_t n_seqs,
                         const uint64_t* d_out_offsets, const uint64_t* d_out_positions,
                         uint64_t* d_edge_offsets, twopaco_edge* d_edges, uint64_t edge_capacity,
                         void* cuda_stream);

/* Edges returned by twopaco_edges_ctx (borrowed from the context). */
typedef struct twopaco_edge_list {
  uint64_t n_seqs;
  uint64_t* offsets;   /* n_seqs + 1 entries */
  twopaco_edge* edges; /* offsets[n_seqs] edges */
} twopaco_edge_list;

/*
 * Reusable build context. It keeps device buffers (input, workspace, output)
 * and pinned host buffers for the result across calls, growing them only
 * when an input needs more, so repeated builds do no allocation. One context
 * serves one host thread at a time; it launches on its own CUDA stream on
 * the device that was current when it was created.
 */
typedef struct twopaco_context twopaco_context;

/* Create a context on the current device. *ctx is NULL on error. */
int twopaco_context_create(twopaco_context** ctx);

/* Release a context and every buffer it holds. NULL is ignored. */
void twopaco_context_destroy(twopaco_context* ctx);

/*
 * As twopaco_build_ex, through a context: host strings in (pageable or
 * pinned), result in *out. out->offsets and out->positions point into the
 * context's pinned buffers and stay valid until the next call on this
 * context or its destruction; do not pass *out to twopaco_result_free.
 * options->cuda_stream is ignored (the context's own stream is used).
 */
int twopaco_build_ctx(twopaco_context* ctx, const char* const* seqs, const uint64_t* lengths,
                      uint64_t n_seqs, int k, uint64_t filter_bits, int rounds,
                      const twopaco_options* opt, twopaco_result* out);

/*
 * Device-resident run that allocates nothing. The paper has no counterpart:
 * this is an interface for callers that are not allowed to allocate device
 * memory -- code running inside a host framework whose pool owns all device
 * memory (a raw cudaMalloc there is forbidden or fragments the pool), or
 * latency-critical callers that cannot afford cudaMalloc's device-wide
 * synchronisation. Instead of a caller workspace it uses one scratch buffer of
 * TWOPACO_NOALLOC_SCRATCH_BYTES (32 MiB) in static device memory, which every
 * GPU that loads the library holds until the process exits.
 *   Arguments and results are those of twopaco_run_device without the
 *   workspace: the caller still passes the input (d_bases, d_offsets) and the
 *   output (d_out_offsets, d_out_positions) in device memory. The call waits
 *   for the run to finish on options->cuda_stream and fills *stats (may be
 *   NULL), returning TWOPACO_EBADBASE / TWOPACO_EOVERFLOW / TWOPACO_ETIMEOUT as
 *   twopaco_read_stats does.
 *   A run whose workspace (twopaco_workspace_size) exceeds the buffer is
 *   rejected with TWOPACO_ESCRATCH before anything is launched; a small
 *   options->table_slots and candidate_records shrink the workspace.
 *   The first call on a device looks up the buffer's device address on that
 *   device; make that first call before any stream capture.
 *   Every call on a device shares the one buffer and the run clears what it
 *   needs; calls whose work overlaps on the GPU (other host threads, other
 *   streams) race on it and must be serialised by the caller.
 */
#define TWOPACO_NOALLOC_SCRATCH_BYTES (32ull << 20)
int twopaco_run_device_noalloc(const uint8_t* d_bases, const uint64_t* d_offsets, uint64_t n_seqs,
                               uint64_t total_bases, int k, uint64_t filter_bits, int rounds,
                               const twopaco_options* opt, uint64_t* d_out_offsets,
                               uint64_t* d_out_positions, uint64_t out_capacity,
                               twopaco_stats* stats);

/*
 * Edges of the last twopaco_build_ctx on this context. out->offsets and
 * out->edges point into the context's pinned buffers, valid until the next
 * call on the context.
 */
int twopaco_edges_ctx(twopaco_context* ctx, twopaco_edge_list* out);

/* Which internal state twopaco_read_state copies out. */
#define TWOPACO_STATE_CANDIDATES 0 /* C_temp of the last round: ceil(total_bases/32) uint32 words */
#define TWOPACO_STATE_JUNCTIONS 1  /* C_final: ceil(total_bases/32) uint32 words */
#define TWOPACO_STATE_BINS 2       /* partition counters e_i (rounds > 1): q uint32 */
#define TWOPACO_STATE_CUTS 3       /* class boundaries: rounds + 1 uint32 */

/*
 * Copy internal state of the last run on this workspace to host memory, for
 * verification. Bitmaps hold one bit per input base (bit g % 32 of word
 * g / 32 is the k-mer starting at global base g). Class r of Algorithm 3
 * owns the partition bins [cuts[r], cuts[r+1]) (section "Multiple Rounds").
 * Synchronises `cuda_stream` first. `bytes` may not exceed the state's size.
 */
int twopaco_read_state(const void* d_workspace, int which, void* host_dst, uint64_t bytes,
                       void* cuda_stream);

/* Kernels launched by this library in this process so far (monotonic). */
unsigned long long twopaco_kernel_launches(void);

/*
 * Per-kernel timing (off by default). While enabled, every kernel launch of
 * the library is bracketed by two CUDA events recorded on its launch stream.
 * twopaco_profile_enable(on) discards what was collected and switches the
 * recording on or off (returns 0).
 * twopaco_profile_kernels waits for the recorded events and fills, for each
 * distinct kernel (in first-launch order, at most `capacity` of them), its
 * name (static string), launch count and summed device time in ms. Any
 * output pointer may be NULL. Returns the number of distinct kernels, or
 * TWOPACO_ECUDA.
 */
int twopaco_profile_enable(int on);
int twopaco_profile_kernels(const char** names, unsigned long long* launches, double* total_ms,
                            int capacity);

#ifdef __cplusplus
}
#endif

#endif /* TWOPACO_H_ */
