/*
 * dnasa.h -- C ABI of the GB300 suffix-array DNA reconstruction library
 * (libdnasa.so).  Method: arxiv 1404.3456, "A Way For Accelerating The DNA
 * Sequence Reconstruction Problem By CUDA".
 *
 * The library reconstructs a DNA sequence from shotgun fragments (Sec. III)
 * through a suffix array over the fragments (Sec. IV), built on the GPU by
 * radix sorting (Sec. IV, Algorithm 1 in Sec. V), then answers the
 * prefix/suffix relations between fragments by searching that suffix array
 * (Sec. IV: a binary search tells whether some fragment starts with a given
 * string).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Text.  Fragments over {A,C,G,T} are joined into one byte text T[0..N); each
 *   fragment is followed by one '$'.  A single genome is one fragment.
 *   Fragment r occupies T[toff[r] .. toff[r+1]-1); toff[n_reads] == N.
 * Order.  Every '$' is its own sentinel, smaller than A < C < G < T; two
 *   suffixes that reach a '$' at the same offset order by start position.  No
 *   comparison and no LCP ever crosses a '$'.
 * Packed form.  Bases only ('$' not stored), 2 bits each (A=0 C=1 G=2 T=3),
 *   32 per uint64 word, first base in bits 63..62 of word 0, so an unsigned
 *   word compare is a lexicographic compare.  The bases of fragment r occupy
 *   base coordinates [toff[r] - r, toff[r+1] - 1 - r).  A packed buffer holds
 *   dnasa_packed_words(N) words (two zero padding words at the end).
 * Memory.  Every buffer argument is a DEVICE pointer (for example from
 *   torch.empty(..., device="cuda")) unless its comment says "host".  The
 *   caller owns all inputs and outputs; the library owns only the workspace
 *   inside its context.  A host pointer where a device pointer is required is
 *   rejected with DNASA_INVALID_ARG: there is no CPU fallback.
 * Streams.  Work is enqueued on the caller's stream (a cudaStream_t passed as
 *   void*; NULL = the legacy default stream).  Entry points that return a
 *   size through a host pointer synchronize that stream before returning.
 * Errors.  Every function returns a dnasa_status; the text of the last error
 *   is available from dnasa_last_error().  Device-side waits are bounded: a
 *   wait that gives up yields DNASA_DEVICE_TIMEOUT and leaves the context
 *   usable.
 * Index width.  idx_width is DNASA_I32 (int32 SA) or DNASA_I64 (int64 SA).
 * Threads.  A context (its workspace, counters and error text) serves one
 *   call at a time: calls on one context from several threads must be
 *   serialized by the caller; separate contexts are independent (the server
 *   gives each of its slots its own).  The server calls are thread-safe.
 */
#ifndef DNASA_H
#define DNASA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DNASA_OK = 0,
    DNASA_INVALID_ARG = -1,    /* bad size, null or non-device pointer, bad option */
    DNASA_BAD_ALPHABET = -2,   /* a byte other than A, C, G, T, '$'; or text not '$'-terminated;
                                  or an empty fragment */
    DNASA_OOM = -3,            /* workspace could not be allocated (or exceeds the cap) */
    DNASA_CAPACITY = -4,       /* an output buffer is too small; the size needed is returned */
    DNASA_DEVICE_TIMEOUT = -5, /* a bounded device-side wait gave up */
    DNASA_CUDA_ERROR = -6      /* a CUDA runtime call failed */
} dnasa_status;

enum { DNASA_I32 = 4, DNASA_I64 = 8 };

typedef struct dnasa_ctx dnasa_ctx;

/* Options of the suffix-array build.  Zero in any field selects the default. */
typedef struct {
    int32_t reserved0;         /* must be 0.  The radix digit is fixed at 8 bits: a onesweep
                                  pass keeps one look-back word per digit and tile, so a
                                  wider digit multiplies that traffic and the per-tile scans
                                  while saving at most one pass of the initial sort (for
                                  which the key is already cut to whole bytes) */
    int32_t tile_items;        /* items per onesweep tile: 3840 (default), 2048 or 5120 */
    int64_t finish_threshold;  /* when the suffixes still unsorted after a doubling round
                                  number at most this many, and every unsorted group has at
                                  most 1024 members, the rest is sorted by direct comparison
                                  of packed words; -1 = never; 0 = default (never: on the
                                  repeat-rich genomes measured, the doubling rounds were
                                  faster; the autotuner tries the switch) */
    int32_t max_rounds;        /* safety bound on doubling rounds (default 63) */
    int32_t lookback;          /* look-back loads in flight per digit in a onesweep pass:
                                  8 (default) or 1 */
    int32_t seg_max;           /* largest group a doubling round sorts on chip (8..12288,
                                  default 12288); larger groups go through global radix
                                  passes */
    int32_t pack_position;     /* initial sort: 0 (default) packs the suffix position under
                                  the key and sorts one 64-bit word per suffix when the
                                  key can still hold enough symbols; -1 never packs and
                                  sorts (key, position) pairs */
    int32_t builder;           /* 0 (default): prefix doubling as described at sa_build;
                                  1: the difference-cover (DC3, skew) algorithm of
                                  Kaerkkaeinen and Sanders, after which the paper names its
                                  GPU kernel (Sec. IV) -- sample positions i mod 3 != 0
                                  radix sorted by triples and named, recursion while names
                                  repeat, then the mod-0 positions by (symbol, rank of
                                  i+1) and a merge; same suffix array; one instance only
                                  (sa_build_batched refuses it); the other options are
                                  ignored */
    int32_t rounds_on_host;    /* 0 (default): after round 0 the doubling rounds run as one
                                  captured CUDA graph -- a device-side loop (a WHILE node,
                                  two rounds per pass) whose kernels read their counts from
                                  device memory, so the stream is synchronized after round 0
                                  and at the end only -- whenever profiling is off, the
                                  direct-comparison finisher is off and every group fits
                                  the on-chip sorts (seg_max); rounds outside those
                                  conditions run from the host.  A graph is captured on
                                  the second build with the same buffers and sizes (the
                                  first runs its rounds from the host), and the context
                                  keeps the graphs of its four most recently used
                                  configurations (a caller that alternates output
                                  buffers reuses one per set).  1: every round from the
                                  host, which reads three counters back after each */
} dnasa_opts;

/* One suffix-prefix overlap: the last L bases of fragment j equal the first L
 * bases of fragment k (Sec. III "fir" relation, generalised). */
typedef struct {
    int32_t j, k, L;
} dnasa_edge;

/* An overlap between oriented fragments allowing substitutions: the last L
 * bases of a and the first L bases of b differ in `mismatches` places. */
typedef struct {
    int32_t a, b, L, mismatches;
} dnasa_aedge;

/* Per-round trace of the last sa_build on a context (host-readable). */
typedef struct {
    int32_t rounds;            /* doubling rounds run after the initial sort */
    int32_t finished_direct;   /* 1 if the direct-comparison finisher ran */
    int32_t h0;                /* symbols in the initial packed key */
    int32_t pack_bits;         /* position bits packed under the initial key (0: pairs) */
    int64_t active[64];        /* unsorted suffixes after the initial sort and each round */
    int32_t graph_rounds;      /* rounds of those run inside the captured graph */
    int32_t reserved;
} dnasa_trace;

/* ---- context --------------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  workspace_cap bounds the device
 * workspace in bytes (0 = no bound).  *out receives the context (host). */
int dnasa_create(int device, size_t workspace_cap, dnasa_ctx **out);
void dnasa_destroy(dnasa_ctx *ctx);
/* Text of the last error on this context (never NULL; "" when none). */
const char *dnasa_last_error(dnasa_ctx *ctx);
/* Synchronizes `stream` and returns the status recorded by device code since
 * the last call (DNASA_OK or DNASA_DEVICE_TIMEOUT); clears it. */
int dnasa_sync_status(dnasa_ctx *ctx, void *stream);
/* Trace of the last sa_build (host struct, copied out). */
int dnasa_get_trace(dnasa_ctx *ctx, dnasa_trace *out);
/* Words a packed buffer for an N-symbol text needs (bases / 32 rounded up, + 2). */
int64_t dnasa_packed_words(int64_t N);

/* ---- profiling ---------------------------------------------------------------- */

/* Kernel classes the profiler aggregates. */
enum {
    DNASA_PROF_ONESWEEP = 0,  /* one radix digit pass (decoupled look-back scatter) */
    DNASA_PROF_HIST = 1,      /* digit histograms of a sort */
    DNASA_PROF_RERANK = 2,    /* head flags, SA writes, staged ranks, compaction */
    DNASA_PROF_GATHER = 3,    /* doubling keys (rank[i], rank[i+h]) */
    DNASA_PROF_INIT = 4,      /* initial packed keys */
    DNASA_PROF_FINISH = 5,    /* direct-comparison finisher */
    DNASA_PROF_LCP = 6,
    DNASA_PROF_OVERLAP = 7,
    DNASA_PROF_LAYOUT = 8,
    DNASA_PROF_PACK = 9,
    DNASA_PROF_OTHER = 10,
    DNASA_PROF_SEGSORT = 11,  /* in-group sorting of a doubling round */
    DNASA_PROF_APPLY = 12,    /* staged rank writes applied bucket by bucket */
    DNASA_PROF_KINDS = 13
};

/* Per kernel class: launches, summed device time (CUDA events recorded on the
 * launching stream around each launch) and summed algorithmic bytes (what the
 * kernel must read and write, a random 4-byte access counted as 4 bytes). */
typedef struct {
    int32_t kind;
    int32_t launches;
    double ms;
    double bytes;
} dnasa_prof_entry;

/* Turns per-launch event recording on (enable != 0) or off; clears records. */
int dnasa_profile(dnasa_ctx *ctx, int enable);
/* Waits for the recorded events, writes one entry per kernel class that ran
 * (at most max_entries; host array) and clears the records. */
int dnasa_profile_read(dnasa_ctx *ctx, dnasa_prof_entry *out, int max_entries, int *n_out);
/* Kernel launches issued through this context since it was created. */
uint64_t dnasa_launch_count(dnasa_ctx *ctx);

/* ---- radix sort utility (Sec. IV radix sort; Algorithm 1 semantics) ---------- */

/* Stable LSD radix sort of n (key, value) pairs by key bits [0, key_bits), with
 * the same onesweep kernels the suffix-array build runs on.  Equal keys keep
 * their input order, as the 1-bit split passes of Algorithm 1 do.
 *   keys        device uint64[n], sorted in place
 *   vals        device uint32[n] permuted with the keys, or NULL (keys only)
 *   key_bits    1..64; tile_items and lookback as in dnasa_opts (0 = default)
 * Enqueues only.  n < 2^32. */
int dnasa_sort_pairs(dnasa_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t n, int key_bits,
                     int tile_items, int lookback, void *stream);

/* Failure-path self-test (no counterpart in the paper): runs one digit pass in
 * which the only tile waits on a predecessor that never publishes its counts.
 * The wait is bounded; the pass writes nothing and the call returns
 * DNASA_DEVICE_TIMEOUT, after which the context works normally.  Hangs and
 * faults nothing.  Synchronizes the stream. */
int dnasa_selftest_timeout(dnasa_ctx *ctx, void *stream);

/* ---- allocation-free radix sort ------------------------------------------------ */

/* Largest n dnasa_sort_pairs_noalloc accepts. */
#define DNASA_NOALLOC_MAX_ITEMS (1 << 20)

/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory -- code running under a host framework whose
 * caching allocator already holds the GPU's memory, or latency-bound loops in
 * which a cudaMalloc/cudaFree (and the device synchronization it implies) is not
 * acceptable.  It sorts like dnasa_sort_pairs (same kernels, same stable order)
 * but needs no context and allocates nothing: its scratch is one fixed device
 * array of about 12.6 MB inside the library, which every device that loads the
 * library keeps until the process exits.
 *   keys, vals, key_bits   as for dnasa_sort_pairs (vals may be NULL)
 *   n                      0 <= n <= DNASA_NOALLOC_MAX_ITEMS, else DNASA_CAPACITY
 * The first call on a device looks up the scratch array's device address (with
 * that device current); make that first call before any stream capture.  All
 * calls share the one scratch array, so calls whose work overlaps on the GPU
 * (for example on two streams at once) race; serialize them.  Synchronizes the
 * stream before returning; DNASA_DEVICE_TIMEOUT if a bounded device wait gave up. */
int dnasa_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, void *stream);

/* ---- pack (Sec. III alphabet; the SA of Sec. IV is over this text) ------- */

/* Validates text[0..N) and writes its packed form and fragment offsets.
 *   text      device, N bytes of A/C/G/T/'$', last byte '$', no empty fragment
 *   packed    device, dnasa_packed_words(N) uint64 words (written entirely)
 *   toff      device, toff_cap int64 entries; receives n_reads + 1 offsets
 *   n_reads   host out: number of fragments (= number of '$')
 * Synchronizes the stream.  DNASA_BAD_ALPHABET on a bad byte or empty
 * fragment; DNASA_CAPACITY when toff_cap < n_reads + 1 (*n_reads still set). */
int dnasa_pack(dnasa_ctx *ctx, const uint8_t *text, int64_t N, uint64_t *packed,
               int64_t *toff, int64_t toff_cap, int64_t *n_reads, void *stream);

/* ---- suffix array (Sec. IV: all suffixes in sorted order, the array Pos) -- */

/* Builds the suffix array of the packed text by prefix doubling: a radix sort of
 * packed initial keys (the first h0 <= 29 bases and the distance to the
 * fragment's '$'), then rounds that order each group of suffixes still equal on
 * their first h symbols by rank[i+h], with an optional direct-comparison
 * finisher.
 *   packed, toff   as written by dnasa_pack (toff: n_reads + 1 entries)
 *   N              text length including every '$' (N >= 1, N < 2^31)
 *   sa             device, N entries of int32 or int64 (idx_width): sa[j] is
 *                  the text position of the j-th smallest suffix
 *   opts           host, may be NULL (defaults)
 * Enqueues on the stream; synchronizes it after round 0 and at the end when the
 * doubling rounds run as a graph (rounds_on_host), else once per round. */
int sa_build(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
             int64_t N, void *sa, int idx_width, const dnasa_opts *opts, void *stream);

/* The suffix array and its LCP array (as lcp_build defines it) in one call: the
 * same SA as sa_build and the same LCP as lcp_build, bit for bit.  Round 0 of the
 * build compares each SA slot's initial key with its predecessor's anyway; for
 * every pair the initial keys separate (all but the pairs sharing their first h0
 * bases) it writes the LCP from the two keys -- the equal leading bases of their
 * packed h0-mers, capped by the bases each has before its '$', 0 across instances
 * -- so that only the remaining pairs are compared on the text afterwards,
 * starting at base h0: their lower suffixes are marked in a bitmap of text
 * positions and walked in text order through the build's final ranks (the
 * inverse SA), each comparison starting where the previous position's ended
 * (Kasai's bound) -- no sort by position.  Arguments as sa_build, plus
 *   lcp   device, N int32 (written entirely)
 * With builder = 1 (DC3) it is sa_build followed by lcp_build.  Synchronizes the
 * stream as sa_build does. */
int sa_lcp_build(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                 int64_t N, void *sa, int idx_width, int32_t *lcp, const dnasa_opts *opts, void *stream);

/* ---- LCP ----------------------------------------------------------------- */

/* lcp[0] = 0; lcp[j] = number of equal bases at the start of suffixes sa[j-1]
 * and sa[j], stopping at the first '$' of either (a '$' never matches).
 *   lcp  device, N int32.  Synchronizes the stream once (to size the pass over
 *   pairs longer than 64 bases, which walks runs of consecutive text positions
 *   and starts each comparison from the previous LCP minus one, after Kasai). */
int lcp_build(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
              int64_t N, const void *sa, int idx_width, int32_t *lcp, void *stream);

/* ---- overlap search + containment (Sec. III "fir", Sec. IV search) ----- */

/* For every fragment j and every suffix X of it with min_overlap <= |X| < |r_j|,
 * finds the fragments k != j whose first |X| bases equal X and |X| < |r_k|,
 * keeping for each ordered pair (j, k) the largest such L = |X|.  Edges are
 * written in (j, k) order.  contained[k] = 1 when fragment k occurs inside
 * another fragment (of two identical fragments, the larger index is marked).
 *   sa, lcp     as written by sa_build / lcp_build for the same text
 *   edges       device, cap entries
 *   n_edges     host out: number of edges (also when > cap)
 *   contained   device, n_reads bytes
 * Synchronizes the stream.  DNASA_CAPACITY when the edges exceed cap. */
int overlap_search(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                   int64_t N, const void *sa, const int32_t *lcp, int idx_width,
                   int32_t min_overlap, dnasa_edge *edges, int64_t cap, int64_t *n_edges,
                   uint8_t *contained, void *stream);

/* ---- overlaps on both strands with errors (Sec. III DEFINITION) ------- */

/* The paper's problem allows each fragment to come from either strand and to
 * carry a rate mu of errors.  Read here as substitutions (Hamming distance) with
 * mu = mu_num / mu_den (0 <= mu < 1): oriented fragments are 2r (fragment r) and
 * 2r + 1 (its reverse complement) when both_strands is 1, else r; (a, b, L) is an
 * overlap when a and b are different fragments, min_overlap <= L < |a|, |b|, and
 * the last L bases of a and the first L bases of b differ in at most
 * floor(L * mu_num / mu_den) places.  The largest L per ordered pair is written,
 * in (a, b) order, with its mismatch count.  Every such overlap contains a run
 * of at least L / (e + 1) equal bases (e = allowed mismatches); the runs are
 * found as LCP intervals of the suffix array of the oriented text (Sec. IV) and
 * each candidate alignment is verified on packed words.
 *   text        device, N bytes ('$'-terminated fragments, as for dnasa_pack)
 *   edges       device, cap entries;  n_edges  host out (also when > cap)
 *   n_oriented  host out: oriented fragments (2 * fragments or fragments)
 * Synchronizes the stream.  DNASA_CAPACITY when the edges exceed cap.  Cost:
 * g^2 seed pairs per position shared by g copies of a repeat. */
int overlap_search_approx(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int32_t min_overlap,
                          int32_t mu_num, int32_t mu_den, int32_t both_strands, dnasa_aedge *edges,
                          int64_t cap, int64_t *n_edges, int64_t *n_oriented, void *stream);

/* ---- whole method on one fragment set (Sec. III, Fig. 3 -> superstring) -- */

/* text -> pack -> SA -> LCP -> overlaps -> greedy layout -> contigs.  Greedy:
 * edges between non-contained fragments in order of (L desc, j asc, k asc);
 * (j, k) is accepted when j has no successor, k no predecessor and they lie on
 * different chains.  Each chain head (no predecessor, ascending index) starts
 * a contig: the head, then each successor without its first L bases.
 *   text        device, N bytes (as for dnasa_pack)
 *   contigs     device, cap bytes: the contigs one after another (ASCII ACGT)
 *   contig_off  device, off_cap int64: contig c = contigs[off[c] .. off[c+1])
 *   n_contigs   host out;  needed  host out: bytes the contigs need
 * Synchronizes the stream.  DNASA_CAPACITY when cap or off_cap is too small. */
int assemble(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int32_t min_overlap,
             uint8_t *contigs, int64_t cap, int64_t *contig_off, int64_t off_cap,
             int64_t *n_contigs, int64_t *needed, void *stream);

/* ---- two-cut reconstruction from fir relations (Sec. III, Figs. 2, 5-8) --- */

/* Status of a fir reconstruction. */
enum { DNASA_FIR_SOLVED = 0, DNASA_FIR_NONE = 1, DNASA_FIR_GAVE_UP = 2 };

/* Rebuilds a sequence cut by two shotguns (Sec. III, Fig. 2: the fragments are
 * the pieces of two cuttings of one sequence, shuffled, every break position
 * different) from "fir" relations, by depth-first search with back-tracking:
 * a start pair is a fragment d_i that is a proper prefix of a fragment d_k
 * (tried for k ascending, then i ascending); with remainder X (what is left of
 * the longer fragment past the shorter), the unused fragments in fir relation
 * with X are tried in ascending index -- a fragment c that is a proper prefix of
 * X leaves X past |c|; X a proper prefix of c leaves c past |X|; c equal to X
 * ends the search when it is the last fragment.  A choice that leaves no fir
 * fragment is undone and the next one tried (Figs. 7-8).  The fir relations of
 * every suffix of every fragment come from one pass over the suffix array of
 * the fragment text (Sec. IV: binary search of a suffix among the fragment
 * starts, then the LCP of consecutive fragment starts).
 *   text        device, N bytes: '$'-terminated fragments (as for dnasa_pack)
 *   max_steps   >= 1: placed fragments (a start pair counts as one) after which
 *               the search gives up (DNASA_FIR_GAVE_UP)
 *   frag_start  device, frag_cap int64: offset of each fragment in the result
 *               (-1 for all when not solved)
 *   rs          device, rs_cap bytes: the reconstructed sequence (ASCII ACGT)
 *   rs_len      host out: its length (0 when not solved)
 *   status      host out: DNASA_FIR_SOLVED, _NONE (no reconstruction exists) or
 *               _GAVE_UP;  steps  host out: steps taken
 * Synchronizes the stream.  DNASA_CAPACITY when frag_cap is below the number
 * of fragments or rs_cap below rs_len (*rs_len is set). */
int fir_reconstruct(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int64_t max_steps,
                    int64_t *frag_start, int64_t frag_cap, uint8_t *rs, int64_t rs_cap,
                    int64_t *rs_len, int32_t *status, int64_t *steps, void *stream);

/* fir_reconstruct of n_inst independent fragment texts stored one after another
 * (inst_off: host, n_inst + 1 offsets, each a fragment start), in one pass: one
 * suffix array, one fir-relation pass and one search thread per instance.
 *   frag_start  device int64[frag_cap]: per fragment (global index), offset in
 *               its own instance's result
 *   rs_off      device int64[n_inst + 1]: instance i's result is
 *               rs[rs_off[i] .. rs_off[i+1]) (empty when not solved)
 *   status      device int32[n_inst];  steps  device int64[n_inst]
 *   rs_total    host out: bytes of all results
 * Synchronizes the stream.  DNASA_CAPACITY as for fir_reconstruct. */
int fir_reconstruct_batched(dnasa_ctx *ctx, const uint8_t *texts, const int64_t *inst_off, int32_t n_inst,
                            int64_t max_steps, int64_t *frag_start, int64_t frag_cap, uint8_t *rs,
                            int64_t rs_cap, int64_t *rs_off, int32_t *status, int64_t *steps,
                            int64_t *rs_total, void *stream);

/* ---- batched -- many independent fragment sets in one pass ------------- */

/* Suffix arrays of n_inst independent fragment texts stored one after another
 * (instance i = text[inst_off[i] .. inst_off[i+1]), itself '$'-terminated
 * fragments), built together: every kernel of the build runs once over all
 * instances, with the instance number as the most significant part of the
 * initial key, so that each instance's suffixes land in its own slot range.
 *   packed, toff, n_reads, N   as for sa_build, over the concatenated text
 *   inst_off   host, n_inst + 1 offsets: 0, ..., N, each a fragment start
 *   sa         device int32[N]: sa[inst_off[i] + j] = position, inside instance
 *              i, of instance i's j-th smallest suffix (its own SA, local coords)
 * Synchronizes the stream once per doubling round (as sa_build). */
int sa_build_batched(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                     int64_t N, const int64_t *inst_off, int32_t n_inst, int32_t *sa,
                     const dnasa_opts *opts, void *stream);

/* The whole method (as assemble) on n_inst independent fragment texts at once.
 * No overlap, containment or chain ever joins two instances.  Contigs are
 * written instance by instance; inst_contig_off (device, n_inst + 1 int64, may
 * be NULL) receives the index of each instance's first contig, so instance i
 * owns contigs [inst_contig_off[i], inst_contig_off[i+1]).  Fragment indices
 * inside an instance, and hence its result, are the same as when the instance
 * is assembled alone.  Other arguments as for assemble.  Synchronizes. */
int assemble_batched(dnasa_ctx *ctx, const uint8_t *texts, const int64_t *inst_off, int32_t n_inst,
                     int32_t min_overlap, const dnasa_opts *opts, uint8_t *contigs, int64_t cap,
                     int64_t *contig_off, int64_t off_cap, int64_t *inst_contig_off,
                     int64_t *n_contigs, int64_t *needed, void *stream);

/* Autotuner of the build options: times sa_build (batched when n_inst > 1) on
 * this text for every tile size (2048, 3840, 5120), doubling-to-direct switch
 * (never, N/64, N/8, as soon as every group fits the finisher) and on-chip group
 * limit (256, 2048, 12288), each once; then times the four fastest three more
 * times each and writes the one with the best median to *best (host) and that
 * median to *best_ms (host, may be NULL).  The radix digit is 8 bits: the only
 * width the kernels implement.
 * With cache_path (may be NULL), a line "key<TAB>tile<TAB>switch<TAB>lookback
 * <TAB>seg_max<TAB>ms" keyed by GPU name, bits of N and bits of n_inst is looked up first
 * and appended after tuning.  inst_off as for sa_build_batched (host).
 * Synchronizes the stream. */
int dnasa_autotune(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                   int64_t N, const int64_t *inst_off, int32_t n_inst, const char *cache_path,
                   dnasa_opts *best, double *best_ms, void *stream);

/* ---- served -- continuous batching of arriving assembly jobs ------------ */

/* One assembly job: a '$'-terminated fragment text in HOST memory (copied at
 * submit, so the caller may free it afterwards). */
typedef struct {
    const uint8_t *text;
    int64_t N;
    int32_t min_overlap;
    int32_t reserved;
} dnasa_job;

/* A finished job.  contigs / contig_off point into server-owned host memory that
 * stays valid until the next dnasa_server_poll or dnasa_server_destroy: contig c
 * is contigs[contig_off[c] .. contig_off[c+1]).  Times are milliseconds since
 * the server was created: submitted, batch started on a slot, result ready. */
typedef struct {
    uint64_t id;
    int32_t status;            /* dnasa_status of the job's batch */
    int32_t reserved;
    int64_t n_contigs;
    int64_t bytes;
    const uint8_t *contigs;
    const int64_t *contig_off;
    double t_submit_ms, t_start_ms, t_done_ms;
} dnasa_result;

typedef struct dnasa_server dnasa_server;

/* Starts a server on `device` with `slots` workers (own context and stream each,
 * 1..16) that admit queued jobs, in arrival order, as batches of at most
 * max_batch jobs of equal min_overlap, while their estimated device memory
 * (dnasa_server_job_bytes each) fits in the budget less what the batches already
 * running reserved.  The budget is hbm_budget (0 = 90 % of the free memory at
 * creation), lowered at each admission to 95 % of the device memory free at that
 * moment plus what the running batches reserved and the admitting slot holds, so
 * that memory taken by other users after creation is respected.  A job larger
 * than the whole budget runs alone once nothing else runs.  Batches of different
 * slots overlap on the GPU.  Each result equals that job assembled alone. */
int dnasa_server_create(int device, size_t hbm_budget, int32_t slots, int32_t max_batch,
                        dnasa_server **out);
/* Queues a job (thread-safe; returns at once after checking the text on the
 * host: DNASA_BAD_ALPHABET for a byte outside A/C/G/T/'$', an empty fragment or
 * a missing final '$', so that a malformed job never enters a batch).  A batch
 * that fails as a whole is run again job by job, so that each job's status is
 * its own. */
int dnasa_server_submit(dnasa_server *srv, const dnasa_job *job, uint64_t id);
/* Moves up to max_results finished jobs into out (host array), waiting up to
 * wait_ms for the first one; *n_out = how many were written. */
int dnasa_server_poll(dnasa_server *srv, dnasa_result *out, int32_t max_results, int32_t wait_ms,
                      int32_t *n_out);
/* Device bytes the server reserves for one job of N text symbols holding n_reads
 * fragments: the suffix-array workspace (~95 bytes per symbol, held with the
 * context's growth margin), the buffers assemble keeps alongside it, the slot's
 * text and contig buffers, and a fixed 32 MB.  -1 for sizes out of range. */
int64_t dnasa_server_job_bytes(int64_t N, int64_t n_reads);
/* Jobs queued or running. */
int dnasa_server_pending(dnasa_server *srv);
/* Finishes every queued job, then stops the workers and frees everything. */
void dnasa_server_destroy(dnasa_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* DNASA_H */
