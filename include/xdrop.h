/*
 * xdrop.h: C ABI of the GB300 X-drop seed-and-extend library (libxdrop.so).
 *
 * The operation.  For each read pair (A, B) that shares an exact seed of
 * seed_len bases at A[seed_a..] and B[seed_b..], the library runs two
 * X-drop extensions (seed-and-extend, Section "Related works", BELLA
 * paragraph) and returns, for each, the best score and where it was
 * reached.  The extension is the anti-diagonal X-drop dynamic program that
 * the paper's GPU schedulers feed (Section "Related works", LOGAN
 * paragraph: cells of one anti-diagonal are independent; Section
 * "Comparison between small dataset and large dataset": Needleman-Wunsch /
 * Smith-Waterman with X-drop).  The paper prints no recurrence; this
 * library computes the following reading exactly (bit-exact; int32 cells,
 * or 16-bit cells in a normalised frame for scorings that fit them, with
 * identical results):
 *
 *   Extension over a[1..m], b[1..n] (right: the bases after the seed;
 *   left: the bases before it, read backwards from the seed).  H(0,0) = 0;
 *   R(i,j) = max(H(i-1,j-1) + s(a_i,b_j), H(i-1,j) + gap, H(i,j-1) + gap)
 *   over predecessors that exist and are live, s = match or mismatch.  With
 *   T_d the best score on anti-diagonals 0..d (T_0 = 0), a cell on diagonal
 *   d = i+j is live iff R >= T_{d-1} - x; otherwise it is pruned.  The
 *   extension ends when two consecutive diagonals are entirely pruned or
 *   at d = m+n.  Its result is the final T and the first cell that reached
 *   it (smallest d, then smallest i).  A pair may name the reverse strand
 *   of read b (XDROP_PAIR_RC below).
 *
 * Read layout (inputs).  2-bit codes A=0, C=1, G=2, T=3, 16 bases per
 * uint32 word, base k of the buffer in bits 2(k mod 16)..2(k mod 16)+1 of
 * word k/16.  read_off[r] is the first base of read r and must be a
 * multiple of 16; read_len[r] its length.  Reads must lie inside the packed
 * buffer, which holds fewer than 2^32 bases.
 *
 * Limits (XDROP_EINVAL otherwise): match > 0, mismatch <= 0, gap < 0,
 * 0 <= x < 2^25; every |score| times (read_len[a] + read_len[b]) of a pair
 * below 2^25; read_len < 2^28; seed_a + seed_len <= read_len[a] and
 * seed_b + seed_len <= read_len[b]; read ids < n_reads.
 *
 * Threads.  xdrop_submit* may be called from many threads at once on one
 * context; xdrop_sync may be called from any thread, once per ticket.
 * Error messages are per thread (xdrop_last_error).
 */
#ifndef XDROP_H
#define XDROP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define XDROP_OK 0
#define XDROP_EINVAL (-1)    /* bad argument; nothing was launched          */
#define XDROP_ENOMEM (-2)    /* exceeds the device memory budget even alone */
#define XDROP_ECUDA (-3)     /* a CUDA call failed; see xdrop_last_error    */
#define XDROP_ETIMEDOUT (-4) /* sync timed out; the ticket stays valid      */
#define XDROP_EBUSY (-5)     /* budget taken by work in flight; retry later */

/* xdrop_init flags. */
#define XDROP_MODE_BATCHED 0u /* default: binned persistent launch in a graph */
#define XDROP_MODE_PLAIN 1u   /* one launch of the first band tile per
                                 10,000-pair sub-batch, in pair order (the
                                 forced tile, else packed 4x16)             */
#define XDROP_MODE_SERVE 2u   /* batched, plus continuous batching of
                                 xdrop_submit_pairs requests (serving)       */

/* xdrop_result.status values (per pair). */
#define XDROP_STATUS_OK 0
#define XDROP_STATUS_INVALID 1 /* device submit only: pair failed the limits
                                  (or asks for the reverse strand there)     */
#define XDROP_STATUS_TOO_LONG 2 /* xdrop_align_static: extension longer than its scratch */

typedef struct xdrop_ctx xdrop_ctx;   /* opaque, owned by the library */
typedef uint64_t xdrop_ticket;

typedef struct {
    int32_t match, mismatch, gap, x;
} xdrop_scoring;

/* Reverse strand: set in a pair's b to align read a against the reverse
 * complement of read (b & ~XDROP_PAIR_RC), whose base k is the complement
 * (code 3 - c) of base len_b - 1 - k of the read; seed_b and the result's
 * b coordinates are positions in that reverse complement.  Accepted by
 * xdrop_submit and by xdrop_submit_pairs (resident reads, serving too):
 * the library stores the reverse complements of the reads beside them.
 * xdrop_submit_device, xdrop_count_cells_device and xdrop_align_static
 * give such a pair XDROP_STATUS_INVALID. */
#define XDROP_PAIR_RC 0x80000000u

typedef struct {
    uint32_t a, b;           /* read ids (b may carry XDROP_PAIR_RC) */
    uint32_t seed_a, seed_b; /* 0-based seed start on each read   */
    uint32_t seed_len;       /* seed length in bases              */
} xdrop_pair;                /* 20 bytes, no padding              */

typedef struct {
    int32_t left_score;   /* best score of the left extension           */
    int32_t left_begin_a; /* seed_a - i* of the left extension          */
    int32_t left_begin_b; /* seed_b - j*                                */
    int32_t right_score;  /* best score of the right extension          */
    int32_t right_end_a;  /* seed_a + seed_len + i* (end, exclusive)    */
    int32_t right_end_b;  /* seed_b + seed_len + j*                     */
    int32_t status;       /* XDROP_STATUS_*                             */
} xdrop_result;           /* 28 bytes                                   */

typedef struct {
    double kernel_ms;        /* device time of the last completed ticket's
                                alignment launches (CUDA events)          */
    double main_kernel_ms;   /* batched mode: device time of the first-tier
                                persistent kernel alone, from events
                                recorded inside the graph (the latest
                                replay); 0 in plain mode                  */
    uint64_t tasks;          /* extensions (2 per pair)                   */
    uint64_t overflow_tasks; /* extensions re-run with a wider band tile  */
    uint64_t wide_tasks;     /* extensions that needed the unbounded tier */
    uint32_t launches;       /* kernel launches of that ticket            */
    uint32_t graph_replays;  /* CUDA graph launches of that ticket        */
    uint32_t tile_lanes;     /* first band tier: lanes per extension      */
    uint32_t tile_cells;     /* first band tier: cells per lane, with
                                XDROP_TILE_PACKED16 set for a packed tile */
    uint64_t device_bytes;   /* device memory the context holds now       */
} xdrop_stats;

typedef struct {
    uint64_t requests_done;   /* serving requests completed                  */
    uint64_t wide_passes;     /* requests whose widest-band extensions ran
                                 the 512-slot / unbounded tiers beside the
                                 serving kernel                              */
    uint64_t relaunches;      /* serving kernel launches                     */
    uint64_t max_in_flight;   /* most requests admitted at once              */
    uint64_t admission_waits; /* admissions deferred for lack of memory      */
    uint64_t published;       /* extensions published to the task ring       */
    uint64_t consumed;        /* extensions taken from it                    */
    uint64_t spill_reserved;  /* extensions handed to the second tier        */
    uint64_t spill_taken;     /* of those, taken by second-tier groups       */
    uint64_t ring_warps;      /* warps of the running serving kernel         */
    uint64_t idle_exits;      /* warps that left because no work came within
                                 the idle bound (hang guard), over all
                                 launches of the serving kernel             */
    uint64_t help_sessions;   /* times a warp left the first tier to serve
                                 the second-tier queue (no warp is reserved
                                 for it), over all launches                 */
    uint64_t surplus_counts;  /* extensions counted past their request's
                                 total: an invariant counter that stays 0
                                 (each extension runs exactly once)         */
} xdrop_serve_stats;

/* Create a context on CUDA device `device`.  device_mem_budget bounds the
 * device memory the context holds at once (0: no bound); in serving mode it
 * bounds the buffers of the requests in flight (memory admission; 0: 1 GiB)
 * and the resident reads and scratch are not counted.  flags:
 * XDROP_MODE_*.  On success *out owns a stream, events and buffers; free
 * it with xdrop_free.  Returns XDROP_OK, XDROP_EINVAL or XDROP_ECUDA. */
int xdrop_init(xdrop_ctx **out, int device, size_t device_mem_budget,
               uint32_t flags);

/* Align n_pairs pairs held in HOST memory (any host memory).  The inputs
 * are copied before the call returns; the caller may reuse them at once.
 * `out` (n_pairs results, host memory) belongs to the caller and must stay
 * valid until xdrop_sync(ticket) returns XDROP_OK; it is written during
 * that sync.  All pairs are validated first: any failure returns
 * XDROP_EINVAL and launches nothing.  If any pair asks for the reverse
 * strand (XDROP_PAIR_RC), the reverse complements of the reads are built
 * on the device too (twice the packed size).  n_pairs == 0 is valid (the
 * ticket completes at once).  Returns XDROP_OK and a ticket, or an error. */
int xdrop_submit(xdrop_ctx *c, const uint32_t *packed, const uint64_t *read_off,
                 const uint32_t *read_len, uint32_t n_reads,
                 const xdrop_pair *pairs, size_t n_pairs,
                 const xdrop_scoring *s, xdrop_result *out, xdrop_ticket *t);

/* As xdrop_submit, but every array is DEVICE memory on the context's
 * device and stays owned by the caller; the arrays must stay valid and
 * unchanged until the ticket's sync returns.  n_words is the length of
 * `packed` in words.  Pairs are validated on the device: a pair that
 * fails the limits (or asks for the reverse strand, XDROP_PAIR_RC, which
 * needs the reverse complements only the host-side calls store) gets
 * status XDROP_STATUS_INVALID and zero scores, the others are aligned,
 * and the ticket's sync returns XDROP_EINVAL.  Results are written to
 * `out` (device) by the time sync returns; until then `out` may also hold
 * the library's scratch (autotuning samples its pairs there). */
int xdrop_submit_device(xdrop_ctx *c, const uint32_t *packed, uint64_t n_words,
                        const uint64_t *read_off, const uint32_t *read_len,
                        uint32_t n_reads, const xdrop_pair *pairs,
                        size_t n_pairs, const xdrop_scoring *s,
                        xdrop_result *out, xdrop_ticket *t);

/* Make a read set resident on the device for xdrop_submit_pairs (host
 * memory, same layout and limits as xdrop_submit; copied before return,
 * together with the reverse complement of every read for reverse-strand
 * pairs: twice the packed size on the device).  Replaces the previous
 * read set; in serving mode it first waits for the requests in flight.
 * Returns XDROP_OK, XDROP_EINVAL or XDROP_ECUDA. */
int xdrop_load_reads(xdrop_ctx *c, const uint32_t *packed, const uint64_t *read_off,
                     const uint32_t *read_len, uint32_t n_reads);

/* Align n_pairs pairs (HOST memory, copied before return) against the
 * resident read set.  In batched mode with a device memory budget too small
 * for the whole pair table, the pairs stream through in chunks sized to the
 * budget, each one a replay of the same CUDA graph (xdrop_stats counts them
 * as graph_replays); XDROP_ENOMEM if not even a 1,024-pair chunk fits.
 * Results go to `out` (host memory, valid until the ticket's sync returns
 * XDROP_OK).  Pairs are validated first (XDROP_EINVAL, nothing queued);
 * reverse-strand pairs (XDROP_PAIR_RC) are accepted.
 *
 * Serving mode (XDROP_MODE_SERVE): thread-safe continuous batching.  The
 * request is queued, admitted once a slot is free and its device buffers
 * fit the context's memory budget (XDROP_ENOMEM if they never can), and
 * its extensions are appended to the work of a persistent kernel that is
 * already running other requests; results are identical to a request run
 * alone.  Other modes: an ordinary submit over the resident reads. */
int xdrop_submit_pairs(xdrop_ctx *c, const xdrop_pair *pairs, size_t n_pairs,
                       const xdrop_scoring *s, xdrop_result *out, xdrop_ticket *t);

/* Counters of the serving loop (all zero outside serving mode). */
int xdrop_get_serve_stats(xdrop_ctx *c, xdrop_serve_stats *st);

/* Serving mode: the hang guard.  A group of the serving kernel that finds
 * no work waits at most idle_ns nanoseconds (default 5 s; 0 restores it),
 * then its warp leaves and counts itself in idle_exits; the kernel ends
 * when every warp has left, and the next request launches it again.  The
 * host normally stops an idle kernel after about 50 ms, so the bound only
 * matters if that stop never arrives.  Takes effect at the next launch of
 * the serving kernel.  Returns XDROP_OK, or XDROP_EINVAL for a NULL c. */
int xdrop_set_serve_idle(xdrop_ctx *c, uint64_t idle_ns);

/* Wait for a ticket.  timeout_ns < 0 waits without bound; otherwise the
 * call returns XDROP_ETIMEDOUT after about timeout_ns and the ticket stays
 * valid for a later sync.  Returns XDROP_OK once the results are in `out`,
 * or an error (XDROP_EINVAL for an unknown or already-synced ticket). */
int xdrop_sync(xdrop_ctx *c, xdrop_ticket t, int64_t timeout_ns);

/* Wait for all work in flight, then release every resource of c. */
void xdrop_free(xdrop_ctx *c);

/* The calling thread's last error message on c (never NULL). */
const char *xdrop_last_error(xdrop_ctx *c);

/* The CUDA stream (cudaStream_t) the context launches its work on. */
void *xdrop_stream(xdrop_ctx *c);

/* Statistics of the most recently synced ticket. */
int xdrop_get_stats(xdrop_ctx *c, xdrop_stats *st);

/* Packed tiles: 16-bit cells, two per 32-bit register, for scorings with
 * match - gap <= 128, mismatch >= -128, mismatch - 2*gap >= 0 and
 * x + match <= 1536, and x + match <= 1022 for the tiles of 32 cells per
 * lane (results identical to the 32-bit tiles; other scorings run the
 * packed 16-cell tile of the same width, else the 32-bit tile of that
 * shape).  Set in `cells` of xdrop_set_tile. */
#define XDROP_TILE_PACKED16 0x100

/* Batched and plain modes: fix the first band tier to `lanes` lanes per extension
 * and `cells` cells per lane (lanes*cells slots per anti-diagonal parity),
 * or pass lanes = 0 to go back to autotuning.  Autotuning (the default)
 * keys the first tile by the scoring and the job's length bucket (the
 * length bin, ceil(log2(max(m, n) + 1)) of an extension, that holds the
 * median of the job's work, read from a device histogram at every batched
 * submit).  The first submit with a new key times the first-tier tiles on
 * a stratified random sample of its pairs (one pair of every 3 with the
 * packed tiles when the scoring fits them, else one of every 8 with the
 * 32-bit tiles) and keeps the fastest for that key.  Tiles: 4x16, 8x8, 16x4,
 * 8x16, 16x8, 32x4, and packed (cells | XDROP_TILE_PACKED16) 4x8, 2x16,
 * 4x16, 8x8, 2x32, 8x16, 16x8, 4x32.  Returns XDROP_EINVAL for another
 * shape.  Serving mode (set the tile before the first xdrop_submit_pairs)
 * runs packed 4x16 by default (a packed tile of 32 cells per lane serves as
 * the 16-cell tile of its width); with a packed first tier, requests whose
 * scoring does not fit 16 bits run on the serving kernel's 32-bit second
 * tier. */
int xdrop_set_tile(xdrop_ctx *c, int lanes, int cells);

/* Several seeds per read pair, keeping the best extension.  Consecutive
 * pair records with the same a and b (b with its strand flag) are the
 * seeds of one read pair, a group.  For every record p, best[p] receives
 * the index of the record of p's group with the highest total score
 * left_score + seed_len * match + right_score among records with status
 * XDROP_STATUS_OK; ties go to the lowest index; a group without such a
 * record gives 0xFFFFFFFF.  pairs, results (as written by a submit) and
 * best are device arrays of n entries (n < 2^31); the kernel runs
 * asynchronously on the context's stream (xdrop_stream), after the work
 * already queued there.  The exact seed scores seed_len matches (the
 * seed-and-extend of Section "Related works", BELLA paragraph).
 * XDROP_EINVAL for NULL arrays or too many records. */
int xdrop_best_seeds_device(xdrop_ctx *c, const xdrop_pair *pairs, const xdrop_result *results,
                            size_t n, int32_t match, uint32_t *best);

/* Seed discovery: the candidate pairs of the resident read set
 * (xdrop_load_reads), the step upstream of seed-and-extend (Section
 * "Related works", diBELLA 2D paragraph: overlaps are the nonzeros of
 * A * A^T, A the read-by-reliable-k-mer matrix; Section "Experimental
 * Setup": k = 31, stride 1, frequency window [20, 30] or [20, 50]).
 *
 * A k-mer is k consecutive bases of a read starting at a multiple of
 * stride; its canonical code is the smaller 2k-bit code (first base most
 * significant) of the k-mer and of its reverse complement.  Its count is
 * its number of occurrences in all reads (repeats in one read included);
 * it is reliable iff lo <= count <= hi.  Reads a < b are a candidate pair
 * iff they share a reliable k-mer (its first occurrence in each read
 * counts).  The pair's seed is the shared k-mer with the smallest position
 * in a (then in b, then the smallest code): seed_a and seed_b are its
 * first positions, seed_len = k; if it was read on opposite strands of a
 * and b, b carries XDROP_PAIR_RC and seed_b = len_b - k - pos_b, a
 * position in b's reverse complement.  The records can be passed as they
 * are to xdrop_submit_pairs.
 *
 * Writes min(cap, total) candidates in increasing (a, b) order to pairs
 * and, unless shared is NULL, the number of shared reliable k-mers of each
 * to shared (host memory); *n = total.  The result stays in the context
 * until the read set or the parameters change, so a call with a larger cap
 * only copies.  Synchronous; other calls on the same context (serving
 * submits too) wait until it returns.  Limits: 1 <= k <= 32, stride >= 1,
 * 1 <= lo <= hi <= 1024 (XDROP_EINVAL; also without resident reads);
 * fewer than 2^31 occurrences and 2^31 (pair, shared k-mer) entries, and
 * the context's memory budget (XDROP_ENOMEM).
 *
 * Two products compute the same candidates.  XDROP_SEEDS_ROWWISE (default)
 * builds A's rows and columns and accumulates each read's partners in a
 * shared-memory hash table of 2,048 slots, one thread block per read,
 * without per-entry tables; a read with more partners than that makes the
 * call run the sort-based product instead.  XDROP_SEEDS_SORT writes one
 * entry per (read pair, shared reliable k-mer), sorts the entries by pair
 * and reduces them.  xdrop_get_seed_stats tells which ran. */
#define XDROP_SEEDS_ROWWISE 0u
#define XDROP_SEEDS_SORT 1u

typedef struct {
    uint32_t k;      /* k-mer length                               */
    uint32_t stride; /* a k-mer starts at every stride-th position */
    uint32_t lo, hi; /* reliable iff lo <= count <= hi             */
    uint32_t flags;  /* XDROP_SEEDS_ROWWISE or XDROP_SEEDS_SORT    */
} xdrop_kmer_params;

int xdrop_find_candidates(xdrop_ctx *c, const xdrop_kmer_params *p, xdrop_pair *pairs,
                          uint32_t *shared, size_t cap, size_t *n);

/* Counters of the last xdrop_find_candidates that computed (not of calls
 * that only copied a kept result). */
typedef struct {
    double ms;            /* device time, CUDA events around the pipeline  */
    uint64_t occurrences; /* k-mer occurrences                             */
    uint64_t runs;        /* k-mers that occur at least twice              */
    uint64_t candidates;  /* candidate pairs                               */
    uint32_t product;     /* XDROP_SEEDS_ROWWISE or XDROP_SEEDS_SORT: the
                             product that produced them                    */
    uint32_t pad;
    uint64_t nonzeros;    /* nonzeros of A (read, reliable k-mer), counted
                             by the row-wise product; 0 if it did not run  */
} xdrop_seed_stats;

int xdrop_get_seed_stats(xdrop_ctx *c, xdrop_seed_stats *st);

/* Adaptive acceptance of aligned pairs (Section "Related works", BELLA
 * paragraph: an adaptive threshold decides which X-drop alignments are
 * kept; the paper gives no formula, so this is the library's reading).
 * For pair p with result r, accept[p] = 1 iff r.status is XDROP_STATUS_OK,
 * both read ids are below n_reads, and
 *   r.left_score + seed_len * match + r.right_score
 *     >= (1 - delta) * L * (phi * match + (1 - phi) * mismatch),
 * where L = min(seed_a, seed_b) + min(len_a - seed_a, len_b - seed_b) is the
 * overlap the seed implies (b's length and positions on the strand the
 * pair names), phi = (1 - e)^2 is the chance that an overlap column pairs
 * two correct bases at per-read error rate e, e = error_e4 / 10^4 and
 * delta = delta_e4 / 10^4.  The comparison is exact (integers).
 * pairs, results, read_len and accept are device arrays (n entries,
 * n_reads lengths, n flags); the kernel runs asynchronously on the
 * context's stream after the work queued there.  XDROP_EINVAL for NULL
 * arrays or error_e4 / delta_e4 above 10,000. */
typedef struct {
    int32_t match, mismatch; /* the scoring the pairs were aligned with */
    uint32_t error_e4;       /* per-read error rate, units of 1e-4      */
    uint32_t delta_e4;       /* slack below the expected score, 1e-4    */
} xdrop_accept_params;

int xdrop_accept_device(xdrop_ctx *c, const xdrop_pair *pairs, const xdrop_result *results,
                        size_t n, const uint32_t *read_len, uint32_t n_reads,
                        const xdrop_accept_params *p, uint8_t *accept);

/* Task ids (2*pair + 1 for a right extension, 2*pair for a left one)
 * that the first band tier handed to a wider tier during the most recently
 * synced ticket.  Copies up to cap ids to dst (host memory) and the total
 * number to *n.  For diagnostics and for separating the first tier's work
 * in rate measurements. */
int xdrop_last_spills(xdrop_ctx *c, uint32_t *dst, size_t cap, size_t *n);

/* Cell counts: for pair p, cells[2p] and cells[2p+1] receive the number of
 * DP cells of its left and right extension (the origin plus every cell of
 * the anti-diagonal ranges of the reading above: the hull of the live
 * extent of d-1 and of d-2 shifted by one, clipped to the rectangle).
 * Inputs as xdrop_submit_device; `cells` is device memory of 2*n_pairs
 * int64.  Synchronous.  Used to compute cell-update rates. */
int xdrop_count_cells_device(xdrop_ctx *c, const uint32_t *packed,
                             uint64_t n_words, const uint64_t *read_off,
                             const uint32_t *read_len, uint32_t n_reads,
                             const xdrop_pair *pairs, size_t n_pairs,
                             const xdrop_scoring *s, int64_t *cells);

/* Allocation-free alignment (the paper has no counterpart; this serves
 * callers that cannot allocate device memory when they align: a process
 * whose device memory belongs to another allocator, a latency-critical
 * path that cannot pay for cudaMalloc/cudaFree and their implicit
 * synchronisation, or work issued while a stream is being captured).
 *
 * Same inputs and results as xdrop_submit_device, all in DEVICE memory of
 * the current device and owned by the caller; the work is enqueued on
 * `stream` (a cudaStream_t, NULL for the default stream) and the call
 * returns without waiting: results are in `out` once that stream has
 * reached this point.  No context is needed and no device memory is
 * allocated: the scratch is a static 32 MiB array inside the library that
 * every device using the library holds until the process exits.  Every
 * call looks up the array's address on the current device; the first call
 * on a device also loads the library's device code there, so make that
 * first call before any stream capture that should contain later calls.
 * All calls on a device share the array: calls whose work may overlap on
 * the GPU race and must be ordered (same stream, or events).  Every extension runs on the
 * unbounded-band tier (one CTA per extension), which is exact for any band
 * but slower than the batched path.
 *
 * max_read_len must bound every read length; it sizes the per-CTA scratch
 * (3*(max_read_len+1) int32 per extension) and values above 2,796,202
 * return XDROP_EINVAL.  Pairs that fail the limits get status
 * XDROP_STATUS_INVALID and zero scores; an extension longer than
 * max_read_len allows gets XDROP_STATUS_TOO_LONG and zeros in that side's
 * score and coordinates.  Returns XDROP_OK once the work is enqueued,
 * XDROP_EINVAL for bad arguments, XDROP_ECUDA if the launch failed
 * (message from xdrop_static_last_error). */
int xdrop_align_static(const uint32_t *packed, uint64_t n_words,
                       const uint64_t *read_off, const uint32_t *read_len,
                       uint32_t n_reads, const xdrop_pair *pairs, size_t n_pairs,
                       const xdrop_scoring *s, uint32_t max_read_len,
                       xdrop_result *out, void *stream);

/* The calling thread's last error message from xdrop_align_static. */
const char *xdrop_static_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
