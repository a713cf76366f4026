/*
 * X-drop seed-and-extend oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of the pairwise X-drop
 * alignment that the paper's GPU schedulers feed (Section "Related works",
 * LOGAN paragraph: X-drop dynamic programming over anti-diagonals; Section
 * "Comparison between small dataset and large dataset": Needleman-Wunsch /
 * Smith-Waterman with X-drop; Section "Related works", BELLA paragraph:
 * seed-and-extend).  The paper names the method but prints no recurrence,
 * pruning rule or tie-break, so this code follows one stated reading
 * ("Definition C", restated at the top of xdrop_oracle.c) step by step.
 *
 * Who may use it: tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg.  It shares no code, header, table or helper with the CUDA
 * library, and the library never calls it.
 */
#ifndef XDROP_ORACLE_H
#define XDROP_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t match;    /* score of an identical base pair                */
    int32_t mismatch; /* score of a substitution                         */
    int32_t gap;      /* score of one inserted or deleted base (linear)  */
    int32_t x;        /* the X-drop threshold, >= 0                      */
} orc_scoring;

/* b's top bit (ORC_PAIR_RC) selects the reverse strand of read b: the
 * pair aligns read a against the reverse complement of read b (base k of
 * it is the complement, code 3 - c, of base len_b - 1 - k of read b), and
 * seed_b and the reported b coordinates are positions in that reverse
 * complement.  The paper's reads come from both strands (overlaps of
 * long reads, Section "Method"); it does not spell out the strand step,
 * so this is the reading the oracle fixes. */
#define ORC_PAIR_RC 0x80000000u

typedef struct {
    uint32_t a, b;           /* read ids (b may carry ORC_PAIR_RC)        */
    uint32_t seed_a, seed_b; /* 0-based start of the exact seed on a / b */
    uint32_t seed_len;       /* seed length in bases                      */
} orc_pair;

typedef struct {
    int32_t left_score, left_begin_a, left_begin_b;
    int32_t right_score, right_end_a, right_end_b; /* end exclusive */
    int32_t status;                                /* 0 = ok         */
} orc_result;

/* One extension over a[1..m], b[1..n] given as 0-based code arrays
 * (a[k-1] holds a_k).  Writes the best score, its cell (i*, j*) and the
 * number of DP cells evaluated (the origin plus every cell of every
 * computed anti-diagonal range).  Returns 0, or -1 on bad arguments. */
int orc_extend(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
               const orc_scoring *sc, int32_t *score, int64_t *best_i,
               int64_t *best_j, int64_t *cells);

/* Unpack bases [off, off+len) of a 2-bit packed buffer (16 bases per
 * 32-bit word, base k in bits 2(k mod 16) .. 2(k mod 16)+1 of word k/16)
 * into one code per byte. */
void orc_unpack(const uint32_t *packed, uint64_t off, uint64_t len,
                uint8_t *codes);

/* Left and right extension of every pair (seed-and-extend), using
 * nthreads worker threads (<= 1 means the calling thread only).  cells
 * may be NULL; otherwise cells[2p] / cells[2p+1] receive the cell counts
 * of the left / right extension of pair p.  Returns 0, or -1 if a pair
 * references a missing read or a seed outside its read (that pair's
 * status is set to 1 and its scores to 0). */
int orc_align_pairs(const uint32_t *packed, const uint64_t *read_off,
                    const uint32_t *read_len, uint32_t n_reads,
                    const orc_pair *pairs, size_t n_pairs,
                    const orc_scoring *sc, orc_result *out, int64_t *cells,
                    int nthreads);

#ifdef __cplusplus
}
#endif
#endif
