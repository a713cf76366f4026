/*
 * X-drop seed-and-extend oracle: TEST INFRASTRUCTURE ONLY (see
 * xdrop_oracle.h for who may call it).  Plain C, no intrinsics, no code
 * shared with the CUDA library.
 *
 * The paper (Section "Related works", LOGAN paragraph) describes X-drop as
 * a dynamic program whose cells on one anti-diagonal are independent, and
 * (Section "Comparison between small dataset and large dataset") as
 * Needleman-Wunsch / Smith-Waterman with X-drop; the BELLA paragraph places
 * it in a seed-and-extend scheme.  It prints no recurrence.  This file
 * computes the following reading, "Definition C", in this order:
 *
 *  1. One extension runs on a[1..m], b[1..n].  Right extension: a_k is the
 *     k-th base after the seed on read A, b_k likewise on B.  Left
 *     extension: a_k = A[seed_a - k], b_k = B[seed_b - k] (the prefixes
 *     read backwards).  s(x,y) = match if x == y else mismatch; gaps are
 *     linear with score `gap` per base.
 *  2. Cells (i,j), 0 <= i <= m, 0 <= j <= n, lie on anti-diagonal d = i+j.
 *     H(0,0) = 0.  R(i,j) = max(H(i-1,j-1) + s(a_i,b_j), H(i-1,j) + gap,
 *     H(i,j-1) + gap), where a term whose predecessor lies outside the
 *     rectangle or is pruned is left out; with no term left the cell is
 *     pruned.
 *  3. X-drop test: T_0 = 0 and T_d = max(T_{d-1}, max live H on d).  A cell
 *     on d >= 1 is live iff R >= T_{d-1} - X, and then H = R; otherwise it
 *     is pruned.  (Strictly below the threshold prunes; the threshold uses
 *     the best score of the earlier diagonals only.)
 *  4. Diagonal d is evaluated for i in the hull of [lo_{d-1}, hi_{d-1}+1]
 *     and [lo_{d-2}+1, hi_{d-2}+1], clipped to [max(0,d-n), min(m,d)],
 *     where lo/hi are the first/last live i of that diagonal (an entirely
 *     pruned diagonal contributes nothing).  The extension stops after
 *     diagonal d if d and d-1 are both entirely pruned, or after d = m+n.
 *  5. The result is T at the end and the first cell that reached it
 *     (smallest d, then smallest i).  Right extension: end = seed + len +
 *     (i*, j*).  Left extension: begin = seed - (i*, j*).
 *  6. The cell count is 1 (the origin) plus the length of every range
 *     evaluated in step 4.
 *
 * Values are held in int64, so nothing here can overflow for any input the
 * library accepts.
 */
#include "xdrop_oracle.h"

#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

/* One anti-diagonal: H and a live flag for i in [lo, hi] (the evaluated
 * range; cells outside it count as pruned), plus the live extent. */
typedef struct {
    int64_t *h;
    uint8_t *live;
    int64_t lo, hi;           /* evaluated range; lo > hi if none */
    int any;                  /* at least one live cell            */
    int64_t live_lo, live_hi; /* first / last live i               */
} diag_t;

static int diag_is_live(const diag_t *dg, int64_t i)
{
    return i >= dg->lo && i <= dg->hi && dg->live[i];
}

static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

int orc_extend(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
               const orc_scoring *sc, int32_t *score, int64_t *best_i,
               int64_t *best_j, int64_t *cells)
{
    if (m < 0 || n < 0 || !sc || sc->x < 0) return -1;

    diag_t dg[3];
    for (int r = 0; r < 3; ++r) {
        dg[r].h = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
        dg[r].live = (uint8_t *)malloc((size_t)(m + 1));
        if (!dg[r].h || !dg[r].live) {
            for (int q = 0; q <= r; ++q) { free(dg[q].h); free(dg[q].live); }
            return -1;
        }
        dg[r].lo = 1; dg[r].hi = 0; dg[r].any = 0;
    }

    /* Diagonal 0: the origin, H(0,0) = 0, live; T_0 = 0. */
    diag_t *d2 = &dg[0], *d1 = &dg[1], *cur = &dg[2];
    d1->lo = d1->hi = 0;
    d1->h[0] = 0;
    d1->live[0] = 1;
    d1->any = 1;
    d1->live_lo = d1->live_hi = 0;

    int64_t T = 0, bi = 0, bj = 0, ncells = 1;

    for (int64_t d = 1; d <= m + n; ++d) {
        /* Step 4: the range of d from the live extents of d-1 and d-2. */
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        if (d1->any) { lo = min64(lo, d1->live_lo); hi = max64(hi, d1->live_hi + 1); }
        if (d2->any) { lo = min64(lo, d2->live_lo + 1); hi = max64(hi, d2->live_hi + 1); }
        lo = max64(lo, max64(0, d - n));
        hi = min64(hi, min64(m, d));

        cur->lo = lo;
        cur->hi = hi;
        cur->any = 0;
        int64_t dmax = 0, dmax_i = -1;

        for (int64_t i = lo; i <= hi; ++i) {
            int64_t j = d - i;
            ++ncells;
            /* Step 2: the three predecessor terms. */
            int have = 0;
            int64_t r = 0;
            if (i >= 1 && j >= 1 && diag_is_live(d2, i - 1)) {
                int64_t s = (a[i - 1] == b[j - 1]) ? sc->match : sc->mismatch;
                int64_t t = d2->h[i - 1] + s;
                if (!have || t > r) r = t;
                have = 1;
            }
            if (i >= 1 && diag_is_live(d1, i - 1)) { /* from (i-1, j) */
                int64_t t = d1->h[i - 1] + sc->gap;
                if (!have || t > r) r = t;
                have = 1;
            }
            if (j >= 1 && diag_is_live(d1, i)) { /* from (i, j-1) */
                int64_t t = d1->h[i] + sc->gap;
                if (!have || t > r) r = t;
                have = 1;
            }
            /* Step 3: the X-drop test against T_{d-1}. */
            int live = have && r >= T - (int64_t)sc->x;
            cur->live[i] = (uint8_t)live;
            cur->h[i] = live ? r : 0;
            if (live) {
                if (!cur->any) cur->live_lo = i;
                cur->live_hi = i;
                cur->any = 1;
                if (dmax_i < 0 || r > dmax) { dmax = r; dmax_i = i; }
            }
        }

        /* Step 3 / 5: T_d, and the first cell that raised it. */
        if (dmax_i >= 0 && dmax > T) {
            T = dmax;
            bi = dmax_i;
            bj = d - dmax_i;
        }

        /* Step 4: stop when d and d-1 are both entirely pruned. */
        int stop = !cur->any && !d1->any;

        diag_t *old2 = d2;
        d2 = d1;
        d1 = cur;
        cur = old2;
        if (stop) break;
    }

    for (int r = 0; r < 3; ++r) { free(dg[r].h); free(dg[r].live); }
    *score = (int32_t)T;
    *best_i = bi;
    *best_j = bj;
    if (cells) *cells = ncells;
    return 0;
}

void orc_unpack(const uint32_t *packed, uint64_t off, uint64_t len,
                uint8_t *codes)
{
    for (uint64_t k = 0; k < len; ++k) {
        uint64_t p = off + k;
        codes[k] = (uint8_t)((packed[p / 16] >> (2 * (p % 16))) & 3u);
    }
}

/* Left and right extension of one pair. */
static int align_one(const uint32_t *packed, const uint64_t *read_off,
                     const uint32_t *read_len, uint32_t n_reads,
                     const orc_pair *p, const orc_scoring *sc, orc_result *o,
                     int64_t *cells2)
{
    memset(o, 0, sizeof(*o));
    if (cells2) { cells2[0] = 0; cells2[1] = 0; }
    const uint32_t rb = p->b & ~ORC_PAIR_RC;  /* read id of b */
    const int rc = (p->b & ORC_PAIR_RC) != 0;
    if (p->a >= n_reads || rb >= n_reads) { o->status = 1; return -1; }
    uint64_t la = read_len[p->a], lb = read_len[rb];
    if ((uint64_t)p->seed_a + p->seed_len > la ||
        (uint64_t)p->seed_b + p->seed_len > lb) {
        o->status = 1;
        return -1;
    }

    uint8_t *A = (uint8_t *)malloc(la ? la : 1);
    uint8_t *B = (uint8_t *)malloc(lb ? lb : 1);
    int64_t m_r = (int64_t)(la - p->seed_a - p->seed_len);
    int64_t n_r = (int64_t)(lb - p->seed_b - p->seed_len);
    int64_t m_l = p->seed_a, n_l = p->seed_b;
    int64_t mx = max64(max64(m_r, n_r), max64(m_l, n_l));
    uint8_t *ea = (uint8_t *)malloc((size_t)mx + 1);
    uint8_t *eb = (uint8_t *)malloc((size_t)mx + 1);
    if (!A || !B || !ea || !eb) {
        free(A); free(B); free(ea); free(eb);
        o->status = 2;
        return -1;
    }
    orc_unpack(packed, read_off[p->a], la, A);
    orc_unpack(packed, read_off[rb], lb, B);
    if (rc) {  /* the reverse complement of read b, written out */
        for (uint64_t k = 0; k < lb / 2; ++k) {
            const uint8_t t = B[k];
            B[k] = B[lb - 1 - k];
            B[lb - 1 - k] = t;
        }
        for (uint64_t k = 0; k < lb; ++k) B[k] = (uint8_t)(3 - B[k]);
    }

    int32_t sc_out;
    int64_t bi, bj, c;

    /* Left extension: a_k = A[seed_a - k], b_k = B[seed_b - k]. */
    for (int64_t k = 1; k <= m_l; ++k) ea[k - 1] = A[p->seed_a - k];
    for (int64_t k = 1; k <= n_l; ++k) eb[k - 1] = B[p->seed_b - k];
    orc_extend(ea, m_l, eb, n_l, sc, &sc_out, &bi, &bj, &c);
    o->left_score = sc_out;
    o->left_begin_a = (int32_t)(p->seed_a - bi);
    o->left_begin_b = (int32_t)(p->seed_b - bj);
    if (cells2) cells2[0] = c;

    /* Right extension: a_k = A[seed_a + seed_len + k - 1]. */
    for (int64_t k = 1; k <= m_r; ++k) ea[k - 1] = A[p->seed_a + p->seed_len + k - 1];
    for (int64_t k = 1; k <= n_r; ++k) eb[k - 1] = B[p->seed_b + p->seed_len + k - 1];
    orc_extend(ea, m_r, eb, n_r, sc, &sc_out, &bi, &bj, &c);
    o->right_score = sc_out;
    o->right_end_a = (int32_t)(p->seed_a + p->seed_len + bi);
    o->right_end_b = (int32_t)(p->seed_b + p->seed_len + bj);
    if (cells2) cells2[1] = c;

    free(A); free(B); free(ea); free(eb);
    return 0;
}

typedef struct {
    const uint32_t *packed;
    const uint64_t *read_off;
    const uint32_t *read_len;
    uint32_t n_reads;
    const orc_pair *pairs;
    size_t n_pairs;
    const orc_scoring *sc;
    orc_result *out;
    int64_t *cells;
    atomic_size_t next;
    atomic_int bad;
} job_t;

static void *worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    for (;;) {
        size_t p = atomic_fetch_add(&jb->next, 1);
        if (p >= jb->n_pairs) break;
        if (align_one(jb->packed, jb->read_off, jb->read_len, jb->n_reads,
                      &jb->pairs[p], jb->sc, &jb->out[p],
                      jb->cells ? &jb->cells[2 * p] : NULL) != 0)
            atomic_store(&jb->bad, 1);
    }
    return NULL;
}

int orc_align_pairs(const uint32_t *packed, const uint64_t *read_off,
                    const uint32_t *read_len, uint32_t n_reads,
                    const orc_pair *pairs, size_t n_pairs,
                    const orc_scoring *sc, orc_result *out, int64_t *cells,
                    int nthreads)
{
    job_t jb;
    jb.packed = packed;
    jb.read_off = read_off;
    jb.read_len = read_len;
    jb.n_reads = n_reads;
    jb.pairs = pairs;
    jb.n_pairs = n_pairs;
    jb.sc = sc;
    jb.out = out;
    jb.cells = cells;
    atomic_init(&jb.next, 0);
    atomic_init(&jb.bad, 0);

    if (nthreads <= 1) {
        worker(&jb);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
        int started = 0;
        for (int t = 0; t < nthreads; ++t)
            if (pthread_create(&th[started], NULL, worker, &jb) == 0) ++started;
        if (started == 0) worker(&jb);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
        free(th);
    }
    return atomic_load(&jb.bad) ? -1 : 0;
}
