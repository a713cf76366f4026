// Device code of the X-drop seed-and-extend path (sm_103a).
//
// Method: the anti-diagonal X-drop extension of the paper's alignment step
// (Section "Related works", LOGAN paragraph: the cells of one anti-diagonal
// are independent; Section "Comparison between small dataset and large
// dataset": Needleman-Wunsch / Smith-Waterman with X-drop), in the reading
// stated in include/xdrop.h.  Everything is int32 and bit-exact.
//
// Band-window tiers (extend_window): a group of LANES lanes owns one
// extension.  Cells are addressed by the diagonal offset k = i - j.  On
// even diagonals k is even and on odd ones odd, so each parity keeps its
// own array of W = LANES*C slots in registers: slot s of lane s/C, entry
// s%C.  With a window base kb (even), even-diagonal slot s is k = kb + 2s and
// odd-diagonal slot s is k = kb + 1 + 2s.  Then
//     even d:  E[s] = max(E[s] + sub, max(O[s-1], O[s]) + gap)
//     odd  d:  O[s] = max(O[s] + sub, max(E[s], E[s+1]) + gap)
// (the diagonal predecessor is the same slot two diagonals back, so it is
// updated in place, and only one value crosses a lane boundary per step).
// A path along the main diagonal keeps k fixed, so the window only moves
// with net indels: when an edge slot becomes live the window shifts by one
// slot; if the opposite edge is live too the band no longer fits, the
// extension is abandoned and re-run by the next wider tier.  Cells outside
// the window are therefore always pruned, so the window computes exactly
// the pruned dynamic program.
//
// Bases: per lane, a 2-bit packed window of the 16 a-bases a_{i0..i0+15}
// (field t pairs with cell t) and of b_{j0}, b_{j0-1}, ... (field t is
// b_{j0-t}), each with a 16-base lookahead register.  Going from an even to
// an odd diagonal moves the a-window by one base, from odd to even the
// b-window; both are one funnel shift.  Equality of the fields of the two
// windows gives the substitution score of all C cells at once.
//
// Unbounded tier (wide_kernel): one CTA per extension, cells of the
// step-4 range spread over the threads, diagonals kept in global scratch.
// It follows the reading directly and has no width limit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "xd_types.cuh"

namespace xd {

// ---------------------------------------------------------------------------
// Base access.  Positions outside the buffer are clamped: such bases only
// ever meet cells outside the DP rectangle, which are masked or pruned.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_word(const Seq &S, int64_t w)
{
    w = w < 0 ? 0 : (w >= S.nw ? S.nw - 1 : w);
    return __ldg(S.pk + w);
}

// field v = base (q + v), v = 0..15
__device__ __forceinline__ uint32_t load16(const Seq &S, int64_t q)
{
    int64_t w = q >> 4;
    uint32_t sh = (uint32_t)(q & 15) * 2u;
    return __funnelshift_r(ld_word(S, w), ld_word(S, w + 1), sh);
}

// reverse the order of the 16 2-bit fields
__device__ __forceinline__ uint32_t rev16(uint32_t x)
{
    x = __brev(x);
    return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

// field u = c_{k+u}
__device__ __forceinline__ uint32_t fwd16(const Seq &S, int32_t k)
{
    if (S.dir > 0) return load16(S, S.s0 + (k - 1));
    return rev16(load16(S, S.s0 - (k - 1) - 15));
}

// field t = c_{k-t}
__device__ __forceinline__ uint32_t back16(const Seq &S, int32_t k)
{
    if (S.dir > 0) return rev16(load16(S, S.s0 + (k - 16)));
    return load16(S, S.s0 - (k - 1));
}

__device__ __forceinline__ int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Register band window: one extension per LANES-lane group.
// Returns 0 when done, 1 when the band outgrew the window.
// ---------------------------------------------------------------------------
template <int LANES, int C>
struct Window {
    static constexpr int W = LANES * C;
    int32_t E[C], O[C];
};

template <int LANES, int C, bool ODD, bool MASKED>
__device__ __forceinline__ int32_t dp_step(int32_t (&V)[C], const int32_t (&U)[C],
                                           int32_t edge, uint32_t eq,
                                           const Scoring &sc, int32_t thr,
                                           int32_t i0, int32_t j0, int32_t m,
                                           int32_t n)
{
    // V: this parity (holds d-2, becomes d); U: the other parity (d-1).
    // ODD:  V[t] <- max(V[t] + s, max(U[t], U[t+1]) + gap), U[C] = edge
    // EVEN: V[t] <- max(V[t] + s, max(U[t-1], U[t]) + gap), U[-1] = edge
    int32_t lmax = NEG;
#pragma unroll
    for (int t = 0; t < C; ++t) {
        int32_t nb;
        if (ODD) nb = imax(U[t], (t + 1 < C) ? U[t + 1] : edge);
        else nb = imax((t > 0) ? U[t - 1] : edge, U[t]);
        int32_t s = ((eq >> (2 * t)) & 1u) ? sc.match : sc.mismatch;
        int32_t r = imax(V[t] + s, nb + sc.gap);
        if (MASKED) {
            if (i0 + t > m || j0 - t > n) r = NEG;
        }
        r = (r >= thr) ? r : NEG;
        V[t] = r;
        lmax = imax(lmax, r);
    }
    return lmax;
}

template <int LANES>
__device__ __forceinline__ unsigned group_mask(int gbase)
{
    if constexpr (LANES == 32) return FULL;
    else return ((1u << LANES) - 1u) << gbase;
}

// Maximum over the LANES lanes of each group, in code every lane of the
// warp runs together (the lockstep loops): a butterfly of log2(LANES)
// shuffle-and-max steps.  A redux with each group's own mask is serialised
// over the warp's groups, about a quarter of the lockstep kernels' time
// when measured; code whose groups diverge keeps the masked redux.
template <int LANES>
__device__ __forceinline__ int32_t lockstep_group_max(int32_t v)
{
    if constexpr (LANES == 32) {
        return __reduce_max_sync(FULL, v);
    } else {
#pragma unroll
        for (int off = 1; off < LANES; off <<= 1) v = max(v, __shfl_xor_sync(FULL, v, off, LANES));
        return v;
    }
}

template <int LANES, int C, bool COUNT>
__device__ int extend_window(const Ext &e, const Scoring sc, int glane, int gbase,
                             int32_t &best, int32_t &best_i, int32_t &best_j,
                             int64_t &cells_out)
{
    constexpr int W = LANES * C;
    const unsigned gm = group_mask<LANES>(gbase);
    const int32_t m = e.m, n = e.n;
    const int32_t dmax = m + n;

    int32_t E[C], O[C];
#pragma unroll
    for (int t = 0; t < C; ++t) {
        E[t] = (glane * C + t == W / 2) ? 0 : NEG;  // origin at k = 0
        O[t] = NEG;
    }
    int32_t kb = -W;  // even-diagonal slot s is k = kb + 2s
    // Lane's first cell on diagonal d: i0 = ceil((d+kb)/2) + glane*C.
    int32_t i0 = ((kb + 1) >> 1) + glane * C;
    int32_t j0 = -((kb + 1) >> 1) - glane * C;
    uint32_t Aw = fwd16(e.A, i0), LA = fwd16(e.A, i0 + 16);
    uint32_t Bw = back16(e.B, j0), LB = back16(e.B, j0 + 16);
    int la_n = 16, lb_n = 16;

    int32_t T = 0, bi = 0, bj = 0;
    bool prev_dead = false;
    int32_t d = 0;

    // Cell counting: live extents (in i) of diagonals d-1 and d-2.
    int32_t lo1 = 0, hi1 = 0, lo2 = 1, hi2 = 0;
    int64_t cells = 1;

    int status = 0;

    auto reload = [&]() {
        Aw = fwd16(e.A, i0);
        LA = fwd16(e.A, i0 + 16);
        Bw = back16(e.B, j0);
        LB = back16(e.B, j0 + 16);
        la_n = 16;
        lb_n = 16;
    };

    // Diagonal bookkeeping shared by both parities.  V holds the new
    // diagonal.  Returns true when the extension is finished.
    auto finish_diag = [&](int32_t (&V)[C], int32_t lmax, bool odd) -> bool {
        const int32_t M = __reduce_max_sync(gm, lmax);
        const int32_t ia = i0 - glane * C;  // group's first i on d
        if (COUNT) {
            int32_t lo = 0x7fffffff, hi = -0x7fffffff;
            if (lo1 <= hi1) { lo = min(lo, lo1); hi = max(hi, hi1 + 1); }
            if (lo2 <= hi2) { lo = min(lo, lo2 + 1); hi = max(hi, hi2 + 1); }
            lo = max(lo, max(0, d - n));
            hi = min(hi, min(m, d));
            if (hi >= lo) cells += (int64_t)(hi - lo + 1);
            int fl = C, ll = -1;
#pragma unroll
            for (int t = C - 1; t >= 0; --t)
                if (V[t] != NEG) fl = t;
#pragma unroll
            for (int t = 0; t < C; ++t)
                if (V[t] != NEG) ll = t;
            unsigned bal = __ballot_sync(gm, fl < C);
            lo2 = lo1;
            hi2 = hi1;
            if (bal) {
                int lf = __ffs(bal) - 1, lh = 31 - __clz(bal);
                int flv = __shfl_sync(gm, fl, lf);
                int llv = __shfl_sync(gm, ll, lh);
                lo1 = ia + (lf - gbase) * C + flv;
                hi1 = ia + (lh - gbase) * C + llv;
            } else {
                lo1 = 1;
                hi1 = 0;
            }
        }
        if (M > T) {  // first cell of the diagonal reaching M
            int ft = C;
#pragma unroll
            for (int t = C - 1; t >= 0; --t)
                if (V[t] == M) ft = t;
            unsigned bal = __ballot_sync(gm, ft < C);
            int src = __ffs(bal) - 1;
            int fts = __shfl_sync(gm, ft, src);
            bi = ia + (src - gbase) * C + fts;
            bj = d - bi;
            T = M;
        }
        const bool dead = (M == NEG);
        if (dead && prev_dead) return true;
        prev_dead = dead;
        if (d >= dmax) return true;
        // Window edges.  After an odd diagonal the top slot may seed a cell
        // above the window on the next (even) diagonal; after an even one
        // the bottom slot may seed a cell below it on the next odd one.
        if (odd) {
            int32_t vhi = __shfl_sync(gm, V[C - 1], gbase + LANES - 1);
            if (vhi != NEG) {
                int32_t vlo = __shfl_sync(gm, V[0], gbase);
                if (vlo != NEG) { status = 1; return true; }
                // shift up: kb += 2, slot s takes slot s+1
                int32_t ne = __shfl_down_sync(gm, E[0], 1, LANES);
                int32_t no = __shfl_down_sync(gm, O[0], 1, LANES);
                if (glane == LANES - 1) { ne = NEG; no = NEG; }
#pragma unroll
                for (int t = 0; t < C - 1; ++t) { E[t] = E[t + 1]; O[t] = O[t + 1]; }
                E[C - 1] = ne;
                O[C - 1] = no;
                kb += 2;
                i0 += 1;
                j0 -= 1;
                reload();
            }
        } else {
            int32_t vlo = __shfl_sync(gm, V[0], gbase);
            if (vlo != NEG) {
                int32_t vhi = __shfl_sync(gm, V[C - 1], gbase + LANES - 1);
                if (vhi != NEG) { status = 1; return true; }
                // shift down: kb -= 2, slot s takes slot s-1
                int32_t pe = __shfl_up_sync(gm, E[C - 1], 1, LANES);
                int32_t po = __shfl_up_sync(gm, O[C - 1], 1, LANES);
                if (glane == 0) { pe = NEG; po = NEG; }
#pragma unroll
                for (int t = C - 1; t > 0; --t) { E[t] = E[t - 1]; O[t] = O[t - 1]; }
                E[0] = pe;
                O[0] = po;
                kb -= 2;
                i0 -= 1;
                j0 += 1;
                reload();
            }
        }
        return false;
    };

    while (d < dmax) {
        // ---------------- odd diagonal: a-window advances ----------------
        ++d;
        ++i0;
        Aw = __funnelshift_r(Aw, LA, 2);
        LA >>= 2;
        if (--la_n == 0) { LA = fwd16(e.A, i0 + 16); la_n = 16; }
        {
            const int32_t thr = T - sc.x;
            const uint32_t xx = Aw ^ Bw;
            const uint32_t eq = ~(xx | (xx >> 1)) & 0x55555555u;
            int32_t edge = __shfl_down_sync(gm, E[0], 1, LANES);
            if (glane == LANES - 1) edge = NEG;
            const int32_t ia = i0 - glane * C, jb = j0 + glane * C;
            const bool masked = (ia + W - 1 > m) || (jb > n);
            int32_t lmax;
            if (masked)
                lmax = dp_step<LANES, C, true, true>(O, E, edge, eq, sc, thr, i0, j0, m, n);
            else
                lmax = dp_step<LANES, C, true, false>(O, E, edge, eq, sc, thr, i0, j0, m, n);
            if (finish_diag(O, lmax, true)) break;
        }
        // ---------------- even diagonal: b-window advances ----------------
        ++d;
        ++j0;
        Bw = __funnelshift_l(LB, Bw, 2);
        LB <<= 2;
        if (--lb_n == 0) { LB = back16(e.B, j0 + 16); lb_n = 16; }
        {
            const int32_t thr = T - sc.x;
            const uint32_t xx = Aw ^ Bw;
            const uint32_t eq = ~(xx | (xx >> 1)) & 0x55555555u;
            int32_t edge = __shfl_up_sync(gm, O[C - 1], 1, LANES);
            if (glane == 0) edge = NEG;
            const int32_t ia = i0 - glane * C, jb = j0 + glane * C;
            const bool masked = (ia + W - 1 > m) || (jb > n);
            int32_t lmax;
            if (masked)
                lmax = dp_step<LANES, C, false, true>(E, O, edge, eq, sc, thr, i0, j0, m, n);
            else
                lmax = dp_step<LANES, C, false, false>(E, O, edge, eq, sc, thr, i0, j0, m, n);
            if (finish_diag(E, lmax, false)) break;
        }
    }
    best = T;
    best_i = bi;
    best_j = bj;
    cells_out = cells;
    return status;
}

// ---------------------------------------------------------------------------
// Kernels of one band tier.
// ---------------------------------------------------------------------------

// One task per group; tasks order[0..n) (identity if order is null).
template <int LANES, int C, bool COUNT>
__global__ void __launch_bounds__(256)
window_kernel(const Job *jp, uint32_t task_base, uint32_t n_tasks, Spill spill)
{
    const Job J = *jp;
    const int lane = threadIdx.x & 31;
    const int glane = lane % LANES;
    const int gbase = lane - glane;
    const uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
    if (g >= n_tasks) return;
    const uint32_t task = task_base + (uint32_t)g;
    Ext e = decode(J, task);
    if (!e.ok) return;
    int32_t sc, bi, bj;
    int64_t cells;
    int st = extend_window<LANES, C, COUNT>(e, J.sc, glane, gbase, sc, bi, bj, cells);
    if (st) {
        if (glane == 0) {
            uint32_t q = atomicAdd(spill.count, 1u);
            spill.list[q] = task;
        }
        return;
    }
    if (glane == 0) {
        if (COUNT) J.cells[task] = cells;
        else write_result(J, e, sc, bi, bj);
    }
}

// Persistent form: groups pull positions of `order` from a global counter
// until *n_tasks_ptr is reached (order is longest-first in batched mode).
template <int LANES, int C>
__global__ void __launch_bounds__(256)
window_persistent_kernel(const Job *jp, const uint32_t *order, const uint32_t *n_tasks_ptr,
                         uint32_t *counter, Spill spill)
{
    const Job J = *jp;
    const int lane = threadIdx.x & 31;
    const int glane = lane % LANES;
    const int gbase = lane - glane;
    const unsigned gm = group_mask<LANES>(gbase);
    const uint32_t n_tasks = *n_tasks_ptr;
    for (;;) {
        uint32_t q = 0;
        if (glane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(gm, q, gbase);
        if (q >= n_tasks) break;
        const uint32_t task = order ? order[q] : q;
        Ext e = decode(J, task);
        if (!e.ok) continue;
        int32_t sc, bi, bj;
        int64_t cells;
        int st = extend_window<LANES, C, false>(e, J.sc, glane, gbase, sc, bi, bj, cells);
        if (glane == 0) {
            if (st) {
                uint32_t s = atomicAdd(spill.count, 1u);
                spill.list[s] = task;
            } else {
                write_result(J, e, sc, bi, bj);
            }
        }
    }
}

// Window kernels take their task list from a spill of the previous tier.
template <int LANES, int C, bool COUNT>
__global__ void __launch_bounds__(256)
window_spill_kernel(const Job *jp, Spill in, Spill out)
{
    const Job J = *jp;
    const int lane = threadIdx.x & 31;
    const int glane = lane % LANES;
    const int gbase = lane - glane;
    const uint32_t n = *in.count;
    const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / LANES;
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES; g < n;
         g += groups) {
        const uint32_t task = in.list[g];
        Ext e = decode(J, task);
        if (!e.ok) continue;
        int32_t sc, bi, bj;
        int64_t cells;
        int st = extend_window<LANES, C, COUNT>(e, J.sc, glane, gbase, sc, bi, bj, cells);
        if (glane == 0) {
            if (st) {
                uint32_t s = atomicAdd(out.count, 1u);
                out.list[s] = task;
            } else if (COUNT) {
                J.cells[task] = cells;
            } else {
                write_result(J, e, sc, bi, bj);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Lockstep band kernel: 32/L extensions per warp that step their
// anti-diagonals together.
//
// Groups of a warp stay convergent: every per-group decision is either
// predicated (best-cell update, termination) or taken under a warp-wide
// vote (masked cells near the rectangle's far edges, window shifts, base
// refills, task switches), so the warp never splits into groups that issue
// separately.  New tasks start only at the top of an odd diagonal, so all
// groups share the diagonal parity.  The lane maximum runs over packed keys
// value*16 + (15 - t): the group maximum of the keys gives both the best
// value and, with one ballot, the first (smallest i) cell holding it.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t ld_word_u(const uint32_t *pk, int64_t nw, int64_t w)
{
    w = w < 0 ? 0 : (w >= nw ? nw - 1 : w);
    return __ldg(pk + w);
}

__device__ __forceinline__ uint32_t load16_u(const uint32_t *pk, int64_t nw, int64_t q)
{
    const int64_t w = q >> 4;
    const uint32_t sh = (uint32_t)(q & 15) * 2u;
    return __funnelshift_r(ld_word_u(pk, nw, w), ld_word_u(pk, nw, w + 1), sh);
}

// field u = c_{k+u} of the stream c_k = base s0 + dir*(k-1)
__device__ __forceinline__ uint32_t fwd16_u(const uint32_t *pk, int64_t nw, int64_t s0, int dir,
                                            int32_t k)
{
    if (dir > 0) return load16_u(pk, nw, s0 + (k - 1));
    return rev16(load16_u(pk, nw, s0 - (k - 1) - 15));
}

// field t = c_{k-t}
__device__ __forceinline__ uint32_t back16_u(const uint32_t *pk, int64_t nw, int64_t s0, int dir,
                                             int32_t k)
{
    if (dir > 0) return rev16(load16_u(pk, nw, s0 + (k - 16)));
    return load16_u(pk, nw, s0 - (k - 1));
}

template <int C, bool ODD, bool MASKED>
__device__ __forceinline__ int32_t dp_step_key(int32_t (&V)[C], const int32_t (&U)[C],
                                               int32_t edge, uint32_t eq, const Scoring &sc,
                                               int32_t thr, int32_t i0, int32_t j0, int32_t m,
                                               int32_t n)
{
    int32_t lkey = NEG * 16;
#pragma unroll
    for (int t = 0; t < C; ++t) {
        int32_t nb;
        if (ODD) nb = imax(U[t], (t + 1 < C) ? U[t + 1] : edge);
        else nb = imax((t > 0) ? U[t - 1] : edge, U[t]);
        const int32_t s = ((eq >> (2 * t)) & 1u) ? sc.match : sc.mismatch;
        int32_t r = imax(V[t] + s, nb + sc.gap);
        if (MASKED) {
            if (i0 + t > m || j0 - t > n) r = NEG;
        }
        r = (r >= thr) ? r : NEG;
        V[t] = r;
        lkey = imax(lkey, r * 16 + (15 - t));
    }
    return lkey;
}

// Result of one finished task (written by the group leader).
__device__ __forceinline__ void store_result(const Job &J, uint32_t task, int32_t T, int32_t bi,
                                             int32_t bj)
{
    const Pair p = J.pairs[task >> 1];
    int32_t *o = J.out + (size_t)(task >> 1) * 7;
    if (task & 1u) {
        o[3] = T;
        o[4] = (int32_t)(p.seed_a + p.seed_len) + bi;
        o[5] = (int32_t)(p.seed_b + p.seed_len) + bj;
    } else {
        o[0] = T;
        o[1] = (int32_t)p.seed_a - bi;
        o[2] = (int32_t)p.seed_b - bj;
    }
}

// Serving rewrites a slot's Job and pair buffer between requests while the
// persistent kernel runs, so those reads must not be served from an SM's
// L1: load them at L2 (ld.global.cg).
__device__ __forceinline__ Job ldcg_job(const Job *gj)
{
    static_assert(sizeof(Job) % 8 == 0, "Job layout");
    Job J;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(gj);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&J);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(Job) / 8); ++k) dst[k] = __ldcg(src + k);
    return J;
}

__device__ __forceinline__ Pair ldcg_pair(const Pair *p)
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(p);
    return Pair{__ldcg(w), __ldcg(w + 1), __ldcg(w + 2), __ldcg(w + 3), __ldcg(w + 4)};
}

// decode() / store_result() for a serving Job (L2 loads of the request's data).
__device__ __forceinline__ Ext decode_cg(const Job &J, uint32_t task)
{
    Job K = J;
    Pair p = ldcg_pair(&J.pairs[task >> 1]);
    // decode() reads the pair through K.pairs; hand it a one-record view.
    K.pairs = &p;
    Ext e = decode(K, (task & 1u));
    e.pair = task >> 1;
    return e;
}

__device__ __forceinline__ void store_result_cg(const Job &J, uint32_t task, int32_t T,
                                                int32_t bi, int32_t bj)
{
    const Pair p = ldcg_pair(&J.pairs[task >> 1]);
    int32_t *o = J.out + (size_t)(task >> 1) * 7;
    if (task & 1u) {
        o[3] = T;
        o[4] = (int32_t)(p.seed_a + p.seed_len) + bi;
        o[5] = (int32_t)(p.seed_b + p.seed_len) + bj;
    } else {
        o[0] = T;
        o[1] = (int32_t)p.seed_a - bi;
        o[2] = (int32_t)p.seed_b - bj;
    }
}

// Task source of the batched form: positions of a longest-first order
// array pulled from a global counter; overflowing tasks go to a spill list.
struct BatchSrc {
    static constexpr bool kCanAbort = false;  // teardown may stop the loop
    const Job *jp;
    const uint32_t *order;
    uint32_t n_tasks;
    uint32_t *counter;
    Spill spill;

    // Warp-level fetch, executed by every lane: the leaders of the groups
    // that need a task are the set bits of needm.  Returns, for this lane's
    // group, 1 (task), 0 (nothing yet) or -1 (no more tasks).
    __device__ __forceinline__ int fetch_warp(unsigned needm, int lane, int gbase, unsigned gm,
                                              bool need, uint32_t &task, const Job *&gj)
    {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(counter, (uint32_t)__popc(needm));
        base = __shfl_sync(FULL, base, 0);
        if (!need) return 0;
        const uint32_t q = base + (uint32_t)__popc(needm & ((1u << gbase) - 1u));
        if (q >= n_tasks) return -1;
        task = order ? order[q] : q;
        gj = jp;
        return 1;
    }
    __device__ __forceinline__ void idle() {}
    __device__ __forceinline__ bool aborted() const { return false; }
    __device__ __forceinline__ Ext open(const Job *gj, uint32_t task, Scoring &sc)
    {
        sc = gj->sc;
        return decode(*gj, task);
    }
    // called by the group leader only
    __device__ __forceinline__ void retire(const Job *gj, uint32_t task, bool overflow, int32_t T,
                                           int32_t bi, int32_t bj)
    {
        if (overflow) {
            const uint32_t q = atomicAdd(spill.count, 1u);
            spill.list[q] = task;
        } else {
            store_result(*gj, task, T, bi, bj);
        }
    }
};

template <int L, int C, class Src>
__device__ __forceinline__ void lockstep_loop(Src &src, const uint32_t *pk, int64_t nw)
{
    static_assert(C <= 16 && 32 % L == 0, "tile shape");
    constexpr int W = L * C;
    const int lane = threadIdx.x & 31;
    const int glane = lane % L;
    const int gbase = lane - glane;
    const unsigned gm = group_mask<L>(gbase);

    // Per-group task state (uniform within a group).
    bool active = false, exhausted = false;
    uint32_t task = 0;
    const Job *gj = nullptr;
    Scoring sc{1, -1, -1, 0};
    int64_t sa0 = 0, sb0 = 0;  // stream anchors of a and b
    int dir = 1;
    int32_t m = 0, n = 0, d = 0, i0 = 0, j0 = 0, T = 0, bi = 0, bj = 0;
    bool prev_dead = false;
    int32_t E[C], O[C];
#pragma unroll
    for (int t = 0; t < C; ++t) { E[t] = NEG; O[t] = NEG; }
    uint32_t Aw = 0, LA = 0, Bw = 0, LB = 0;
    int la_n = 16, lb_n = 16;  // warp-uniform lookahead counters

    // End of a task: result (or hand-off to the next tier) by the leader.
    auto retire = [&](bool overflow) {
        if (glane == 0) src.retire(gj, task, overflow, T, bi, bj);
        active = false;
    };

    // Bookkeeping after diagonal d (V holds it, U the other parity).
    auto finish = [&](int32_t (&V)[C], int32_t lkey, const bool odd) {
        // The key orders cells within a lane only: take the lowest lane
        // whose maximum is M, then that lane's first cell holding it.
        const int32_t mkey = lockstep_group_max<L>(lkey);
        const int32_t M = mkey >> 4;
        const unsigned hits = __ballot_sync(FULL, (lkey >> 4) == M) & gm;
        const int src_lane = __ffs(hits) - 1;
        const int32_t skey = __shfl_sync(FULL, lkey, src_lane);
        if (active && M > T) {
            bi = (i0 - glane * C) + (src_lane - gbase) * C + (15 - (skey & 15));
            bj = d - bi;
            T = M;
        }
        const bool dead = (M == NEG);
        bool fin = active && ((dead && prev_dead) || d >= m + n);
        prev_dead = dead;
        // Window edges: after an odd diagonal the top slot may seed a cell
        // above the window, after an even one the bottom slot one below it.
        const int32_t vedge = odd ? __shfl_sync(FULL, V[C - 1], L - 1, L)
                                  : __shfl_sync(FULL, V[0], 0, L);
        const bool want = active && !fin && vedge != NEG;
        bool ovf = false;
        if (__any_sync(FULL, want)) {
            const int32_t vopp = odd ? __shfl_sync(FULL, V[0], 0, L)
                                     : __shfl_sync(FULL, V[C - 1], L - 1, L);
            ovf = want && vopp != NEG;
            const bool sh = want && !ovf;
            if (odd) {  // shift up: slot s takes slot s+1
                int32_t ne = __shfl_down_sync(FULL, E[0], 1, L);
                int32_t no = __shfl_down_sync(FULL, O[0], 1, L);
                if (glane == L - 1) { ne = NEG; no = NEG; }
                if (sh) {
#pragma unroll
                    for (int t = 0; t < C - 1; ++t) { E[t] = E[t + 1]; O[t] = O[t + 1]; }
                    E[C - 1] = ne;
                    O[C - 1] = no;
                    i0 += 1;
                    j0 -= 1;
                }
            } else {    // shift down: slot s takes slot s-1
                int32_t pe = __shfl_up_sync(FULL, E[C - 1], 1, L);
                int32_t po = __shfl_up_sync(FULL, O[C - 1], 1, L);
                if (glane == 0) { pe = NEG; po = NEG; }
                if (sh) {
#pragma unroll
                    for (int t = C - 1; t > 0; --t) { E[t] = E[t - 1]; O[t] = O[t - 1]; }
                    E[0] = pe;
                    O[0] = po;
                    i0 -= 1;
                    j0 += 1;
                }
            }
            if (sh) {
                Aw = fwd16_u(pk, nw, sa0, dir, i0);
                LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
                Bw = back16_u(pk, nw, sb0, dir, j0);
                LB = back16_u(pk, nw, sb0, dir, j0 + 16);
            }
            fin = fin || ovf;
        }
        if (fin) retire(ovf);
    };

    unsigned turn = 0;
    for (;;) {
        // A serving kernel can be told to leave at once (teardown).
        if ((++turn & 255u) == 0 && __any_sync(FULL, src.aborted())) break;
        // ---------------- task switches (top of an odd diagonal) ----------------
        const bool need = !active && !exhausted;
        const unsigned needm = __ballot_sync(FULL, need && glane == 0);
        if (needm) {
            const int r = src.fetch_warp(needm, lane, gbase, gm, need, task, gj);
            if (need) {
                if (r < 0) {
                    exhausted = true;
                } else if (r > 0) {
                    const Ext e = src.open(gj, task, sc);
                    if (e.ok) {
                        sa0 = e.A.s0;
                        sb0 = e.B.s0;
                        dir = e.A.dir;
                        m = e.m;
                        n = e.n;
#pragma unroll
                        for (int t = 0; t < C; ++t) {
                            E[t] = (glane * C + t == W / 2) ? 0 : NEG;  // origin at k = 0
                            O[t] = NEG;
                        }
                        i0 = -(W / 2) + glane * C;
                        j0 = (W / 2) - glane * C;
                        Aw = fwd16_u(pk, nw, sa0, dir, i0);
                        LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
                        Bw = back16_u(pk, nw, sb0, dir, j0);
                        LB = back16_u(pk, nw, sb0, dir, j0 + 16);
                        d = 0;
                        T = 0;
                        bi = 0;
                        bj = 0;
                        prev_dead = false;
                        active = true;
                    }
                }
            }
        }
        if (__all_sync(FULL, exhausted && !active)) break;
        if (!__any_sync(FULL, active)) {
            src.idle();
            continue;
        }

        // ---------------- odd diagonal: a-window advances ----------------
        ++d;
        ++i0;
        Aw = __funnelshift_r(Aw, LA, 2);
        LA >>= 2;
        if (--la_n == 0) {
            LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
            la_n = 16;
        }
        {
            const int32_t thr = T - sc.x;
            const uint32_t xx = Aw ^ Bw;
            const uint32_t eq = ~(xx | (xx >> 1)) & 0x55555555u;
            int32_t edge = __shfl_down_sync(FULL, E[0], 1, L);
            if (glane == L - 1) edge = NEG;
            const bool nm = active && ((i0 - glane * C + W - 1 > m) || (j0 + glane * C > n));
            int32_t lkey;
            if (__any_sync(FULL, nm))
                lkey = dp_step_key<C, true, true>(O, E, edge, eq, sc, thr, i0, j0, m, n);
            else
                lkey = dp_step_key<C, true, false>(O, E, edge, eq, sc, thr, i0, j0, m, n);
            finish(O, lkey, true);
        }
        // ---------------- even diagonal: b-window advances ----------------
        ++d;
        ++j0;
        Bw = __funnelshift_l(LB, Bw, 2);
        LB <<= 2;
        if (--lb_n == 0) {
            LB = back16_u(pk, nw, sb0, dir, j0 + 16);
            lb_n = 16;
        }
        {
            const int32_t thr = T - sc.x;
            const uint32_t xx = Aw ^ Bw;
            const uint32_t eq = ~(xx | (xx >> 1)) & 0x55555555u;
            int32_t edge = __shfl_up_sync(FULL, O[C - 1], 1, L);
            if (glane == 0) edge = NEG;
            const bool nm = active && ((i0 - glane * C + W - 1 > m) || (j0 + glane * C > n));
            int32_t lkey;
            if (__any_sync(FULL, nm))
                lkey = dp_step_key<C, false, true>(E, O, edge, eq, sc, thr, i0, j0, m, n);
            else
                lkey = dp_step_key<C, false, false>(E, O, edge, eq, sc, thr, i0, j0, m, n);
            finish(E, lkey, false);
        }
    }
}

template <int L, int C>
__global__ void __launch_bounds__(256)
lockstep_kernel(const Job *jp, const uint32_t *order, const uint32_t *n_tasks_ptr,
                uint32_t *counter, Spill spill)
{
    BatchSrc src{jp, order, *n_tasks_ptr, counter, spill};
    lockstep_loop<L, C>(src, jp->packed, jp->n_words);
}

// ---------------------------------------------------------------------------
// Unbounded tier: one CTA per extension, step-4 ranges, global scratch.
// ---------------------------------------------------------------------------
constexpr int WIDE_THREADS = 256;

__device__ __forceinline__ uint32_t base_at(const Seq &S, int32_t k)
{
    int64_t q = S.s0 + (int64_t)S.dir * (k - 1);
    uint32_t w = ld_word(S, q >> 4);
    return (w >> (2 * (uint32_t)(q & 15))) & 3u;
}

struct WideRed {
    unsigned long long key;  // (value + 2^31) << 32 | ~i : max = best, first i
    int32_t lo, hi;          // live extent
};

__device__ __forceinline__ unsigned long long wide_key(int32_t v, int32_t i)
{
    return ((unsigned long long)(uint32_t)(v + 0x80000000u) << 32) | (uint32_t)(~(uint32_t)i);
}

// Extends one task with the whole CTA; diag points at 3*(m+1) int32.
template <bool COUNT>
__device__ void extend_wide(const Ext &e, const Scoring sc, int32_t *diag,
                            int32_t &best, int32_t &best_i, int32_t &best_j,
                            int64_t &cells_out)
{
    __shared__ WideRed red[WIDE_THREADS / 32];
    __shared__ WideRed tot;
    const int32_t m = e.m, n = e.n;
    int32_t *D[3] = {diag, diag + (m + 1), diag + 2 * (m + 1)};
    // D[c1]: diagonal d-1, D[c2]: d-2, D[c0]: d
    int c0 = 0, c1 = 1, c2 = 2;
    if (threadIdx.x == 0) D[c1][0] = 0;
    int32_t r1lo = 0, r1hi = 0, l1lo = 0, l1hi = 0;   // range / live extent of d-1
    int32_t r2lo = 1, r2hi = 0, l2lo = 1, l2hi = 0;   // of d-2 (none)
    int32_t T = 0, bi = 0, bj = 0;
    int64_t cells = 1;
    bool prev_dead = false;
    __syncthreads();
    for (int32_t d = 1; d <= m + n; ++d) {
        int32_t lo = 0x7fffffff, hi = -0x7fffffff;
        if (l1lo <= l1hi) { lo = min(lo, l1lo); hi = max(hi, l1hi + 1); }
        if (l2lo <= l2hi) { lo = min(lo, l2lo + 1); hi = max(hi, l2hi + 1); }
        lo = max(lo, max(0, d - n));
        hi = min(hi, min(m, d));
        if (hi >= lo) cells += hi - lo + 1;
        const int32_t thr = T - sc.x;
        unsigned long long key = 0;
        int32_t llo = 0x7fffffff, lhi = -0x7fffffff;
        for (int32_t i = lo + (int32_t)threadIdx.x; i <= hi; i += WIDE_THREADS) {
            const int32_t j = d - i;
            int32_t r = NEG;
            bool have = false;
            if (i >= 1 && j >= 1 && i - 1 >= r2lo && i - 1 <= r2hi && D[c2][i - 1] != NEG) {
                int32_t s = (base_at(e.A, i) == base_at(e.B, j)) ? sc.match : sc.mismatch;
                r = D[c2][i - 1] + s;
                have = true;
            }
            if (i >= 1 && i - 1 >= r1lo && i - 1 <= r1hi && D[c1][i - 1] != NEG) {
                int32_t t = D[c1][i - 1] + sc.gap;
                r = have ? imax(r, t) : t;
                have = true;
            }
            if (j >= 1 && i >= r1lo && i <= r1hi && D[c1][i] != NEG) {
                int32_t t = D[c1][i] + sc.gap;
                r = have ? imax(r, t) : t;
                have = true;
            }
            const bool live = have && r >= thr;
            D[c0][i] = live ? r : NEG;
            if (live) {
                unsigned long long k2 = wide_key(r, i);
                key = k2 > key ? k2 : key;
                llo = min(llo, i);
                lhi = max(lhi, i);
            }
        }
        // CTA reduction
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long ok = __shfl_xor_sync(FULL, key, off);
            key = ok > key ? ok : key;
        }
        llo = __reduce_min_sync(FULL, llo);
        lhi = __reduce_max_sync(FULL, lhi);
        const int wid = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) red[wid] = WideRed{key, llo, lhi};
        __syncthreads();
        if (threadIdx.x == 0) {
            WideRed t = red[0];
            for (int w = 1; w < WIDE_THREADS / 32; ++w) {
                t.key = red[w].key > t.key ? red[w].key : t.key;
                t.lo = min(t.lo, red[w].lo);
                t.hi = max(t.hi, red[w].hi);
            }
            tot = t;
        }
        __syncthreads();
        const WideRed t = tot;
        const bool dead = t.lo > t.hi;
        if (!dead) {
            const int32_t v = (int32_t)((uint32_t)(t.key >> 32) - 0x80000000u);
            const int32_t iv = (int32_t)(~(uint32_t)(t.key & 0xffffffffu));
            if (v > T) { T = v; bi = iv; bj = d - iv; }
        }
        r2lo = r1lo; r2hi = r1hi; l2lo = l1lo; l2hi = l1hi;
        r1lo = lo; r1hi = hi;
        l1lo = dead ? 1 : t.lo;
        l1hi = dead ? 0 : t.hi;
        int c = c2; c2 = c1; c1 = c0; c0 = c;
        __syncthreads();  // red/tot and D reuse
        if (dead && prev_dead) break;
        prev_dead = dead;
    }
    best = T;
    best_i = bi;
    best_j = bj;
    cells_out = cells;
}

template <bool COUNT>
__global__ void __launch_bounds__(WIDE_THREADS)
wide_kernel(const Job *jp, Spill in, int32_t *scratch, int64_t scratch_per_cta)
{
    const Job J = *jp;
    const uint32_t n = *in.count;
    int32_t *diag = scratch + (int64_t)blockIdx.x * scratch_per_cta;
    for (uint32_t q = blockIdx.x; q < n; q += gridDim.x) {
        const uint32_t task = in.list[q];
        Ext e = decode(J, task);
        if (!e.ok) continue;
        if ((int64_t)3 * (e.m + 1) > scratch_per_cta) continue;  // sized by the host
        int32_t sc, bi, bj;
        int64_t cells;
        extend_wide<COUNT>(e, J.sc, diag, sc, bi, bj, cells);
        if (threadIdx.x == 0) {
            if (COUNT) J.cells[task] = cells;
            else write_result(J, e, sc, bi, bj);
        }
        __syncthreads();
    }
}

}  // namespace xd
