// Packed 16-bit lockstep band kernel: two window slots per 32-bit register.
//
// Same extension, same reading of the X-drop recurrence and the same
// results as lockstep_loop (xd_device.cuh); only the arithmetic changes.
// It is exact whenever the scoring passes packed16_ok():
//   match - gap <= 128, mismatch >= -128, x + match <= 1536.
//
// Normalised scores.  A cell on anti-diagonal d holds
//   r = H + x + d*|gap| - B          (B: multiples of kRebase taken off)
// stored as 16*r.  Then the two gap predecessors enter unchanged and the
// diagonal one with s + 2|gap|:
//   r(d) = max(r_diag(d-2) + s + 2|gap|,  r_up(d-1),  r_left(d-1)),
// one DPX max and one DPX add-max per register (two cells).  The
// threshold of diagonal d (T of d-1 minus x) becomes thr = T + d*|gap| - B,
// a cell is live iff r >= thr, and r - thr <= x + match.
//
// Key.  One more DPX add-max gives each slot's key
//   16*(r - thr) + (S-1-slot), floored at -16,
// which is negative exactly for the cells the X-drop test prunes (their
// stored value becomes kDead by the key's sign mask) and, for live cells,
// orders by value and then by lowest slot.  The lane's best key becomes
// (key >> 4) * 512 + (31 - lane) * 16 + (key & 15) in 32 bits, so one
// group max gives the largest value and, among equal values, the lowest
// window slot: the first cell in order of increasing i on the diagonal.
//
// Layout.  Lane g of a group of L lanes holds the window slots g*S .. g*S+S-1
// (S = 2*C2 slots).  Register t holds slot t in its low half and slot t+C2
// in its high half, so the neighbour slot s+1 (s-1) of every slot in
// register t sits in register t+1 (t-1) at the same half; only the end
// registers need a byte permute and one shuffle per diagonal.
//
// Ranges, in units of r (no 16-bit wrap anywhere, all values times 16 below
// 2^15): the frame is rebased by kRebase = 256 once thr would reach it, and
// thr grows by at most 2*(match+|gap|) <= 256 per diagonal pair, so thr
// stays in [0, 512); live values stay at or below 511 + x + match <= 2047
// and at or above -256 right after a rebase; dead slots hold -512, and a
// value built from dead predecessors stays at or below -512 + match +
// 2|gap| <= -256 < thr; the lowest value formed is above -640 and the
// lowest key sum above -18432.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "xd_device.cuh"

namespace xd {

namespace p16 {

constexpr int32_t kScale = 16;            // stored value = 16 * r
constexpr int32_t kDead = -512 * kScale;  // stored value of a pruned slot
constexpr uint32_t kDead2 = 0xE000E000u;  // kDead in both halves
constexpr int32_t kRebase = 256;          // frame step, in units of r

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

__device__ __forceinline__ uint32_t pack2(int32_t v) { return ((uint32_t)v & 0xFFFFu) * 0x10001u; }

// Byte-permute selector giving 0xFFFF in the low half where slot t's match
// bit is set and likewise in the high half for slot t+C2.  Match bits sit
// at the msb of byte (s >> 2) of R[s & 3] (see dp16); msb-replicating
// selectors (8 | byte) turn them into half-word masks.
template <int C2>
__host__ __device__ constexpr uint32_t mask_sel(int t)
{
    return (uint32_t)((8 | (t >> 2)) | ((8 | (t >> 2)) << 4) | ((8 | ((t + C2) >> 2)) << 8) |
                      ((8 | ((t + C2) >> 2)) << 12));
}

template <int C2>
__host__ __device__ constexpr uint32_t idx2(int t)
{
    return (uint32_t)(2 * C2 - 1 - t) | ((uint32_t)(2 * C2 - 1 - (t + C2)) << 16);
}

// Lane slots of register t (low: t, high: t + C2) and their negations.
template <int C2>
__host__ __device__ constexpr uint32_t slot2(int t)
{
    return (uint32_t)t | ((uint32_t)(t + C2) << 16);
}
template <int C2>
__host__ __device__ constexpr uint32_t nslot2(int t)
{
    return ((uint32_t)(-t) & 0xFFFFu) | (((uint32_t)(-(t + C2)) & 0xFFFFu) << 16);
}

template <int N>
__device__ __forceinline__ uint32_t tree_max2(const uint32_t (&k)[N])
{
    if constexpr (N == 1) {
        return k[0];
    } else if constexpr (N == 2) {
        return __vmaxs2(k[0], k[1]);
    } else {
        constexpr int M = (N + 2) / 3;
        uint32_t r[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (3 * i + 2 < N) r[i] = __vimax3_s16x2(k[3 * i], k[3 * i + 1], k[3 * i + 2]);
            else if (3 * i + 1 < N) r[i] = __vmaxs2(k[3 * i], k[3 * i + 1]);
            else r[i] = k[3 * i];
        }
        return tree_max2<M>(r);
    }
}

// One anti-diagonal for one lane: V (diagonal d-2, overwritten with d) and
// U (d-1).  edge: the neighbouring lane's end register of U (next lane's
// register 0 on odd diagonals, previous lane's register C2-1 on even ones).
// Returns the lane's 16-bit key, sign-extended.
template <int C2, bool ODD, bool MASKED>
__device__ __forceinline__ int32_t dp16(uint32_t (&V)[C2], const uint32_t (&U)[C2],
                                        uint32_t edge, uint32_t eq, uint32_t ma2, uint32_t mi2,
                                        uint32_t nthr2, uint32_t lo1_2, uint32_t nhi1_2)
{
    const uint32_t R[4] = {eq << 7, eq << 5, eq << 3, eq << 1};
    uint32_t key[C2];
#pragma unroll
    for (int t = 0; t < C2; ++t) {
        uint32_t sh;
        if (ODD) sh = (t + 1 < C2) ? U[t + 1] : prmt(U[0], edge, 0x5432);
        else sh = (t > 0) ? U[t - 1] : prmt(edge, U[C2 - 1], 0x5432);
        const uint32_t nb = __vmaxs2(U[t], sh);
        const uint32_t mk = prmt(R[t & 3], R[t & 3], mask_sel<C2>(t));
        const uint32_t s2 = (mk & ma2) | (~mk & mi2);
        uint32_t r = __viaddmax_s16x2(V[t], s2, nb);
        if (MASKED) {
            // slot s lies in the rectangle iff lo <= s <= hi (lo = j0 - n,
            // hi = m - i0): max(s - hi - 1, lo - 1 - s) < 0, per half
            const uint32_t c = __viaddmax_s16x2(nslot2<C2>(t), lo1_2, 0x80008000u);
            const uint32_t u = __viaddmax_s16x2(slot2<C2>(t), nhi1_2, c);
            const uint32_t in = prmt(u, u, 0xBB99);  // 0xFFFF where inside
            r = (r & in) | (kDead2 & ~in);
        }
        // 16*(r - thr) + (S-1-slot), floored at -16: negative iff pruned
        const uint32_t kc = __viaddmax_s16x2(idx2<C2>(t), nthr2, 0x80008000u);
        const uint32_t k = __viaddmax_s16x2(r, kc, 0xFFF0FFF0u);
        const uint32_t pm = prmt(k, k, 0xBB99);  // 0xFFFF where pruned
        V[t] = (r & ~pm) | (kDead2 & pm);
        key[t] = k;
    }
    const uint32_t kk = tree_max2<C2>(key);
    const int32_t hi = (int32_t)kk >> 16;
    const int32_t lo = (int32_t)prmt(kk, 0u, 0x9910);  // sign-extended low half
    return hi > lo ? hi : lo;
}

}  // namespace p16

__host__ __device__ inline bool packed16_ok(const Scoring &sc)
{
    return sc.match - sc.gap <= 128 && sc.mismatch >= -128 && sc.x >= 0 &&
           sc.x + sc.match <= 1536;
}

template <int L, int C2, class Src>
__device__ __forceinline__ void lockstep16_loop(Src &src, const uint32_t *pk, int64_t nw)
{
    using namespace p16;
    constexpr int S = 2 * C2;  // slots per lane
    constexpr int W = L * S;
    static_assert(S <= 16 && 32 % L == 0 && C2 % 4 == 0, "packed tile shape");
    const int lane = threadIdx.x & 31;
    const int glane = lane % L;
    const int gbase = lane - glane;
    const unsigned gm = group_mask<L>(gbase);

    // Per-group task state (uniform within a group).
    bool active = false, exhausted = false;
    uint32_t task = 0;
    const Job *gj = nullptr;
    Scoring sc{1, -1, -1, 0};
    int64_t sa0 = 0, sb0 = 0;
    int dir = 1;
    int32_t m = 0, n = 0, d = 0, i0 = 0, j0 = 0, T = 0, bi = 0, bj = 0;
    int32_t Q = 0;              // frame offset: thr = T + Q
    int32_t bkey = 0, bbase = 0, bd = 0;  // best cell: group key, window base i, diagonal
    int32_t ng = 1;             // |gap|
    uint32_t ma2 = 0, mi2 = 0;  // packed match / mismatch + 2|gap|
    bool prev_dead = false, fin = false, want = false;
    uint32_t E[C2], O[C2];
#pragma unroll
    for (int t = 0; t < C2; ++t) { E[t] = kDead2; O[t] = kDead2; }
    uint32_t Aw = 0, LA = 0, Bw = 0, LB = 0;
    int la_n = 16, lb_n = 16;  // warp-uniform lookahead counters
    int32_t budget = 0;        // warp-uniform: half-steps known to stay inside every rectangle
    const int32_t lane_bits = (31 - glane) << 4;
    const uint32_t dead16 = (uint32_t)kDead & 0xFFFFu;

    auto retire = [&](bool overflow) {
        if (bd > 0) {
            bi = bbase + (31 - ((bkey >> 4) & 31)) * S + (S - 1 - (bkey & 15));
            bj = bd - bi;
        }
        if (glane == 0) src.retire(gj, task, overflow, T, bi, bj);
        active = false;
        ng = 0;  // the frame offset stays put while the group waits
    };

    // Half-steps until a cell of this group's window can leave the
    // rectangle: each half-step moves the top slot's i or the bottom
    // slot's j up by one (window shifts recompute it).
    auto refresh_budget = [&]() {
        const int32_t mg = min(m - (i0 - glane * S + W - 1), n - (j0 + glane * S));
        budget = __reduce_min_sync(FULL, active ? mg : INT32_MAX);
    };

    // One anti-diagonal.  Returns the warp-wide "something to do" vote:
    // a window edge went live, a task ended, a lookahead word ran out, the
    // frame needs a rebase, the masking-free budget ran low, or a group
    // waits for a task.  Everything else is straight-line code.
    auto half = [&](auto odd_tag, auto masked_tag) -> bool {
        constexpr bool ODD = decltype(odd_tag)::value;
        constexpr bool MASKED = decltype(masked_tag)::value;
        ++d;
        Q += ng;
        --budget;
        if (ODD) {
            ++i0;
            Aw = __funnelshift_r(Aw, LA, 2);
            LA >>= 2;
            --la_n;
        } else {
            ++j0;
            Bw = __funnelshift_l(LB, Bw, 2);
            LB <<= 2;
            --lb_n;
        }
        const uint32_t nthr2 = pack2(-kScale * (T + Q));
        // rectangle bounds of this lane's slots, clamped into 16 bits (only
        // the masked copy reads them)
        uint32_t lo1_2 = 0, nhi1_2 = 0;
        if (MASKED) {
            const int32_t lo = j0 - n, hi = m - i0;
            lo1_2 = pack2(min(max(lo - 1, -1024), 1024));
            nhi1_2 = pack2(min(max(-hi - 1, -1024), 1024));
        }
        const uint32_t xx = Aw ^ Bw;
        const uint32_t eq = ~(xx | (xx >> 1)) & 0x55555555u;
        int32_t lkey;
        uint32_t vedge;
        if (ODD) {
            uint32_t edge = __shfl_down_sync(FULL, E[0], 1, L);
            if (glane == L - 1) edge = kDead2;
            lkey = dp16<C2, true, MASKED>(O, E, edge, eq, ma2, mi2, nthr2, lo1_2, nhi1_2);
            vedge = __shfl_sync(FULL, O[C2 - 1], L - 1, L) >> 16;
        } else {
            uint32_t edge = __shfl_up_sync(FULL, O[C2 - 1], 1, L);
            if (glane == 0) edge = kDead2;
            lkey = dp16<C2, false, MASKED>(E, O, edge, eq, ma2, mi2, nthr2, lo1_2, nhi1_2);
            vedge = __shfl_sync(FULL, E[0], 0, L) & 0xFFFFu;
        }
        // Group key: value above lane above slot in lane, so one max finds
        // the lowest window slot among the cells holding the maximum.
        const int32_t mkey = __reduce_max_sync(gm, (lkey >> 4) * 512 + ((lkey & 15) | lane_bits));
        const int32_t xm = mkey >> 9;  // best r - thr on the diagonal (-1: none live)
        const bool up = active && xm > sc.x;
        T = up ? T - sc.x + xm : T;
        bkey = up ? mkey : bkey;           // decoded at retire
        bbase = up ? i0 - glane * S : bbase;
        bd = up ? d : bd;
        const bool dead = (mkey < 0);
        fin = active && ((dead && prev_dead) || d >= m + n);
        prev_dead = dead;
        want = active && !fin && vedge != dead16;
        bool ev = want || fin || (ODD ? la_n == 0 : lb_n == 0);
        if (!ODD) {
            ev = ev || (active && T + Q + ng >= kRebase) || !active;
            if (!MASKED) ev = ev || budget < 2;
        }
        return __any_sync(FULL, ev);
    };

    // The rare work behind an event.  After an even diagonal, returns true
    // when the loop must go back to the task switch (a group waits for a
    // task, no group is left running, or the masking-free budget no longer
    // covers a diagonal pair).
    auto handle = [&](const bool odd, const bool masked) -> bool {
        bool ovf = false;
        if (__any_sync(FULL, want)) {
            // After an odd diagonal the top slot may seed a cell above the
            // window, after an even one the bottom slot one below it; with
            // the opposite edge live too the task goes to a wider tier.
            const uint32_t vopp = odd ? __shfl_sync(FULL, O[0], 0, L) & 0xFFFFu
                                      : __shfl_sync(FULL, E[C2 - 1], L - 1, L) >> 16;
            ovf = want && vopp != dead16;
            const bool sh = want && !ovf;
            if (odd) {  // shift up: slot s takes slot s+1
                uint32_t ne = __shfl_down_sync(FULL, E[0], 1, L);
                uint32_t no = __shfl_down_sync(FULL, O[0], 1, L);
                if (glane == L - 1) { ne = kDead2; no = kDead2; }
                if (sh) {
                    const uint32_t te = prmt(E[0], ne, 0x5432), to = prmt(O[0], no, 0x5432);
#pragma unroll
                    for (int t = 0; t < C2 - 1; ++t) { E[t] = E[t + 1]; O[t] = O[t + 1]; }
                    E[C2 - 1] = te;
                    O[C2 - 1] = to;
                    i0 += 1;
                    j0 -= 1;
                }
            } else {    // shift down: slot s takes slot s-1
                uint32_t pe = __shfl_up_sync(FULL, E[C2 - 1], 1, L);
                uint32_t po = __shfl_up_sync(FULL, O[C2 - 1], 1, L);
                if (glane == 0) { pe = kDead2; po = kDead2; }
                if (sh) {
                    const uint32_t te = prmt(pe, E[C2 - 1], 0x5432);
                    const uint32_t to = prmt(po, O[C2 - 1], 0x5432);
#pragma unroll
                    for (int t = C2 - 1; t > 0; --t) { E[t] = E[t - 1]; O[t] = O[t - 1]; }
                    E[0] = te;
                    O[0] = to;
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
        if (la_n == 0) {
            LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
            la_n = 16;
        }
        if (lb_n == 0) {
            LB = back16_u(pk, nw, sb0, dir, j0 + 16);
            lb_n = 16;
        }
        if (odd) {
            if (!masked) refresh_budget();
            return false;
        }
        // Keep thr = T + Q of the next diagonal below 2 * kRebase (see the
        // header comment): rebase once it would reach kRebase.
        const bool rb = active && T + Q + ng >= kRebase;
        if (rb) {
            const uint32_t mr = pack2(-kScale * kRebase);
#pragma unroll
            for (int t = 0; t < C2; ++t) {
                E[t] = __viaddmax_s16x2(E[t], mr, kDead2);
                O[t] = __viaddmax_s16x2(O[t], mr, kDead2);
            }
            Q -= kRebase;
        }
        if (!masked) refresh_budget();
        if constexpr (Src::kCanAbort) {
            if (__any_sync(FULL, src.aborted())) return true;
        }
        return __any_sync(FULL, !active && !exhausted) || !__any_sync(FULL, active) ||
               (!masked && budget < 2);
    };

    using T0 = std::integral_constant<bool, false>;
    using T1 = std::integral_constant<bool, true>;
    for (;;) {
        // A serving kernel can be told to leave at once (teardown).
        if constexpr (Src::kCanAbort) {
            if (__any_sync(FULL, src.aborted())) break;
        }
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
                    if (e.ok && !packed16_ok(sc)) {
                        // A scoring 16-bit cells cannot hold exactly (a serving
                        // request's own): hand the task to the next, 32-bit tier.
                        if (glane == 0) src.retire(gj, task, true, 0, 0, 0);
                    } else if (e.ok) {
                        sa0 = e.A.s0;
                        sb0 = e.B.s0;
                        dir = e.A.dir;
                        m = e.m;
                        n = e.n;
                        ng = -sc.gap;
                        ma2 = pack2(kScale * (sc.match + 2 * ng));
                        mi2 = pack2(kScale * (sc.mismatch + 2 * ng));
                        // origin (H = 0) at window slot W/2, stored as 16 * (0 + x)
#pragma unroll
                        for (int t = 0; t < C2; ++t) {
                            const int slo = glane * S + t, shi = slo + C2;
                            const uint32_t lo = (slo == W / 2) ? (uint32_t)(kScale * sc.x) : dead16;
                            const uint32_t hi = (shi == W / 2) ? (uint32_t)(kScale * sc.x) : dead16;
                            E[t] = lo | (hi << 16);
                            O[t] = kDead2;
                        }
                        i0 = -(W / 2) + glane * S;
                        j0 = (W / 2) - glane * S;
                        Aw = fwd16_u(pk, nw, sa0, dir, i0);
                        LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
                        Bw = back16_u(pk, nw, sb0, dir, j0);
                        LB = back16_u(pk, nw, sb0, dir, j0 + 16);
                        d = 0;
                        T = 0;
                        Q = 0;
                        bi = 0;
                        bj = 0;
                        bd = 0;
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
        refresh_budget();
        if (budget >= 2) {
            for (;;) {  // no cell of any window can leave its rectangle
                if (half(T1{}, T0{})) handle(true, false);
                if (half(T0{}, T0{}) && handle(false, false)) break;
            }
        } else {
            for (;;) {
                if (half(T1{}, T1{})) handle(true, true);
                if (half(T0{}, T1{}) && handle(false, true)) break;
            }
        }
    }
}

// Batched form of the packed kernel (same task source as lockstep_kernel).
template <int L, int C2>
__global__ void __launch_bounds__(256)
lockstep16_kernel(const Job *jp, const uint32_t *order, const uint32_t *n_tasks_ptr,
                  uint32_t *counter, Spill spill)
{
    BatchSrc src{jp, order, *n_tasks_ptr, counter, spill};
    lockstep16_loop<L, C2>(src, jp->packed, jp->n_words);
}

// Serving form: ring warps run the packed tile, the spill warps (one warp
// in kSpillWarpEvery, plus ring warps that help when the second-tier
// backlog grows) the 32-bit tile L2 x C2, which also takes every task
// whose scoring does not fit 16 bits.  Same protocol as serve_kernel.
template <int L1, int C2a, int L2, int C2>
__global__ void __launch_bounds__(256, (L1 * 2 * C2a <= 64) ? 3 : 2)
serve16_kernel(ServeArgs a, const uint32_t *pk, int64_t nw)
{
    const unsigned warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp_global % kSpillWarpEvery == kSpillWarpEvery - 1) {
        SpillSrc src{a, 0, 0, false, false};
        lockstep_loop<L2, C2>(src, pk, nw);
        return;
    }
    for (;;) {
        RingSrc src{a, 0ull, 0, 0, false};
        lockstep16_loop<L1, C2a>(src, pk, nw);
        if (__any_sync(FULL, src.leaving || src.aborted())) break;
        SpillSrc help{a, 0, 0, true, false};
        lockstep_loop<L2, C2>(help, pk, nw);
        if (__any_sync(FULL, help.failed || help.aborted())) break;
    }
    if ((threadIdx.x & 31) == 0) atomicSub(&a.ctl->ring_alive, 1u);
}

}  // namespace xd
