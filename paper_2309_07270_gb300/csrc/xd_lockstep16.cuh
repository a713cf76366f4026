// Packed 16-bit lockstep band kernel: two window slots per 32-bit register.
//
// Same extension, same reading of the X-drop recurrence and the same
// results as lockstep_loop (xd_device.cuh); only the arithmetic changes.
// It is exact whenever the scoring passes packed16_ok():
//   match - gap <= 128, mismatch >= -128, mismatch + 2|gap| >= 0,
//   x + match <= 1536.
//
// Normalised scores.  A cell on anti-diagonal d holds
//   r = H + x + d*|gap| - B          (B: the rebase steps taken off)
// stored as 16*r.  Then the two gap predecessors enter unchanged and the
// diagonal one with s + 2|gap| >= 0:
//   r(d) = max(r_diag(d-2) + s + 2|gap|,  r_up(d-1),  r_left(d-1)),
// one plain 32-bit add (both halves at once, see below) and one DPX
// three-way max per register (two cells).  The threshold of diagonal d
// (T of d-1 minus x) becomes thr = T + d*|gap| - B, a cell is live iff
// r >= thr, and r - thr <= x + match.
//
// Key.  One more 32-bit add and a DPX add-max give each slot's key
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
// Ranges, in units of r, with kR the rebase step of the scoring
// (rebase_step16, between 128 and 1792 inside the range above).  After
// every pair of diagonals (odd d-1, even d) the frame is rebased by kR
// once thr of d-1 reaches kR.  Every live value of d-1 and d is at least
// that threshold, so live values stay >= 0 (>= thr >= 0) at all times and
// pruned ones hold kDead = -256.  thr grows by at most 3|gap| + 2 match
// over the three diagonals between two tests, so thr < kR + 3|gap| +
// 2 match <= 1666 and every live value is at most thr + x + match <= 2047
// (16 times that fits a signed half).  A value built from a pruned
// predecessor stays below -256 + 255 < 0 <= thr.  No value formed is
// below kDead (substitutions are >= 0 here), the lowest key sum is
// 16 kDead/16 - 16 * 1666 > -32768, and a rebase takes kDead to
// kDead - 16 kR >= -32768 before the floor restores it.
//
// Carry-free adds.  V + s2 (stored value plus packed substitution, s2 in
// [0, 16*255]) and idx + (-16 thr) (idx <= 15 < 16 thr unless thr = 0) are
// plain 32-bit adds: the low halves, read unsigned, never reach 2^16 (a
// live half is < 2^15 - s2, kDead is 0xF000 and 0xF000 + 0x0FF0 < 2^16),
// so nothing carries into the high half.
//
// Window edges.  Live values are >= 0 and pruned ones negative, so the
// sign bit of a half tells whether that slot is live.  The edges are
// tested once per pair of diagonals, after the even one: no live cell of
// diagonals d+1, d+2 can leave the window unless E's top slot (diagonal d)
// or O's top slot (d-1) is live, or E's bottom slot is.  The window then
// shifts up one slot if E's two bottom slots and O's bottom slot are dead,
// or down one slot if the two top slots of E and of O are dead; otherwise
// the band has outgrown the window and the task goes to a wider tier.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "xd_device.cuh"

namespace xd {

namespace p16 {

constexpr int32_t kScale = 16;            // stored value = 16 * r
constexpr int32_t kDead = -256 * kScale;  // stored value of a pruned slot
constexpr uint32_t kDead2 = 0xF000F000u;  // kDead in both halves

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

__host__ __device__ inline uint32_t pack2(int32_t v) { return ((uint32_t)v & 0xFFFFu) * 0x10001u; }

// a * one + b with one == 1 at run time: the same value as a + b (and as
// a << s for one << s), issued as a multiply-add on the FMA pipe.  Every DPX,
// byte-permute, logic and min/max instruction of the loop issues on the ALU
// pipe, which bounds it; the compiler would issue these adds and shifts there
// too.  `one` is a kernel argument, so the compiler cannot fold the multiply.
__device__ __forceinline__ uint32_t fma_add(uint32_t a, uint32_t one, uint32_t b)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(one), "r"(b));
    return r;
}

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

// A slot is live iff its half is non-negative (pruned slots hold kDead).
__device__ __forceinline__ bool live_lo(uint32_t v) { return (v & 0x8000u) == 0; }
__device__ __forceinline__ bool live_hi(uint32_t v) { return (int32_t)v >= 0; }

// One anti-diagonal for one lane: V (diagonal d-2, overwritten with d) and
// U (d-1).  edge: the neighbouring lane's end register of U (next lane's
// register 0 on odd diagonals, previous lane's register C2-1 on even ones).
// eq7: bit 2s+1 set iff slot s's bases match.  Returns the lane's 16-bit
// key, sign-extended.
template <int C2, bool ODD, bool MASKED>
__device__ __forceinline__ int32_t dp16(uint32_t (&V)[C2], const uint32_t (&U)[C2],
                                        uint32_t edge, uint32_t eq7, uint32_t ma2, uint32_t mi2,
                                        uint32_t nthr2, uint32_t lo1_2, uint32_t nhi1_2,
                                        uint32_t one)
{
    // R[q]: the match bit of slot 4b + q at the msb of byte b
    const uint32_t R[4] = {fma_add(eq7, one << 6, 0u), fma_add(eq7, one << 4, 0u),
                           fma_add(eq7, one << 2, 0u), eq7};
    uint32_t key[C2];
#pragma unroll
    for (int t = 0; t < C2; ++t) {
        uint32_t sh;
        if (ODD) sh = (t + 1 < C2) ? U[t + 1] : prmt(U[0], edge, 0x5432);
        else sh = (t > 0) ? U[t - 1] : prmt(edge, U[C2 - 1], 0x5432);
        const uint32_t mk = prmt(R[t & 3], R[t & 3], mask_sel<C2>(t));
        const uint32_t s2 = (mk & ma2) | (~mk & mi2);
        uint32_t r = __vimax3_s16x2(fma_add(V[t], one, s2), U[t], sh);  // carry-free add (header)
        if (MASKED) {
            // slot s lies in the rectangle iff lo <= s <= hi (lo = j0 - n,
            // hi = m - i0): max(s - hi - 1, lo - 1 - s) < 0, per half
            const uint32_t c = __viaddmax_s16x2(nslot2<C2>(t), lo1_2, 0x80008000u);
            const uint32_t u = __viaddmax_s16x2(slot2<C2>(t), nhi1_2, c);
            const uint32_t in = prmt(u, u, 0xBB99);  // 0xFFFF where inside
            r = (r & in) | (kDead2 & ~in);
        }
        // 16*(r - thr) + (S-1-slot), floored at -16: negative iff pruned
        const uint32_t k = __viaddmax_s16x2(r, fma_add(nthr2, one, idx2<C2>(t)), 0xFFF0FFF0u);
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
    return sc.match - sc.gap <= 128 && sc.mismatch >= -128 && sc.mismatch - 2 * sc.gap >= 0 &&
           sc.x >= 0 && sc.x + sc.match <= 1536;
}

// Frame step of one rebase (units of r) for a scoring that passes
// packed16_ok: at least 128 there (see the header comment's ranges).
__host__ __device__ inline int32_t rebase_step16(const Scoring &sc)
{
    const int32_t ng = -sc.gap;
    int32_t k = 1792;
    k = k < 1667 - 3 * ng - 2 * sc.match ? k : 1667 - 3 * ng - 2 * sc.match;
    k = k < 2048 - sc.x - 3 * sc.match - 3 * ng ? k : 2048 - sc.x - 3 * sc.match - 3 * ng;
    return k;
}

// one: 1 (see fma_add).
template <int L, int C2, class Src>
__device__ __forceinline__ void lockstep16_loop(Src &src, const uint32_t *pk, int64_t nw,
                                                uint32_t one)
{
    using namespace p16;
    constexpr int S = 2 * C2;  // slots per lane
    constexpr int W = L * S;
    static_assert(S <= 16 && 32 % L == 0 && L >= 2 && C2 % 4 == 0, "packed tile shape");
    const int lane = threadIdx.x & 31;
    const int glane = lane % L;
    const int gbase = lane - glane;
    const unsigned gm = group_mask<L>(gbase);
    const bool bot_lane = glane == 0, top_lane = glane == L - 1;

    // Per-group task state (uniform within a group).
    bool active = false, exhausted = false;
    uint32_t task = 0;
    const Job *gj = nullptr;
    Scoring sc{1, -1, -1, 0};
    int64_t sa0 = 0, sb0 = 0;
    int dir = 1;
    int32_t mn = 0, m = 0, n = 0, d = 0, i0 = 0, j0 = 0, T = 0, bi = 0, bj = 0;
    int32_t Q = 0;                      // frame offset: thr = T + Q
    int32_t kR = 0;                     // rebase step
    int32_t xup = 0;                    // (x + 1) * 512: a group key this large raises T
    int32_t bkey = 0, bi0 = 0, bd = 0;  // best cell: group key, this lane's i0, diagonal
    int32_t ng = 1;                     // |gap|
    uint32_t ma2 = 0, mi2 = 0;          // packed 16 * (match / mismatch + 2|gap|)
    bool prev_dead = false, fin = false, rb = false;
    uint32_t E[C2], O[C2];
#pragma unroll
    for (int t = 0; t < C2; ++t) { E[t] = kDead2; O[t] = kDead2; }
    uint32_t Aw = 0, LA = 0, Bw = 0, LB = 0;
    int la_n = 16;        // warp-uniform: diagonal pairs the lookahead words still cover
    int32_t budget = 0;   // warp-uniform: diagonal pairs known to stay inside every rectangle
    const int32_t lane_bits = (31 - glane) << 4;
    const uint32_t dead16 = (uint32_t)kDead & 0xFFFFu;

    auto retire = [&](bool overflow) {
        if (bd > 0) {
            bi = (bi0 - glane * S) + (31 - ((bkey >> 4) & 31)) * S + (S - 1 - (bkey & 15));
            bj = bd - bi;
        }
        if (glane == 0) src.retire(gj, task, overflow, T, bi, bj);
        active = false;
        ng = 0;  // the frame offset stays put while the group waits
    };

    // Diagonal pairs until a cell of this group's window can leave the
    // rectangle: each pair moves the top slot's i and the bottom slot's j
    // up by one (window shifts recompute it).
    auto refresh_budget = [&]() {
        const int32_t mg = min(m - (i0 - glane * S + W - 1), n - (j0 + glane * S));
        budget = __reduce_min_sync(FULL, active ? mg : INT32_MAX);
    };

    // One anti-diagonal and the bookkeeping that cannot wait for the end of
    // the pair: T and the best cell.  Returns the group key (negative iff
    // every cell of the diagonal was pruned) and the diagonal's threshold.
    auto diag = [&](auto odd_tag, auto masked_tag, int32_t &thr) -> int32_t {
        constexpr bool ODD = decltype(odd_tag)::value;
        constexpr bool MASKED = decltype(masked_tag)::value;
        ++d;
        Q += ng;
        if (ODD) {
            ++i0;
            Aw = __funnelshift_r(Aw, LA, 2);
            LA >>= 2;
        } else {
            ++j0;
            Bw = __funnelshift_l(LB, Bw, 2);
            LB <<= 2;
        }
        thr = T + Q;
        const uint32_t nthr2 = prmt((uint32_t)(-kScale * thr), 0u, 0x1010);
        // rectangle bounds of this lane's slots, clamped into 16 bits (only
        // the masked copy reads them)
        uint32_t lo1_2 = 0, nhi1_2 = 0;
        if (MASKED) {
            const int32_t lo = j0 - n, hi = m - i0;
            lo1_2 = pack2(min(max(lo - 1, -1024), 1024));
            nhi1_2 = pack2(min(max(-hi - 1, -1024), 1024));
        }
        const uint32_t xx = Aw ^ Bw;
        const uint32_t eq7 = ~(xx | (xx << 1));
        int32_t lkey;
        if (ODD) {
            uint32_t edge = __shfl_down_sync(FULL, E[0], 1, L);
            if (top_lane) edge = kDead2;
            lkey = dp16<C2, true, MASKED>(O, E, edge, eq7, ma2, mi2, nthr2, lo1_2, nhi1_2, one);
        } else {
            uint32_t edge = __shfl_up_sync(FULL, O[C2 - 1], 1, L);
            if (bot_lane) edge = kDead2;
            lkey = dp16<C2, false, MASKED>(E, O, edge, eq7, ma2, mi2, nthr2, lo1_2, nhi1_2, one);
        }
        // Group key: value above lane above slot in lane, so one max finds
        // the lowest window slot among the cells holding the maximum.
        const int32_t mkey = lockstep_group_max<L>((lkey >> 4) * 512 + ((lkey & 15) | lane_bits));
        if (mkey >= xup) {  // best value - thr > x: T rises (decoded at retire)
            T += (mkey >> 9) - sc.x;
            bkey = mkey;
            bi0 = i0;
            bd = d;
        }
        return mkey;
    };

    // One pair of anti-diagonals (odd, then even).  Returns the warp-wide
    // "something to do" vote: a window edge went live, a task ended, the
    // lookahead words ran out, a frame needs a rebase, the masking-free
    // budget ran out, or a group waits for a task.
    auto pair = [&](auto masked_tag) -> bool {
        constexpr bool MASKED = decltype(masked_tag)::value;
        int32_t thr_o, thr_e;
        const int32_t key_o = diag(std::true_type{}, masked_tag, thr_o);
        const int32_t key_e = diag(std::false_type{}, masked_tag, thr_e);
        const bool dead_o = key_o < 0, dead_e = key_e < 0;
        fin = active && ((dead_o && (prev_dead || dead_e)) || d >= mn);
        prev_dead = dead_e;
        --budget;
        --la_n;
        rb = active && thr_o >= kR;
        // window edges: this group's bottom lane tests E's bottom slot, its
        // top lane the top slots of E and O (sign bit set = pruned)
        const uint32_t ew = top_lane ? (E[C2 - 1] & O[C2 - 1]) : (E[0] << 16);
        const bool edge = active && (bot_lane || top_lane) && (int32_t)ew >= 0;
        bool ev = edge || fin || rb || la_n == 0 || (!active && !exhausted);
        if (!MASKED) ev = ev || budget < 1;
        return __any_sync(FULL, ev);
    };

    // The rare work behind an event, after the even diagonal of a pair.
    // Returns true when the loop must go back to the task switch (a group
    // waits for a task, no group is left running, the masking-free budget
    // no longer covers a pair, or, masked, it covers one again).
    auto handle = [&](const bool masked) -> bool {
        bool ovf = false;
        const bool go = active && !fin;
        const bool need_dn_l = bot_lane && live_lo(E[0]);
        const bool need_up_l = top_lane && (live_hi(E[C2 - 1]) || live_hi(O[C2 - 1]));
        if (__any_sync(FULL, go && (need_dn_l || need_up_l))) {
            // Per group: the decision of its bottom and top lanes.
            const bool blk_up_l = live_lo(E[0]) || live_lo(E[1]) || live_lo(O[0]);
            const bool blk_dn_l = live_hi(E[C2 - 1]) || live_hi(O[C2 - 1]) ||
                                  live_hi(E[C2 - 2]) || live_hi(O[C2 - 2]);
            // every lane takes part in every shuffle (no short-circuit
            // around a warp-wide collective)
            const bool up_g = __shfl_sync(FULL, (int)need_up_l, L - 1, L) != 0;
            const bool dn_g = __shfl_sync(FULL, (int)need_dn_l, 0, L) != 0;
            const bool bu = __shfl_sync(FULL, (int)blk_up_l, 0, L) != 0;
            const bool bdn = __shfl_sync(FULL, (int)blk_dn_l, L - 1, L) != 0;
            const bool nu = go && up_g;
            const bool nd = go && dn_g;
            ovf = (nu && bu) || (!nu && nd && bdn);
            const bool su = nu && !bu;           // shift up: slot s takes slot s+1
            const bool sd = !nu && nd && !bdn;   // shift down: slot s takes slot s-1
            if (__any_sync(FULL, su)) {
                uint32_t ne = __shfl_down_sync(FULL, E[0], 1, L);
                uint32_t no = __shfl_down_sync(FULL, O[0], 1, L);
                if (top_lane) { ne = kDead2; no = kDead2; }
                if (su) {
                    const uint32_t te = prmt(E[0], ne, 0x5432), to = prmt(O[0], no, 0x5432);
#pragma unroll
                    for (int t = 0; t < C2 - 1; ++t) { E[t] = E[t + 1]; O[t] = O[t + 1]; }
                    E[C2 - 1] = te;
                    O[C2 - 1] = to;
                    i0 += 1;
                    j0 -= 1;
                }
            }
            if (__any_sync(FULL, sd)) {
                uint32_t pe = __shfl_up_sync(FULL, E[C2 - 1], 1, L);
                uint32_t po = __shfl_up_sync(FULL, O[C2 - 1], 1, L);
                if (bot_lane) { pe = kDead2; po = kDead2; }
                if (sd) {
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
            if (su || sd) {
                Aw = fwd16_u(pk, nw, sa0, dir, i0);
                LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
                Bw = back16_u(pk, nw, sb0, dir, j0);
                LB = back16_u(pk, nw, sb0, dir, j0 + 16);
            }
            fin = fin || ovf;
        }
        if (fin) retire(ovf);
        const bool refill = la_n == 0;
        if (refill) {
            LA = fwd16_u(pk, nw, sa0, dir, i0 + 16);
            LB = back16_u(pk, nw, sb0, dir, j0 + 16);
            la_n = 16;
        }
        // Every live value of the pair is >= 16 thr of its odd diagonal:
        // once that threshold reaches kR, take kR off the frame.
        if (active && rb) {
            const uint32_t mr = pack2(-kScale * kR);
#pragma unroll
            for (int t = 0; t < C2; ++t) {
                E[t] = __viaddmax_s16x2(E[t], mr, kDead2);
                O[t] = __viaddmax_s16x2(O[t], mr, kDead2);
            }
            Q -= kR;
        }
        if constexpr (Src::kCanAbort) {
            if (__any_sync(FULL, src.aborted())) return true;
        }
        if (__any_sync(FULL, !active && !exhausted) || !__any_sync(FULL, active)) return true;
        if (!masked) {
            refresh_budget();
            return budget < 1;
        }
        // Masked pairs are dearer: look again every 16 pairs (with the
        // refill) and go back to the unmasked copy once it is safe.
        if (refill) {
            refresh_budget();
            return budget >= 1;
        }
        return false;
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
                        mn = m + n;
                        ng = -sc.gap;
                        kR = rebase_step16(sc);
                        xup = (sc.x + 1) * 512;
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
        if (budget >= 1) {
            for (;;) {  // no cell of any window can leave its rectangle
                if (pair(T0{}) && handle(false)) break;
            }
        } else {
            for (;;) {
                if (pair(T1{}) && handle(true)) break;
            }
        }
    }
}

// Batched form of the packed kernel (same task source as lockstep_kernel).
// 128-thread blocks: with the FMA-pipe adds the loop holds about 85
// registers, five such blocks fit an SM (20 warps), and that measured faster
// than capping the registers for more warps.
constexpr int kPackedThreads = 128;
template <int L, int C2>
__global__ void __launch_bounds__(kPackedThreads)
lockstep16_kernel(const Job *jp, const uint32_t *order, const uint32_t *n_tasks_ptr,
                  uint32_t *counter, Spill spill, uint32_t one)
{
    BatchSrc src{jp, order, *n_tasks_ptr, counter, spill};
    lockstep16_loop<L, C2>(src, jp->packed, jp->n_words, one);
}

}  // namespace xd
