// Packed 16-bit lockstep band kernel: two window slots per 32-bit register.
//
// Same extension, same reading of the X-drop recurrence and the same
// results as lockstep_loop (xd_device.cuh); only the arithmetic changes.
// It is exact whenever the scoring passes packed16_ok():
//   match - gap <= 128, mismatch >= -128, mismatch + 2|gap| >= 0,
//   x + match <= 1536,
// and, for lanes of 32 slots, packed32_ok(): also x + match <= 1022.
//
// Biased, normalised scores.  A live cell on anti-diagonal d holds
//   r = H + x + d*|gap| - B + beta     (B: the rebase steps taken off,
//                                       beta = match + |gap| + 1)
// stored as 16*r in an unsigned half; a pruned cell holds 0.  The two gap
// predecessors enter unchanged and the diagonal one with s + 2|gap| >= 0:
//   r(d) = max(r_diag(d-2) + s + 2|gap|,  r_up(d-1),  r_left(d-1)),
// one 32-bit add (both halves at once, see below) and one u16x2 three-way
// max per register (two cells).  The X-drop threshold of diagonal d (T of
// d-1 minus x) becomes thr = T + d*|gap| - B + beta, a cell is live iff
// r >= thr, and r - thr <= x + match.  Every threshold is at least
// match + 2|gap| + 1, so a pruned predecessor (0, or 16*(s + 2|gap|) after
// the diagonal add) can never lift a cell to its threshold: a cell with no
// live predecessor stays pruned, and one with a live predecessor takes the
// same maximum as the recurrence over live predecessors.
//
// Key.  One more 32-bit multiply-add gives each slot's key
//   0x8000 + KS*(r - thr) + (S-1-slot),
// with KS = 16 key units per unit of r for lanes of up to 16 slots (a
// 4-bit slot index; the add takes the stored 16 r as it is) and KS = 32
// for lanes of 32 (a 5-bit index; the multiply-add doubles 16 r).  Bit 15
// is set exactly for the live cells (a byte permute spreads that bit into
// the mask that zeroes the pruned ones) and, for live cells, the key
// orders by value and then by lowest slot.  The lane's best key becomes
// value * 2^(SB+5) + (31 - lane) * 2^SB + slot bits in 32 bits (SB = 4 or
// 5 slot bits), so one group max gives the largest value and, among equal
// values, the lowest window slot: the first cell in order of increasing i
// on the diagonal.
//
// Substitution.  The match bits of each 16 slots of a lane come from one
// XOR of two 2-bit base-window words (a lane of 32 slots keeps two words
// per read, and byte permutes merge its two match words for each half of
// its 16 registers).  For register t the two bits (slots t and t+C2) are
// moved to bits p and p+16, p = 13 or 15, by a left shift (a multiply on
// the FMA pipe) and masked; a high multiply by 16 (match - mismatch) *
// 2^(32-p) turns them into the per-half match bonus, and its addend is the
// mismatch substitution.  One ALU instruction (the mask) per register.
//
// Layout.  Lane g of a group of L lanes holds the window slots g*S .. g*S+S-1
// (S = 2*C2 slots).  Register t holds slot t in its low half and slot t+C2
// in its high half, so the neighbour slot s+1 (s-1) of every slot in
// register t sits in register t+1 (t-1) at the same half; only the end
// registers need a byte permute and one shuffle per diagonal.
//
// Ranges, in units of r, with kR = (0x8000 / KS - 8) - 3 match - 3|gap|
// the rebase step (rebase_step16: at least 1656 for KS = 16 and 632 for
// KS = 32 inside the ranges above, and at least match + 2|gap|, the most
// one pair of diagonals can raise a threshold); the figures below are for
// KS = 16, and for KS = 32 they halve (thresholds <= 1016, keys below
// 2^16 by x + match <= 1022, 32 r below 2^16).
// After every pair of diagonals (odd d-1, even d) the frame is rebased by
// kR once thr of d-1 reaches kR + match + 1.  Every live value of d-1 and d
// is at least that threshold, so it stays above match + 1 > 0 after the
// rebase, and the next threshold is again at least match + 2|gap| + 1.
// thr grows by at most 3|gap| + 2 match over the three diagonals between
// two tests, so thr <= 2040 always (16 thr < 0x8000: the key's pruned
// range stays non-negative) and every live value is at most
// thr + x + match <= 3576 (16 times that < 2^16).
//
// Carry-free adds.  V + s2 (stored value plus packed substitution, s2 <=
// 16*256), z + idx (z = 0x8000 - 16 thr per half) and r + (z + idx) are
// plain 32-bit adds: by the ranges above no low half, read unsigned,
// reaches 2^16, so nothing carries into the high half.
//
// Window edges.  Live values are > 0 and pruned ones 0, so a half is live
// iff it is nonzero.  The edges are tested once per pair of diagonals,
// after the even one: no live cell of diagonals d+1, d+2 can leave the
// window unless E's top slot (diagonal d) or O's top slot (d-1) is live,
// or E's bottom slot is.  The window then shifts up one slot if E's two
// bottom slots and O's bottom slot are dead, or down one slot if the two
// top slots of E and of O are dead; otherwise the band has outgrown the
// window and the task goes to a wider tier.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "xd_device.cuh"

namespace xd {

namespace p16 {

constexpr int32_t kScale = 16;       // stored value = 16 * r
constexpr uint32_t kKey2 = 0x80008000u;  // key offset in both halves: live iff bit 15

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

// The high word of a * b, plus c (FMA pipe).
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
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

// Register t's match bits: shifted left by 12 - 4 (t >> 1) they sit at
// bits p and p + 16, p = 13 + 2 (t & 1) (see the header).
__host__ __device__ constexpr int subst_shift(int t) { return 12 - 4 * (t >> 1); }
__host__ __device__ constexpr uint32_t subst_mask(int t)
{
    return (1u << (13 + 2 * (t & 1))) | (1u << (29 + 2 * (t & 1)));
}

template <int N>
__device__ __forceinline__ uint32_t tree_max2(const uint32_t (&k)[N])
{
    if constexpr (N == 1) {
        return k[0];
    } else if constexpr (N == 2) {
        return __vmaxu2(k[0], k[1]);
    } else {
        constexpr int M = (N + 2) / 3;
        uint32_t r[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (3 * i + 2 < N) r[i] = __vimax3_u16x2(k[3 * i], k[3 * i + 1], k[3 * i + 2]);
            else if (3 * i + 1 < N) r[i] = __vmaxu2(k[3 * i], k[3 * i + 1]);
            else r[i] = k[3 * i];
        }
        return tree_max2<M>(r);
    }
}

// A slot is live iff its half is nonzero (pruned slots hold 0).
__device__ __forceinline__ bool live_lo(uint32_t v) { return (v & 0xFFFFu) != 0; }
__device__ __forceinline__ bool live_hi(uint32_t v) { return (v >> 16) != 0; }

// Key units per unit of r, and slot bits of a key: lanes of up to 16 slots
// keep 16 r and a 4-bit slot index; lanes of 32 slots a 5-bit index, with
// keys in units of 32 r (the key add doubles the stored value).
template <int S>
__host__ __device__ constexpr int key_scale() { return S <= 16 ? 16 : 32; }
template <int S>
__host__ __device__ constexpr int slot_bits() { return S <= 16 ? 4 : 5; }

// One anti-diagonal for one lane: V (diagonal d-2, overwritten with d) and
// U (d-1).  edge: the neighbouring lane's end register of U (next lane's
// register 0 on odd diagonals, previous lane's register C2-1 on even ones),
// 0 beyond the group.  eq7: bit 2s+1 set iff slot s's bases match (slots
// 0-15); eqh: the same for slots 16-31 (C2 = 16 only).  k13, k15:
// 16 (match - mismatch) << 19 and << 17; mi2: the packed mismatch
// substitution 16 (mismatch + 2|gap|); z: 0x8000 - KS thr in both halves
// (KS = key_scale).  Returns the lane's largest key (0 .. 0xFFFF; below
// 0x8000 iff every slot was pruned).
template <int C2, bool ODD, bool MASKED>
__device__ __forceinline__ uint32_t dp16(uint32_t (&V)[C2], const uint32_t (&U)[C2],
                                         uint32_t edge, uint32_t eq7, uint32_t eqh,
                                         uint32_t mi2, uint32_t k13, uint32_t k15, uint32_t z,
                                         uint32_t lo1_2, uint32_t nhi1_2, uint32_t one)
{
    static_assert(C2 == 4 || C2 == 8 || C2 == 16, "packed registers per lane");
    constexpr int NE = C2 == 16 ? 2 : 1;
    // e[h]: slot t's match bit at 2t+1, slot t+C2's at 2t+17 (registers
    // 8h .. 8h+7)
    uint32_t e[NE];
    if constexpr (C2 == 4) e[0] = prmt(eq7, eq7, 0x2100);
    else if constexpr (C2 == 8) e[0] = eq7;
    else { e[0] = prmt(eq7, eqh, 0x5410); e[1] = prmt(eq7, eqh, 0x7632); }
    uint32_t es[4 * NE];
#pragma unroll
    for (int h = 0; h < NE; ++h) {
        es[4 * h] = fma_add(e[h], one << 12, 0u);
        es[4 * h + 1] = fma_add(e[h], one << 8, 0u);
        es[4 * h + 2] = fma_add(e[h], one << 4, 0u);
        es[4 * h + 3] = e[h];
    }
    uint32_t key[C2];
#pragma unroll
    for (int t = 0; t < C2; ++t) {
        uint32_t sh;
        if (ODD) sh = (t + 1 < C2) ? U[t + 1] : prmt(U[0], edge, 0x5432);
        else sh = (t > 0) ? U[t - 1] : prmt(edge, U[C2 - 1], 0x5432);
        const uint32_t w = es[t >> 1] & subst_mask(t);
        const uint32_t s2 = mad_hi(w, (t & 1) ? k15 : k13, mi2);
        uint32_t r = __vimax3_u16x2(fma_add(V[t], one, s2), U[t], sh);  // carry-free (header)
        if (MASKED) {
            // slot s lies in the rectangle iff lo <= s <= hi (lo = j0 - n,
            // hi = m - i0): max(s - hi - 1, lo - 1 - s) < 0, per half
            const uint32_t c = __viaddmax_s16x2(nslot2<C2>(t), lo1_2, 0x80008000u);
            const uint32_t u = __viaddmax_s16x2(slot2<C2>(t), nhi1_2, c);
            r &= prmt(u, u, 0xBB99);  // 0xFFFF where inside
        }
        // 0x8000 + KS*(r - thr) + (S-1-slot): bit 15 set iff live
        const uint32_t k = fma_add(r, (key_scale<2 * C2>() == 16) ? one : one << 1,
                                   fma_add(z, one, idx2<C2>(t)));
        V[t] = r & prmt(k, k, 0xBB99);
        key[t] = k;
    }
    const uint32_t kk = tree_max2<C2>(key);
    return max(kk >> 16, kk & 0xFFFFu);
}

}  // namespace p16

__host__ __device__ inline bool packed16_ok(const Scoring &sc)
{
    return sc.match - sc.gap <= 128 && sc.mismatch >= -128 && sc.mismatch - 2 * sc.gap >= 0 &&
           sc.x >= 0 && sc.x + sc.match <= 1536;
}

// Lanes of 32 slots keep keys in units of 32 r, so their keys (0x8000 +
// 32 (x + match) + 31 at most) need x + match <= 1022 as well.
__host__ __device__ inline bool packed32_ok(const Scoring &sc)
{
    return packed16_ok(sc) && sc.x + sc.match <= 1022;
}

// Frame step of one rebase (units of r) for a scoring that passes
// packed16_ok: the threshold cap 0x8000 / KS - 8 (2040 or 1016) less
// 3 match + 3|gap|, so between 1656 and 2033 for lanes of up to 16 slots
// and between 632 and 1009 for lanes of 32 (see the header comment's
// ranges).
template <int S>
__host__ __device__ inline int32_t rebase_step16(const Scoring &sc)
{
    return (0x8000 / p16::key_scale<S>() - 8) - 3 * sc.match + 3 * sc.gap;
}

// one: 1 (see fma_add).
template <int L, int C2, class Src>
__device__ __forceinline__ void lockstep16_loop(Src &src, const uint32_t *pk, int64_t nw,
                                                uint32_t one)
{
    using namespace p16;
    constexpr int S = 2 * C2;  // slots per lane
    constexpr int W = L * S;
    constexpr bool WIDE = S == 32;              // two base-window words per read
    constexpr int SB = slot_bits<S>();          // slot bits of a key
    constexpr int VS = SB + 5;                  // value shift of a group key
    constexpr uint32_t SMASK = (1u << SB) - 1u;
    // -KS * 0x10001: z = 0x80008000 - KS thr in both halves
    constexpr uint32_t ZMUL = 0u - (uint32_t)key_scale<S>() * 0x10001u;
    static_assert(S <= 32 && 32 % L == 0 && L >= 2 && C2 % 4 == 0, "packed tile shape");
    const int lane = threadIdx.x & 31;
    const int glane = lane % L;
    const int gbase = lane - glane;
    const unsigned gm = group_mask<L>(gbase);
    const bool bot_lane = glane == 0, top_lane = glane == L - 1;
    // per-lane constants: 0/1 factors that clear the shuffled-in edge
    // beyond the group, and the halves the window-edge test reads
    const uint32_t keep_up = top_lane ? 0u : 1u, keep_dn = bot_lane ? 0u : 1u;
    const uint32_t tmask = top_lane ? 0xFFFF0000u : 0u, bmask = bot_lane ? 0x0000FFFFu : 0u;

    // Per-group task state (uniform within a group).
    bool active = false, exhausted = false;
    uint32_t task = 0;
    const Job *gj = nullptr;
    Scoring sc{1, -1, -1, 0};
    int64_t sa0 = 0, sb0 = 0;
    int dir = 1;
    int32_t mn = 0, m = 0, n = 0, d = 0, i0 = 0, j0 = 0, T = 0, bi = 0, bj = 0;
    int32_t Q = 0;                      // frame offset: thr = T + Q
    int32_t kR = 0, kRL = 0;            // rebase step, and the threshold that triggers one
    int32_t xup = 0;                    // (x + 1) << VS: a group key this large raises T
    int32_t bkey = 0, bi0 = 0, bd = 0;  // best cell: group key, this lane's i0, diagonal
    int32_t ng = 1;                     // |gap|
    uint32_t mi2 = 0;                   // packed 16 * (mismatch + 2|gap|)
    uint32_t k13 = 0, k15 = 0;          // 16 (match - mismatch) << 19, << 17
    bool prev_dead = false, fin = false, rb = false;
    uint32_t E[C2], O[C2];
#pragma unroll
    for (int t = 0; t < C2; ++t) { E[t] = 0u; O[t] = 0u; }
    // base windows (slots 0-15; Aw1, Bw1: slots 16-31 of 32-slot lanes) and
    // the lookahead words
    uint32_t Aw = 0, Aw1 = 0, LA = 0, Bw = 0, Bw1 = 0, LB = 0;
    int la_n = 16;        // warp-uniform: diagonal pairs the lookahead words still cover
    int32_t budget = 0;   // warp-uniform: diagonal pairs known to stay inside every rectangle
    // (31 - lane) * 16, less the key offset's share of the group key
    const int32_t lane_bits = ((31 - glane) << SB) - (0x8000 << 5);

    auto retire = [&](bool overflow) {
        if (bd > 0) {
            bi = (bi0 - glane * S) + (31 - ((bkey >> SB) & 31)) * S + (S - 1 - (int)(bkey & SMASK));
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

    // The base windows of this lane's slots at the current i0, j0: slot s
    // holds a[i0 + s] and b[j0 - s]; the lookahead words the next 16 bases.
    auto load_windows = [&]() {
        Aw = fwd16_u(pk, nw, sa0, dir, i0);
        Bw = back16_u(pk, nw, sb0, dir, j0);
        if constexpr (WIDE) {
            Aw1 = fwd16_u(pk, nw, sa0, dir, i0 + 16);
            Bw1 = back16_u(pk, nw, sb0, dir, j0 - 16);
        }
        LA = fwd16_u(pk, nw, sa0, dir, i0 + (WIDE ? 32 : 16));
        LB = back16_u(pk, nw, sb0, dir, j0 + 16);
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
            if constexpr (WIDE) {
                Aw = __funnelshift_r(Aw, Aw1, 2);
                Aw1 = __funnelshift_r(Aw1, LA, 2);
            } else {
                Aw = __funnelshift_r(Aw, LA, 2);
            }
            LA >>= 2;
        } else {
            ++j0;
            if constexpr (WIDE) Bw1 = __funnelshift_l(Bw, Bw1, 2);
            Bw = __funnelshift_l(LB, Bw, 2);
            LB <<= 2;
        }
        thr = T + Q;
        // 0x8000 - 16 thr in both halves (no borrow: 16 thr <= 0x8000)
        const uint32_t z = (uint32_t)thr * ZMUL + kKey2;
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
        uint32_t eqh = 0u;
        if constexpr (WIDE) {
            const uint32_t xh = Aw1 ^ Bw1;
            eqh = ~(xh | (xh << 1));
        }
        uint32_t lk;
        if (ODD) {
            const uint32_t edge = fma_add(__shfl_down_sync(FULL, E[0], 1, L), keep_up, 0u);
            lk = dp16<C2, true, MASKED>(O, E, edge, eq7, eqh, mi2, k13, k15, z, lo1_2, nhi1_2,
                                        one);
        } else {
            const uint32_t edge = fma_add(__shfl_up_sync(FULL, O[C2 - 1], 1, L), keep_dn, 0u);
            lk = dp16<C2, false, MASKED>(E, O, edge, eq7, eqh, mi2, k13, k15, z, lo1_2, nhi1_2,
                                         one);
        }
        // Group key: value above lane above slot in lane, so one max finds
        // the lowest window slot among the cells holding the maximum.  With
        // lk = 0x8000 + 2^SB v + i: 32 lk - 31 i = 0x8000 * 32 + 2^VS v + i
        // (multiply-adds).
        const int32_t mkey = lockstep_group_max<L>(
            (int32_t)fma_add(lk, one << 5, fma_add(lk & SMASK, 0u - 31u, (uint32_t)lane_bits)));
        if (mkey >= xup) {  // best value - thr > x: T rises (decoded at retire)
            T += (mkey >> VS) - sc.x;
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
        rb = active && thr_o >= kRL;
        // window edges: this group's bottom lane tests E's bottom slot, its
        // top lane the top slots of E and O (a nonzero half is live)
        const uint32_t ew = ((E[C2 - 1] | O[C2 - 1]) & tmask) | (E[0] & bmask);
        const bool edge = active && ew != 0u;
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
                if (top_lane) { ne = 0u; no = 0u; }
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
                if (bot_lane) { pe = 0u; po = 0u; }
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
                load_windows();
            }
            fin = fin || ovf;
        }
        if (fin) retire(ovf);
        const bool refill = la_n == 0;
        if (refill) {
            LA = fwd16_u(pk, nw, sa0, dir, i0 + (WIDE ? 32 : 16));
            LB = back16_u(pk, nw, sb0, dir, j0 + 16);
            la_n = 16;
        }
        // Every live value of the pair is >= 16 thr of its odd diagonal:
        // once that threshold reaches kR + match + 1, take kR off the frame
        // (pruned halves stay 0; no half borrows).
        if (active && rb) {
            const uint32_t mr = pack2(kScale * kR);
#pragma unroll
            for (int t = 0; t < C2; ++t) {
                E[t] = __vmaxu2(E[t], mr) - mr;
                O[t] = __vmaxu2(O[t], mr) - mr;
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
                    if (e.ok && !(WIDE ? packed32_ok(sc) : packed16_ok(sc))) {
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
                        kR = rebase_step16<S>(sc);
                        kRL = kR + sc.match + 1;
                        xup = (sc.x + 1) << VS;
                        mi2 = pack2(kScale * (sc.mismatch + 2 * ng));
                        k13 = (uint32_t)(kScale * (sc.match - sc.mismatch)) << 19;
                        k15 = (uint32_t)(kScale * (sc.match - sc.mismatch)) << 17;
                        // origin (H = 0) at window slot W/2, stored as
                        // 16 * (x + beta), beta = match + |gap| + 1
                        const int32_t beta = sc.match + ng + 1;
                        const uint32_t orig = (uint32_t)(kScale * (sc.x + beta));
#pragma unroll
                        for (int t = 0; t < C2; ++t) {
                            const int slo = glane * S + t, shi = slo + C2;
                            const uint32_t lo = (slo == W / 2) ? orig : 0u;
                            const uint32_t hi = (shi == W / 2) ? orig : 0u;
                            E[t] = lo | (hi << 16);
                            O[t] = 0u;
                        }
                        i0 = -(W / 2) + glane * S;
                        j0 = (W / 2) - glane * S;
                        load_windows();
                        d = 0;
                        T = 0;
                        Q = beta;
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
// 128-thread blocks: the loop holds about 96 registers with 16 slots per
// lane (five such blocks fit an SM, 20 warps) and 128 with 32 (four blocks),
// and that measured faster than capping the registers for more warps.
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
