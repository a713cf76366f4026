"""Bit-level CPU model of the packed 16-bit band kernel (test infrastructure).

This is neither the oracle nor the CUDA path: it restates, in plain Python
integers, the arithmetic that ``lockstep16_loop`` in
``paper_2309_07270_gb300/csrc/xd_lockstep16.cuh`` performs for one group of
lanes (two window slots per 32-bit register, unsigned u16x2 max, plain
32-bit adds and multiply-adds of packed halves, byte permutes, the biased
and scaled frame in which a pruned slot holds 0, rebasing, the packed key,
the substitution built from match bits by multiplication, the window-edge
test after every pair of diagonals and the window shifts), so that
``test_packed16_model.py`` can check on the CPU that this arithmetic
reaches the oracle's result exactly, never wraps a 16-bit half and never
carries from one half into the other.  Any change to the kernel's
arithmetic must be made here too.
"""

M32 = 0xFFFFFFFF
SCALE = 16            # stored value = 16 * r
KEY0 = 0x8000         # key offset: a slot is live iff its key has bit 15 set


class Wrap(AssertionError):
    """A 16-bit half overflowed, or a 32-bit add carried from the low half
    into the high one: the kernel would have computed garbage."""


def s16(v):
    v &= 0xFFFF
    return v - 0x10000 if v & 0x8000 else v


def halves(x):
    return s16(x), s16(x >> 16)


def uhalves(x):
    return x & 0xFFFF, (x >> 16) & 0xFFFF


def mk(lo, hi):
    return ((lo & 0xFFFF) | ((hi & 0xFFFF) << 16)) & M32


def umk(lo, hi):
    for v in (lo, hi):
        if not 0 <= v <= 0xFFFF:
            raise Wrap(v)
    return lo | (hi << 16)


def prmt(a, b, sel):
    """PTX prmt.b32 (default mode): byte select with optional sign replication."""
    src = [(a >> (8 * k)) & 0xFF for k in range(4)] + [(b >> (8 * k)) & 0xFF for k in range(4)]
    out = 0
    for k in range(4):
        nib = (sel >> (4 * k)) & 0xF
        byte = src[nib & 7]
        if nib & 8:
            byte = 0xFF if byte & 0x80 else 0
        out |= byte << (8 * k)
    return out


def add2(a, b):
    """DPX-style per-half signed add (no carry between halves); wrap is an error."""
    la, ha = halves(a)
    lb, hb = halves(b)
    for v in (la + lb, ha + hb):
        if not -32768 <= v <= 32767:
            raise Wrap(v)
    return mk(la + lb, ha + hb)


def uadd32(a, b):
    """A plain 32-bit add (or multiply-add by one) of two packed registers:
    exact per half only when neither half, read unsigned, reaches 2^16."""
    la, ha = uhalves(a)
    lb, hb = uhalves(b)
    return umk(la + lb, ha + hb)


def usub32(a, b):
    """A plain 32-bit subtraction: exact per half only when no half borrows."""
    la, ha = uhalves(a)
    lb, hb = uhalves(b)
    return umk(la - lb, ha - hb)


def umax2(a, b):
    la, ha = uhalves(a)
    lb, hb = uhalves(b)
    return umk(max(la, lb), max(ha, hb))


def umax3(a, b, c):
    return umax2(umax2(a, b), c)


def max2(a, b):
    la, ha = halves(a)
    lb, hb = halves(b)
    return mk(max(la, lb), max(ha, hb))


def addmax2(a, b, c):
    return max2(add2(a, b), c)


def pack2(v):
    return ((v & 0xFFFF) * 0x10001) & M32


def fits(match, mismatch, gap, x, slots=16):
    """The packed tiles' range (packed16_ok in the kernel); tiles with 32
    slots per lane also need x + match <= 1022 (their keys carry 5 slot
    bits)."""
    ok = (match - gap <= 128 and mismatch >= -128 and mismatch - 2 * gap >= 0 and x >= 0
          and x + match <= 1536)
    return ok and (slots <= 16 or x + match <= 1022)


def key_scale(slots):
    """Key units per unit of r: 16 for up to 16 slots per lane, 32 for 32."""
    return 16 if slots <= 16 else 32


def slot_bits(slots):
    return 4 if slots <= 16 else 5


def rebase_step(match, gap, x, slots=16):
    """The frame step of one rebase (rebase_step16 in the kernel)."""
    ng = -gap
    return (0x8000 // key_scale(slots) - 8) - 3 * match - 3 * ng


def frame_bias(match, gap):
    """The frame's offset at the origin (threshold of diagonal 1 minus |gap|):
    every threshold is then at least match + 2|gap| + 1, so a pruned slot
    (stored 0) can never feed a live cell."""
    return match - gap + 1


def rebase_margin(match):
    """A rebase happens once the odd diagonal's threshold reaches kR plus this."""
    return match + 1


def live_lo(v):
    return (v & 0xFFFF) != 0


def live_hi(v):
    return (v >> 16) != 0


# Substitution of register t from the match bits.  e holds slot t's match
# bit at 2t+1 and slot t+C2's at 2t+17 (for C2 = 4 after one byte permute;
# for C2 = 16 registers 0-7 and 8-15 each take one of two byte-permuted
# merges of the two match words, eq7 of slots 0-15 and eqh of slots 16-31).
# Shifted left by 12 - 4*(t >> 1), the two bits sit at p = 13 + 2*(t & 1)
# and p + 16; a high multiply by dm * 2^(32-p), with dm = 16 (match -
# mismatch) < 2^13, turns them into the per-half match bonus, and the
# multiply-add's addend is the mismatch substitution.
def substitution(eq7, t, C2, mi2, dm, eqh=0):
    if C2 == 4:
        e = prmt(eq7, eq7, 0x2100)  # bytes 0, 0, 1, 2: slot t+4 moves up by 8
    elif C2 == 16:
        e = prmt(eq7, eqh, 0x5410) if t < 8 else prmt(eq7, eqh, 0x7632)
        t &= 7
    else:
        e = eq7
    sh, p = 12 - 4 * (t >> 1), 13 + 2 * (t & 1)
    src = (e << sh) & M32
    w = src & ((1 << p) | (1 << (p + 16)))
    K = dm << (32 - p)
    assert K <= M32 and (w * K) & M32 == 0
    return uadd32((w * K) >> 32, mi2)


def extend(a, b, match, mismatch, gap, x, lanes=4, regs=8, stats=None):
    """One extension over base codes a (length m) and b (length n) on a
    group of `lanes` lanes with `regs` registers (2*regs slots) per lane.

    Returns (score, best_i, best_j, overflow); with overflow True the
    kernel would hand the task to a wider tier and the other fields are
    meaningless.  ``stats`` (a dict) receives counts of window shifts up
    and down, rebases and masked pairs."""
    if stats is None:
        stats = {}
    for k in ("up", "down", "rebase", "masked"):
        stats.setdefault(k, 0)
    C2, S = regs, 2 * regs
    assert C2 in (4, 8, 16)
    assert fits(match, mismatch, gap, x, S)
    KS, SB = key_scale(S), slot_bits(S)
    W = lanes * S
    m, n = len(a), len(b)
    ng = -gap
    kR = rebase_step(match, gap, x, S)
    kRL = kR + rebase_margin(match)
    assert kR >= match + 2 * ng

    def base_a(i):  # 1-based; out-of-range positions get arbitrary codes
        return int(a[i - 1]) if 1 <= i <= m else (i * 7 + 1) & 3

    def base_b(j):
        return int(b[j - 1]) if 1 <= j <= n else (j * 5 + 2) & 3

    mi2 = pack2(SCALE * (mismatch + 2 * ng))
    dm = SCALE * (match - mismatch)
    E = [[0] * C2 for _ in range(lanes)]
    O = [[0] * C2 for _ in range(lanes)]
    beta = frame_bias(match, gap)
    origin = SCALE * (x + beta)
    for g in range(lanes):
        for t in range(C2):
            lo = origin if g * S + t == W // 2 else 0
            hi = origin if g * S + t + C2 == W // 2 else 0
            E[g][t] = umk(lo, hi)
    i0 = [-(W // 2) + g * S for g in range(lanes)]
    j0 = [(W // 2) - g * S for g in range(lanes)]
    d = T = 0
    Q = beta
    best = None  # (group key, window base i, diagonal)
    prev_dead = False

    def margin():  # diagonal pairs before a window cell can leave the rectangle
        return min(m - (i0[0] + W - 1), n - j0[0])

    def diagonal(odd, masked):
        """One anti-diagonal of the whole group; returns its group key."""
        nonlocal d, Q, T, best
        d += 1
        Q += ng
        for g in range(lanes):
            if odd:
                i0[g] += 1
            else:
                j0[g] += 1
        if not masked and margin() < 0:
            raise AssertionError("unmasked diagonal leaves the rectangle")
        V, U = (O, E) if odd else (E, O)
        thr = T + Q
        if not match + 2 * ng + 1 <= thr <= 0x8000 // KS:
            raise Wrap(("threshold", thr))
        z = umk(KEY0 - KS * thr, KEY0 - KS * thr)  # 0x80008000 - KS thr * 0x10001
        lane_keys = []
        newV = [list(v) for v in V]
        for g in range(lanes):
            eqs = []  # the kernel's base windows hold 2-bit fields, 16 slots a word
            for w0 in range(0, max(S, 16), 16):
                xx = 0
                for s in range(16):
                    xx |= ((base_a(i0[g] + w0 + s) ^ base_b(j0[g] - w0 - s)) & 3) << (2 * s)
                eqs.append(~(xx | (xx << 1)) & M32)  # bit 2s+1: slot w0+s matches
            eq7, eqh = eqs[0], eqs[-1]
            if odd:
                edge = U[g + 1][0] if g + 1 < lanes else 0
            else:
                edge = U[g - 1][C2 - 1] if g > 0 else 0
            keys = []
            for t in range(C2):
                if odd:
                    sh = U[g][t + 1] if t + 1 < C2 else prmt(U[g][0], edge, 0x5432)
                else:
                    sh = U[g][t - 1] if t > 0 else prmt(edge, U[g][C2 - 1], 0x5432)
                s2 = substitution(eq7, t, C2, mi2, dm, eqh)
                r = umax3(uadd32(V[g][t], s2), U[g][t], sh)
                if masked:
                    # slot s lies in the rectangle iff lo <= s <= hi:
                    # max(s - hi - 1, lo - 1 - s) < 0, bounds clamped to 16 bits
                    lo, hi = j0[g] - n, m - i0[g]
                    lo1_2 = pack2(min(max(lo - 1, -1024), 1024))
                    nhi1_2 = pack2(min(max(-hi - 1, -1024), 1024))
                    c = addmax2(mk(-t, -(t + C2)), lo1_2, 0x80008000)
                    u = addmax2(mk(t, t + C2), nhi1_2, c)
                    inside = prmt(u, u, 0xBB99)
                    r &= inside
                idx = (S - 1 - t) | ((S - 1 - (t + C2)) << 16)
                key = uadd32(r if KS == 16 else uadd32(r, r), uadd32(z, idx))
                lm = prmt(key, key, 0xBB99)  # 0xFFFF where live
                newV[g][t] = r & lm
                keys.append(key)
            kk = keys[0]
            for k_ in keys[1:]:
                kk = umax2(kk, k_)
            lk = max(uhalves(kk))
            lkey = lk - KEY0
            smask = (1 << SB) - 1
            lane_bits = ((31 - g) << SB) - 32 * KEY0
            mkey = 32 * lk - 31 * (lk & smask) + lane_bits
            assert mkey == (lkey >> SB) * (1 << (SB + 5)) + ((lkey & smask) | ((31 - g) << SB))
            lane_keys.append(mkey)
        for g in range(lanes):
            V[g][:] = newV[g]
        mkey = max(lane_keys)
        if mkey >= (x + 1) << (SB + 5):  # the diagonal's best value exceeds T
            T = T - x + (mkey >> (SB + 5))
            best = (mkey, i0[0], d)
        return mkey, thr

    def shift(up):
        if up:  # slot s takes slot s+1
            ne = [E[g + 1][0] if g + 1 < lanes else 0 for g in range(lanes)]
            no = [O[g + 1][0] if g + 1 < lanes else 0 for g in range(lanes)]
            for g in range(lanes):
                te, to = prmt(E[g][0], ne[g], 0x5432), prmt(O[g][0], no[g], 0x5432)
                E[g], O[g] = E[g][1:] + [te], O[g][1:] + [to]
                i0[g] += 1
                j0[g] -= 1
        else:   # slot s takes slot s-1
            pe = [E[g - 1][C2 - 1] if g > 0 else 0 for g in range(lanes)]
            po = [O[g - 1][C2 - 1] if g > 0 else 0 for g in range(lanes)]
            for g in range(lanes):
                te, to = prmt(pe[g], E[g][C2 - 1], 0x5432), prmt(po[g], O[g][C2 - 1], 0x5432)
                E[g], O[g] = [te] + E[g][:-1], [to] + O[g][:-1]
                i0[g] -= 1
                j0[g] += 1

    budget = margin()
    while True:
        masked = budget < 1
        stats["masked"] += masked
        key_o, thr_o = diagonal(True, masked)
        key_e, _ = diagonal(False, masked)
        dead_o, dead_e = key_o < 0, key_e < 0
        fin = (dead_o and (prev_dead or dead_e)) or d >= m + n
        prev_dead = dead_e
        budget -= 1
        if fin:
            if best is None:
                return T, 0, 0, False
            key, ibase, bd = best
            bi = ibase + (31 - ((key >> SB) & 31)) * S + (S - 1 - (key & ((1 << SB) - 1)))
            return T, bi, bd - bi, False
        # Window edges after the even diagonal (live slots hold values > 0,
        # pruned ones 0).  Up: the top slot of E (diagonal d) or of O (d-1)
        # is live, and E's two bottom slots and O's bottom slot are dead.
        # Down: E's bottom slot is live and the two top slots of E and of O
        # are dead.  Otherwise, with an edge live, the band has outgrown the
        # window.
        top, bot = lanes - 1, 0
        need_up = live_hi(E[top][C2 - 1]) or live_hi(O[top][C2 - 1])
        need_dn = live_lo(E[bot][0])
        blk_up = live_lo(E[bot][0]) or live_lo(E[bot][1]) or live_lo(O[bot][0])
        blk_dn = need_up or live_hi(E[top][C2 - 2]) or live_hi(O[top][C2 - 2])
        if need_up:
            if blk_up:
                return T, 0, 0, True
            stats["up"] += 1
            shift(True)
            budget = margin()
        elif need_dn:
            if blk_dn:
                return T, 0, 0, True
            stats["down"] += 1
            shift(False)
            budget = margin()
        if thr_o >= kRL:  # every live value is >= 16 (kR + margin): rebase
            stats["rebase"] += 1
            mr = pack2(SCALE * kR)
            for g in range(lanes):
                for t in range(C2):
                    E[g][t] = usub32(umax2(E[g][t], mr), mr)
                    O[g][t] = usub32(umax2(O[g][t], mr), mr)
            Q -= kR
        if budget < 1:
            budget = margin()
