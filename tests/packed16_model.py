"""Bit-level CPU model of the packed 16-bit band kernel (test infrastructure).

This is neither the oracle nor the CUDA path: it restates, in plain Python
integers, the arithmetic that ``lockstep16_loop`` in
``paper_2309_07270_gb300/csrc/xd_lockstep16.cuh`` performs for one group of
lanes (two window slots per 32-bit register, s16x2 max / add-max, byte
permutes, the normalised and scaled frame, rebasing, the packed key and the
window shifts), so that ``test_packed16_model.py`` can check on the CPU that
this arithmetic reaches the oracle's result exactly and never wraps a 16-bit
half.  Any change to the kernel's arithmetic must be made here too.
"""

M32 = 0xFFFFFFFF
SCALE = 16            # stored value = 16 * r
DEAD = -512 * SCALE   # stored value of a pruned slot
DEAD2 = 0xE000E000
REBASE = 256          # frame step, in units of r


class Wrap(AssertionError):
    """A 16-bit half overflowed: the kernel would have computed garbage."""


def s16(v):
    v &= 0xFFFF
    return v - 0x10000 if v & 0x8000 else v


def halves(x):
    return s16(x), s16(x >> 16)


def mk(lo, hi):
    return ((lo & 0xFFFF) | ((hi & 0xFFFF) << 16)) & M32


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
    la, ha = halves(a)
    lb, hb = halves(b)
    for v in (la + lb, ha + hb):
        if not -32768 <= v <= 32767:
            raise Wrap(v)
    return mk(la + lb, ha + hb)


def max2(a, b):
    la, ha = halves(a)
    lb, hb = halves(b)
    return mk(max(la, lb), max(ha, hb))


def addmax2(a, b, c):
    return max2(add2(a, b), c)


def pack2(v):
    return ((v & 0xFFFF) * 0x10001) & M32


def fits(match, mismatch, gap, x):
    """The packed tiles' range (packed16_ok in the kernel)."""
    return match - gap <= 128 and mismatch >= -128 and x >= 0 and x + match <= 1536


def extend(a, b, match, mismatch, gap, x, lanes=4, regs=8, stats=None):
    """One extension over base codes a (length m) and b (length n) on a
    group of `lanes` lanes with `regs` registers (2*regs slots) per lane.

    Returns (score, best_i, best_j, overflow); with overflow True the
    kernel would hand the task to a wider tier and the other fields are
    meaningless.  ``stats`` (a dict) receives counts of window shifts up
    and down, rebases and masked diagonals."""
    if stats is None:
        stats = {}
    for k in ("up", "down", "rebase", "masked"):
        stats.setdefault(k, 0)
    C2, S = regs, 2 * regs
    W = lanes * S
    m, n = len(a), len(b)
    ng = -gap

    def base_a(i):  # 1-based; out-of-range positions get codes no base has
        return int(a[i - 1]) if 1 <= i <= m else 4 + (i & 3)

    def base_b(j):
        return int(b[j - 1]) if 1 <= j <= n else 8 + (j & 3)

    ma2 = pack2(SCALE * (match + 2 * ng))
    mi2 = pack2(SCALE * (mismatch + 2 * ng))
    E = [[0] * C2 for _ in range(lanes)]
    O = [[DEAD2] * C2 for _ in range(lanes)]
    for g in range(lanes):
        for t in range(C2):
            lo = SCALE * x if g * S + t == W // 2 else DEAD
            hi = SCALE * x if g * S + t + C2 == W // 2 else DEAD
            E[g][t] = mk(lo, hi)
    i0 = [-(W // 2) + g * S for g in range(lanes)]
    j0 = [(W // 2) - g * S for g in range(lanes)]
    d = T = Q = 0
    best = None  # (group key, window base i, diagonal)
    prev_dead = False

    def margin():
        return min(m - (i0[0] + W - 1), n - j0[0])

    budget = margin()
    masked = budget < 2
    while True:
        for odd in (True, False):
            d += 1
            Q += ng
            budget -= 1
            for g in range(lanes):
                if odd:
                    i0[g] += 1
                else:
                    j0[g] += 1
            if not masked and margin() < 0:
                raise AssertionError("unmasked diagonal leaves the rectangle")
            V, U = (O, E) if odd else (E, O)
            stats["masked"] += masked
            nthr2 = pack2(-SCALE * (T + Q))
            lane_keys = []
            for g in range(lanes):
                eq = 0
                for s in range(16):
                    if base_a(i0[g] + s) == base_b(j0[g] - s):
                        eq |= 1 << (2 * s)
                R = [(eq << (7 - 2 * k)) & M32 for k in range(4)]
                if odd:
                    edge = U[g + 1][0] if g + 1 < lanes else DEAD2
                else:
                    edge = U[g - 1][C2 - 1] if g > 0 else DEAD2
                keys, newV = [], list(V[g])
                for t in range(C2):
                    if odd:
                        sh = U[g][t + 1] if t + 1 < C2 else prmt(U[g][0], edge, 0x5432)
                    else:
                        sh = U[g][t - 1] if t > 0 else prmt(edge, U[g][C2 - 1], 0x5432)
                    nb = max2(U[g][t], sh)
                    sel = ((8 | (t >> 2)) | ((8 | (t >> 2)) << 4) |
                           ((8 | ((t + C2) >> 2)) << 8) | ((8 | ((t + C2) >> 2)) << 12))
                    mk_ = prmt(R[t & 3], R[t & 3], sel)
                    s2 = (mk_ & ma2) | (~mk_ & mi2 & M32)
                    r = addmax2(V[g][t], s2, nb)
                    if masked:
                        # slot s lies in the rectangle iff lo <= s <= hi:
                        # max(s - hi - 1, lo - 1 - s) < 0, bounds clamped to 16 bits
                        lo, hi = j0[g] - n, m - i0[g]
                        lo1_2 = pack2(min(max(lo - 1, -1024), 1024))
                        nhi1_2 = pack2(min(max(-hi - 1, -1024), 1024))
                        slot2 = mk(t, t + C2)
                        nslot2 = mk(-t, -(t + C2))
                        c = addmax2(nslot2, lo1_2, 0x80008000)
                        u = addmax2(slot2, nhi1_2, c)
                        inside = prmt(u, u, 0xBB99)
                        r = ((r & inside) | (DEAD2 & ~inside)) & M32
                    idx = (S - 1 - t) | ((S - 1 - (t + C2)) << 16)
                    kc = addmax2(idx, nthr2, 0x80008000)
                    key = addmax2(r, kc, 0xFFF0FFF0)
                    pm = prmt(key, key, 0xBB99)
                    newV[t] = ((r & ~pm) | (DEAD2 & pm)) & M32
                    keys.append(key)
                V[g][:] = newV
                kk = keys[0]
                for k_ in keys[1:]:
                    kk = max2(kk, k_)
                lk = max(halves(kk))
                lane_keys.append((lk >> 4) * 512 + ((lk & 15) | ((31 - g) << 4)))
            mkey = max(lane_keys)
            xm = mkey >> 9
            if xm > x:
                T = T - x + xm
                best = (mkey, i0[0], d)
            dead = mkey < 0
            fin = (dead and prev_dead) or d >= m + n
            prev_dead = dead
            dead16 = DEAD & 0xFFFF
            # window edges: after an odd diagonal a live top slot may seed a
            # cell above the window (shift up), after an even one a live
            # bottom slot one below it (shift down); with the opposite edge
            # live too the band outgrew the window
            vtop, vbot = V[lanes - 1][C2 - 1] >> 16, V[0][0] & 0xFFFF
            if not fin and (vtop if odd else vbot) != dead16:
                if (vbot if odd else vtop) != dead16:
                    return T, 0, 0, True
                stats["up" if odd else "down"] += 1
                if odd:  # shift up: slot s takes slot s+1
                    ne = [E[g + 1][0] if g + 1 < lanes else DEAD2 for g in range(lanes)]
                    no = [O[g + 1][0] if g + 1 < lanes else DEAD2 for g in range(lanes)]
                    for g in range(lanes):
                        te, to = prmt(E[g][0], ne[g], 0x5432), prmt(O[g][0], no[g], 0x5432)
                        E[g], O[g] = E[g][1:] + [te], O[g][1:] + [to]
                        i0[g] += 1
                        j0[g] -= 1
                else:    # shift down: slot s takes slot s-1
                    pe = [E[g - 1][C2 - 1] if g > 0 else DEAD2 for g in range(lanes)]
                    po = [O[g - 1][C2 - 1] if g > 0 else DEAD2 for g in range(lanes)]
                    for g in range(lanes):
                        te, to = prmt(pe[g], E[g][C2 - 1], 0x5432), prmt(po[g], O[g][C2 - 1], 0x5432)
                        E[g], O[g] = [te] + E[g][:-1], [to] + O[g][:-1]
                        i0[g] -= 1
                        j0[g] += 1
                if not masked:
                    budget = margin()
            if fin:
                if best is None:
                    return T, 0, 0, False
                key, ibase, bd = best
                bi = ibase + (31 - ((key >> 4) & 31)) * S + (S - 1 - (key & 15))
                return T, bi, bd - bi, False
            if not odd:
                if T + Q + ng >= REBASE:
                    stats["rebase"] += 1
                    mr = pack2(-SCALE * REBASE)
                    for g in range(lanes):
                        for t in range(C2):
                            E[g][t] = addmax2(E[g][t], mr, DEAD2)
                            O[g][t] = addmax2(O[g][t], mr, DEAD2)
                    Q -= REBASE
                if not masked and budget < 2:
                    budget = margin()
                    masked = budget < 2
