"""CPU check of the packed 16-bit band arithmetic against the oracle.

``packed16_model`` restates the kernel's 16-bit arithmetic bit by bit
(two slots per register, u16x2 max and carry-free 32-bit adds and
multiply-adds of packed halves, the biased frame in which a pruned slot
holds 0, rebases, packed keys, the substitution from multiplied match bits,
window shifts decided once per pair of diagonals).  On seeded random
extensions, including scorings at the edges of the packed range, it must
reach the oracle's (score, best_i, best_j) exactly whenever the band fits
the window, and no 16-bit half may ever wrap.  This pins the exactness
argument of the packed tiles without a GPU; the GPU tests pin the kernel
itself.
"""
import numpy as np
import pytest

import packed16_model as P
from paper_2309_07270_gb300 import workloads as W

SCORINGS = [
    (1, -1, -1, 50),
    (1, 0, -1, 20),         # mismatch + 2|gap| > 0, many ties
    (2, -3, -2, 30),
    (64, -128, -64, 1472),  # every limit at once
    (3, -2, -125, 100),     # the frame grows fastest through the gap
    (127, -1, -1, 1409),    # largest match
    (1, -2, -1, 1535),      # largest x, mismatch = 2 gap
    (7, -1, -2, 0),         # x = 0
]


def cases(seed, n, slots=16):
    rng = np.random.default_rng(seed)
    scorings = [sc for sc in SCORINGS if P.fits(*sc, slots)]
    for k in range(n):
        sc = scorings[k % len(scorings)]
        la, lb = int(rng.integers(0, 260)), int(rng.integers(0, 260))
        t = rng.integers(0, 4, max(la, lb) + 40).astype(np.uint8)
        kind = k % 3
        if kind == 0:    # related: the second read mutated at 12 %
            b, *_ = W.mutate(t, rng)
            yield sc, t[:la], b[:lb]
        elif kind == 1:  # unrelated
            yield sc, rng.integers(0, 4, la).astype(np.uint8), rng.integers(0, 4, lb).astype(np.uint8)
        else:            # identical prefixes
            yield sc, t[:la], t[:lb].copy()


def test_scorings_are_in_the_packed_range():
    assert all(P.fits(*sc) for sc in SCORINGS)
    assert not P.fits(1, -1, -1, 1536) and not P.fits(128, -1, -1, 10)
    assert not P.fits(1, -129, -1, 10) and not P.fits(1, -1, -128, 10)
    assert not P.fits(1, -3, -1, 10)  # mismatch + 2|gap| < 0: 32-bit tiles
    # Over the whole packed range: the rebase step is at least what one pair
    # of diagonals can add to a threshold (so rebasing keeps up), every
    # threshold stays <= 2040 (16 thr < 0x8000: pruned keys stay >= 0),
    # every live value times 16 fits an unsigned half, every key fits 16
    # bits, and the high-multiply constant of the substitution fits 32 bits.
    for match in range(1, 128):
        for ng in range(1, 129 - match):
            x = 1536 - match
            kR = P.rebase_step(match, -ng, x)
            assert kR >= max(128, match + 2 * ng)
            thr_max = kR + P.rebase_margin(match) + 2 * match + 3 * ng - 1
            assert thr_max <= 2040
            assert P.SCALE * (thr_max + x + match) + P.SCALE * (match + 2 * ng) <= 0xFFFF
            assert P.KEY0 + P.SCALE * (x + match) + 15 <= 0xFFFF
            assert P.frame_bias(match, -ng) + ng == match + 2 * ng + 1
            assert P.SCALE * (match + 128) < 1 << 13  # mismatch >= -128
    # Lanes of 32 slots: keys in units of 32 r, thresholds <= 1016, and
    # x + match <= 1022 keeps every key within 16 bits.
    for match in range(1, 128):
        for ng in range(1, 129 - match):
            x = 1022 - match
            assert P.fits(match, -1, -ng, x, 32) and not P.fits(match, -1, -ng, x + 1, 32)
            kR = P.rebase_step(match, -ng, x, 32)
            assert kR >= max(128, match + 2 * ng)
            thr_max = kR + P.rebase_margin(match) + 2 * match + 3 * ng - 1
            assert P.key_scale(32) * thr_max <= P.KEY0
            assert P.KEY0 + P.key_scale(32) * (x + match) + 31 <= 0xFFFF
            assert 2 * P.SCALE * (thr_max + x + match) <= 0xFFFF


@pytest.mark.parametrize("lanes,regs,seed", [(4, 8, 1), (8, 4, 2), (2, 16, 3)])
def test_model_matches_oracle(orc, lanes, regs, seed):
    done = overflow = 0
    for sc, a, b in cases(seed, 48, 2 * regs):
        want = orc.extend(a, b, *sc)[:3]
        got = P.extend(a, b, *sc, lanes=lanes, regs=regs)
        if got[3]:
            overflow += 1
            continue
        assert tuple(got[:3]) == tuple(want), (sc, len(a), len(b), got, want)
        done += 1
    assert done >= 30 and overflow <= 18


@pytest.mark.parametrize("lanes,regs,scorings", [
    (4, 8, [(127, -1, -1, 1409), (64, -128, -64, 1472)]),
    (2, 16, [(127, -1, -1, 895), (64, -128, -64, 958)]),  # x + match <= 1022
])
def test_model_long_identical_reads_rebase_many_times(orc, lanes, regs, scorings):
    """Identical 1,500-base reads with the largest match: the score
    grows by up to 127 per diagonal pair, so the frame is rebased over and
    over: every 9 to 13 pairs with 16-slot lanes, every 3 to 5 with 32-slot
    ones, whose keys leave half the threshold range."""
    rng = np.random.default_rng(9)
    t = rng.integers(0, 4, 1500).astype(np.uint8)
    for sc in scorings:
        want = orc.extend(t, t, *sc)[:3]
        st = {}
        got = P.extend(t, t, *sc, lanes=lanes, regs=regs, stats=st)
        assert not got[3] and tuple(got[:3]) == tuple(want), (sc, got, want)
        assert st["rebase"] >= 100, st


def _drifting(t, rng, every):
    """t with one random base inserted after every `every` bases."""
    out = []
    for k in range(0, len(t), every):
        out.append(t[k:k + every])
        out.append(rng.integers(0, 4, 1).astype(np.uint8))
    return np.concatenate(out)


@pytest.mark.parametrize("lanes,regs", [(4, 8), (2, 8), (2, 16)])
def test_model_drifting_band_shifts_the_window(orc, lanes, regs):
    """One read gains a base every 8 (then the other does): the optimal
    path drifts one diagonal per 8 bases, so the window must shift many
    slots up in one case and down in the other while the band stays
    narrow."""
    rng = np.random.default_rng(17)
    t = rng.integers(0, 4, 480).astype(np.uint8)
    d = _drifting(t, rng, 8)
    shifted = {"up": 0, "down": 0}
    for a, b in [(t, d), (d, t)]:
        for sc in [(1, -1, -1, 20), (2, -2, -1, 30)]:
            st = {}
            got = P.extend(a, b, *sc, lanes=lanes, regs=regs, stats=st)
            assert not got[3], (sc, lanes, regs)
            assert tuple(got[:3]) == tuple(orc.extend(a, b, *sc)[:3]), (sc, lanes, regs, got)
            shifted["up"] += st["up"]
            shifted["down"] += st["down"]
    assert shifted["up"] >= 8 and shifted["down"] >= 8, shifted
