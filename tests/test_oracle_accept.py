"""Pins of the oracle's adaptive acceptance (oracle.accept) against values
worked out by hand and against invariants of the threshold."""
import numpy as np

from paper_2309_07270_gb300 import workloads as W


def one(orc, total_right, seed_a=0, seed_b=0, len_a=1000, len_b=1000, seed_len=17, left=0,
        status=0, b_flag=0, **kw):
    pairs = np.zeros(1, orc.ORC_PAIR)
    pairs[0] = (0, 1 | b_flag, seed_a, seed_b, seed_len)
    res = np.zeros(1, orc.ORC_RESULT)
    res["left_score"] = left
    res["right_score"] = total_right
    res["status"] = status
    return int(orc.accept(pairs, res, np.array([len_a, len_b], np.uint32), **kw)[0])


def test_hand_example_error_15_percent(orc):
    """e = 0.15, delta = 0.1, +1/-1, overlap 1,000: phi = 0.7225, expected
    0.445 per column, threshold 0.9 * 445 = 400.5.  Seed 17 + right 383 =
    400 is rejected, 401 accepted."""
    kw = dict(match=1, mismatch=-1, error_e4=1500, delta_e4=1000)
    assert one(orc, 383, **kw) == 0
    assert one(orc, 384, **kw) == 1


def test_exact_reads_need_the_full_score(orc):
    """e = 0, delta = 0: the threshold is L * match exactly."""
    kw = dict(match=2, mismatch=-3, error_e4=0, delta_e4=0)
    # L = min(100, 30) + min(500 - 100, 200 - 30) = 30 + 170 = 200: threshold 400
    geo = dict(seed_a=100, seed_b=30, len_a=500, len_b=200, seed_len=10, left=60)
    assert one(orc, 400 - 60 - 20, **geo, **kw) == 1
    assert one(orc, 400 - 60 - 20 - 1, **geo, **kw) == 0
    # the strand flag on b changes nothing: positions are on the named strand
    assert one(orc, 400 - 60 - 20, b_flag=W.PAIR_RC, **geo, **kw) == 1


def test_full_slack_accepts_every_nonnegative_score(orc):
    kw = dict(match=1, mismatch=-1, error_e4=1500, delta_e4=10_000)
    assert one(orc, -17, **kw) == 1      # total 0
    assert one(orc, -18, **kw) == 0      # total -1


def test_failed_alignments_are_never_accepted(orc):
    kw = dict(match=1, mismatch=-1, error_e4=0, delta_e4=10_000)
    assert one(orc, 10_000, status=1, **kw) == 0
    assert one(orc, 10_000, status=2, **kw) == 0


def test_threshold_monotone_in_slack_and_error(orc):
    """More slack or a higher assumed error rate never rejects a pair that
    was accepted (for mismatch < match)."""
    rng = np.random.default_rng(3)
    n = 400
    pairs = np.zeros(n, orc.ORC_PAIR)
    pairs["a"] = 0
    pairs["b"] = 1
    pairs["seed_a"] = rng.integers(0, 800, n)
    pairs["seed_b"] = rng.integers(0, 800, n)
    pairs["seed_len"] = 17
    res = np.zeros(n, orc.ORC_RESULT)
    res["right_score"] = rng.integers(-50, 900, n)
    lens = np.array([900, 900], np.uint32)
    prev = None
    for d in (0, 500, 1000, 3000, 10_000):
        cur = orc.accept(pairs, res, lens, 1, -1, 1500, d)
        if prev is not None:
            assert np.all(cur >= prev)
        prev = cur
    prev = None
    for e in (0, 500, 1500, 3000):
        cur = orc.accept(pairs, res, lens, 1, -1, e, 1000)
        if prev is not None:
            assert np.all(cur >= prev)
        prev = cur
    assert 0 < prev.sum() < n
