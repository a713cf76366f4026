"""GPU parity: the CUDA path against the oracle, element by element.

Every field of every result (scores, coordinates, status) must be identical
(integer work: bit-exact).  Cell counts from the library's counting pass
must equal the oracle's.  Inputs are seeded synthetic workloads.
"""
import dataclasses

import numpy as np
import pytest

from paper_2309_07270_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODES = ["plain", "batched"]


@pytest.fixture(scope="module")
def X():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_07270_gb300 import build, xdrop
    build.build()
    return xdrop


@pytest.fixture(scope="module")
def aligners(X):
    al = {"plain": X.Aligner(mode=X.XDROP_MODE_PLAIN),
          "batched": X.Aligner(mode=X.XDROP_MODE_BATCHED)}
    yield al
    for a in al.values():
        a.close()


def oracle_results(orc, w, x=None, nthreads=8, cells=False):
    x = w.x if x is None else x
    return orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs, w.match, w.mismatch,
                           w.gap, x, nthreads=nthreads, with_cells=cells)


def assert_same(got, want, what=""):
    g = got.view(np.int32).reshape(-1, 7)
    e = want.view(np.int32).reshape(-1, 7)
    bad = np.flatnonzero((g != e).any(axis=1))
    assert bad.size == 0, f"{what}: {bad.size} pairs differ, first {bad[:5]}: gpu {g[bad[:3]]} oracle {e[bad[:3]]}"


def run_host(X, al, w):
    return al.align(w.packed, w.read_off, w.read_len, w.pairs,
                    X.scoring(w.match, w.mismatch, w.gap, w.x))


@pytest.mark.parametrize("mode", MODES)
def test_template_pairs_200(X, aligners, orc, mode):
    """200 template pairs, 2-4 kb, 12 % errors, X = 50, +1/-1/-1."""
    w = W.template_pairs()
    assert_same(run_host(X, aligners[mode], w), oracle_results(orc, w), mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("x", [0, 1, 7, 20])
def test_tiny_and_ragged(X, aligners, orc, mode, x):
    """Lengths 0..200 around the seed: empty extensions, ragged bands."""
    w = W.tiny_pairs(n_pairs=300, seed=11 + x, x=x)
    assert_same(run_host(X, aligners[mode], w), oracle_results(orc, w), f"{mode} x={x}")


def _edge_workload(rng, x):
    seqs_a, seqs_b, seeds = [], [], []
    def add(a, b, sa, sb, L):
        seqs_a.append(np.asarray(a, np.uint8)); seqs_b.append(np.asarray(b, np.uint8)); seeds.append((sa, sb, L))
    t = rng.integers(0, 4, 3000).astype(np.uint8)
    add(t, t, 0, 0, 17)                      # seed at both read starts
    add(t, t, 3000 - 17, 3000 - 17, 17)      # seed at both read ends
    add(t, t, 1500, 1500, 17)                # identical reads
    add(t[:17], t[:17], 0, 0, 17)            # reads equal to the seed
    add(t[:18], t[:17], 1, 0, 17)            # one base on one side
    u = rng.integers(0, 4, 2000).astype(np.uint8)
    v = (u + 1) & 3                          # every base mismatches
    add(np.concatenate([u, t[:17], u]), np.concatenate([v, t[:17], v]), 2000, 2000, 17)
    r1 = rng.integers(0, 4, 2500).astype(np.uint8)
    r2 = rng.integers(0, 4, 1800).astype(np.uint8)
    add(r1, r2, 700, 900, 0)                 # unrelated reads, empty seed
    add(t, t[::-1].copy(), 100, 2000, 5)     # unrelated orientation
    a, *_ = W.mutate(t, rng)
    b, *_ = W.mutate(t, rng)
    add(a, b, 0, 0, 0)                       # seedless start, related reads
    add(a, b, len(a) - 1, len(b) - 1, 1)     # 1-base seed at the ends
    return W.from_sequences(seqs_a, seqs_b, seeds, x=x)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("x", [0, 3, 50, 100])
def test_edge_cases(X, aligners, orc, mode, x):
    w = _edge_workload(np.random.default_rng(x), x)
    assert_same(run_host(X, aligners[mode], w), oracle_results(orc, w), f"{mode} x={x}")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scores", [(2, -3, -2), (1, 0, -1), (5, -4, -3)])
def test_other_scorings(X, aligners, orc, mode, scores):
    w = W.template_pairs(n_pairs=40, len_lo=300, len_hi=1500, seed=4)
    w.match, w.mismatch, w.gap = scores
    w.x = 30
    assert_same(run_host(X, aligners[mode], w), oracle_results(orc, w), f"{mode} {scores}")


P16 = 0x100  # XDROP_TILE_PACKED16
TILES = [(4, 16), (8, 8), (16, 4), (8, 16), (16, 8), (32, 4),
         (4, 8 | P16), (2, 16 | P16), (4, 16 | P16), (8, 8 | P16), (8, 16 | P16), (16, 8 | P16),
         (2, 32 | P16), (4, 32 | P16)]


def tile_id(t):
    return f"{t[0]}x{t[1] & 0xff}" + ("p16" if t[1] & P16 else "")


@pytest.mark.parametrize("tile", TILES, ids=tile_id)
def test_every_first_tile(X, orc, tile):
    """Each first-tier tile (forced, no autotuning) is exact on long,
    ragged and wide-band inputs."""
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.set_tile(*tile)
        for w in (W.template_pairs(n_pairs=60, seed=21),
                  W.tiny_pairs(n_pairs=200, seed=22, x=9),
                  W.template_pairs(n_pairs=16, len_lo=500, len_hi=900, seed=23, x=300)):
            got = run_host(X, al, w)
            assert al.tile() == tile
            assert_same(got, oracle_results(orc, w), f"tile {tile} {w.name}")


PACKED_LIMIT_SCORINGS = [
    (64, -128, -64, 1472),  # every limit at once: the frame is rebased every diagonal pair
    (1, -2, -1, 1535),      # largest x, mismatch = 2 gap
    (3, -2, -125, 100),     # gap-dominated frame growth
    (127, -1, -1, 1409),    # largest match
    (1, 0, -1, 50),         # mismatch + 2|gap| > 0
    (7, -1, -2, 0),         # x = 0
]


@pytest.mark.parametrize("scores", PACKED_LIMIT_SCORINGS, ids=lambda s: "_".join(map(str, s)))
@pytest.mark.parametrize("tile", [(4, 16 | P16), (8, 8 | P16)], ids=tile_id)
def test_packed_tiles_at_their_limits(X, orc, tile, scores):
    """Scorings at the edges of the packed 16-bit range stay exact, on long
    near-identical pairs (scores and the normalised frame grow fast) and on
    ragged ones."""
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.set_tile(*tile)
        for w in (W.template_pairs(n_pairs=24, len_lo=1500, len_hi=3000, seed=31),
                  W.tiny_pairs(n_pairs=150, seed=32, x=9)):
            w.match, w.mismatch, w.gap, w.x = scores
            got = run_host(X, al, w)
            assert al.tile() == tile
            assert_same(got, oracle_results(orc, w), f"{tile_id(tile)} {scores} {w.name}")


# The same limits for the tiles of 32 cells per lane, whose keys also need
# x + match <= 1022.
PACKED32_LIMIT_SCORINGS = [
    (64, -128, -64, 958),   # every limit at once
    (1, -2, -1, 1021),      # largest x
    (3, -2, -125, 100),
    (127, -1, -1, 895),     # largest match
    (1, 0, -1, 50),
    (7, -1, -2, 0),
]


@pytest.mark.parametrize("scores", PACKED32_LIMIT_SCORINGS, ids=lambda s: "_".join(map(str, s)))
@pytest.mark.parametrize("tile", [(2, 32 | P16), (4, 32 | P16)], ids=tile_id)
def test_packed32_tiles_at_their_limits(X, orc, tile, scores):
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.set_tile(*tile)
        for w in (W.template_pairs(n_pairs=24, len_lo=1500, len_hi=3000, seed=34),
                  W.tiny_pairs(n_pairs=150, seed=35, x=9)):
            w.match, w.mismatch, w.gap, w.x = scores
            got = run_host(X, al, w)
            assert al.tile() == tile
            assert_same(got, oracle_results(orc, w), f"{tile_id(tile)} {scores} {w.name}")


@pytest.mark.parametrize("scores,want_tile", [((1, -1, -1, 1022), (4, 16 | P16)),
                                              ((127, -1, -1, 896), (4, 16 | P16)),
                                              ((1, -3, -1, 30), (4, 16))],
                         ids=["x1022", "match127_x896", "not16bit"])
def test_packed32_tile_falls_back_outside_its_range(X, orc, scores, want_tile):
    """A forced 2x32 packed tile runs the packed 4x16 tile (same width) when
    x + match exceeds 1022, and the 32-bit 4x16 tile when the scoring does
    not fit 16 bits at all; the results are the same."""
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.set_tile(2, 32 | P16)
        w = W.template_pairs(n_pairs=12, len_lo=300, len_hi=800, seed=36)
        w.match, w.mismatch, w.gap, w.x = scores
        got = run_host(X, al, w)
        assert al.tile() == want_tile
        assert_same(got, oracle_results(orc, w), f"fallback {scores}")


@pytest.mark.parametrize("scores", [(1, -1, -1, 1536), (128, -1, -1, 10), (1, -129, -1, 10),
                                    (1, -1, -128, 10), (1, -128, -1, 1535), (2, -3, -1, 30)],
                         ids=lambda s: "_".join(map(str, s)))
def test_packed_tile_falls_back_outside_its_range(X, orc, scores):
    """A forced packed tile runs the 32-bit tile of its shape when the
    scoring does not fit 16 bits, with the same results."""
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.set_tile(4, 16 | P16)
        w = W.template_pairs(n_pairs=12, len_lo=300, len_hi=800, seed=33)
        w.match, w.mismatch, w.gap, w.x = scores
        got = run_host(X, al, w)
        assert al.tile() == (4, 16)
        assert_same(got, oracle_results(orc, w), f"fallback {scores}")


@pytest.mark.parametrize("mode", MODES)
def test_wide_bands_use_every_tier(X, aligners, orc, mode):
    """Large X widens the live band past the 64-, 128- and 512-slot
    windows, so tasks spill to the wider tiers and to the unbounded one."""
    w = W.template_pairs(n_pairs=24, len_lo=600, len_hi=1400, seed=9)
    for x in (150, 400, 1500):
        wx = w.with_x(x)
        got = run_host(X, aligners[mode], wx)
        st = aligners[mode].stats()
        assert_same(got, oracle_results(orc, wx), f"{mode} x={x}")
        if x >= 400:
            assert st["overflow_tasks"] > 0
        if x >= 1500:
            assert st["wide_tasks"] > 0


@pytest.mark.parametrize("mode", MODES)
def test_device_submit_and_invalid_pairs(X, aligners, orc, mode):
    w = W.template_pairs(n_pairs=64, len_lo=500, len_hi=1500, seed=12)
    want = oracle_results(orc, w)
    bad = w.pairs.copy()
    bad[5]["seed_a"] = w.read_len[bad[5]["a"]]  # seed past the read end
    bad[9]["b"] = w.n_reads + 3                 # missing read
    dev = X.DeviceInputs(w.packed, w.read_off, w.read_len, bad)
    al = aligners[mode]
    with pytest.raises(X.XdropError) as ei:
        al.align_device(dev, X.scoring(w.match, w.mismatch, w.gap, w.x))
    assert ei.value.code == X.XDROP_EINVAL
    got = dev.results()
    ok = np.ones(w.n_pairs, bool)
    ok[[5, 9]] = False
    assert (got["status"][~ok] == X.XDROP_STATUS_INVALID).all()
    assert (got.view(np.int32).reshape(-1, 7)[~ok, :6] == 0).all()
    assert_same(got[ok], want[ok], mode)
    # the host path rejects the same input before launching anything
    out = np.zeros(w.n_pairs, X.RESULT_DTYPE)
    with pytest.raises(X.XdropError) as ei:
        X.xdrop_submit(al.ctx, w.packed, w.read_off, w.read_len, bad,
                       X.scoring(1, -1, -1, 50), out)
    assert ei.value.code == X.XDROP_EINVAL


def test_bad_scoring_rejected(X, aligners):
    w = W.tiny_pairs(n_pairs=4)
    for sc in [(0, -1, -1, 5), (1, 1, -1, 5), (1, -1, 0, 5), (1, -1, -1, -1)]:
        with pytest.raises(X.XdropError) as ei:
            aligners["batched"].align(w.packed, w.read_off, w.read_len, w.pairs, X.scoring(*sc))
        assert ei.value.code == X.XDROP_EINVAL


def test_empty_submit(X, aligners):
    w = W.tiny_pairs(n_pairs=4)
    for al in aligners.values():
        got = al.align(w.packed, w.read_off, w.read_len, w.pairs[:0], X.scoring())
        assert got.shape == (0,)


def test_cell_counts_match_oracle(X, aligners, orc):
    w = W.template_pairs(n_pairs=60, len_lo=200, len_hi=3000, seed=13)
    for x in (0, 20, 50, 700):
        wx = w.with_x(x)
        _, want = oracle_results(orc, wx, cells=True)
        dev = X.DeviceInputs.from_workload(wx)
        got = aligners["batched"].count_cells_device(dev, X.scoring(1, -1, -1, x)).cpu().numpy()
        assert np.array_equal(got.reshape(-1, 2), want), f"x={x}"


def test_modes_agree_and_repeat(X, aligners):
    """Plain and batched forms give identical results, twice in a row."""
    w = W.template_pairs(n_pairs=300, len_lo=200, len_hi=5000, seed=14)
    r = [run_host(X, aligners[m], w) for m in MODES for _ in range(2)]
    for k in range(1, 4):
        assert np.array_equal(r[0], r[k])


@pytest.mark.parametrize("mode", MODES)
def test_reverse_strand_pairs(X, aligners, orc, mode):
    """Half the pairs on the reverse strand (read b stored reverse-
    complemented, XDROP_PAIR_RC set): identical to the oracle and to the
    forward workload's results."""
    w = W.template_pairs(n_pairs=60, len_lo=500, len_hi=2500, seed=41)
    r = W.reverse_strand(w, 0.5, 3)
    got = run_host(X, aligners[mode], r)
    assert_same(got, oracle_results(orc, r), f"{mode} reverse strand")
    assert np.array_equal(got.view(np.int32), run_host(X, aligners[mode], w).view(np.int32))


def test_reverse_strand_resident_reads_and_device_submit(X, orc):
    """Over resident reads (xdrop_submit_pairs) reverse-strand pairs are
    exact; a device submit marks them invalid and keeps the others exact."""
    w = W.reverse_strand(W.template_pairs(n_pairs=40, len_lo=500, len_hi=2000, seed=42), 0.5, 4)
    sc = X.scoring(1, -1, -1, 50)
    rcm = (w.pairs["b"] >> 31) == 1
    assert rcm.sum() >= 10
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        X.xdrop_load_reads(al.ctx, w.packed, w.read_off, w.read_len)
        out = np.zeros(w.n_pairs, X.RESULT_DTYPE)
        X.xdrop_sync(al.ctx, X.xdrop_submit_pairs(al.ctx, w.pairs, sc, out))
        assert_same(out, oracle_results(orc, w), "resident reverse strand")
        dev = X.DeviceInputs.from_workload(w)
        with pytest.raises(X.XdropError) as ei:
            al.align_device(dev, sc)
        assert ei.value.code == X.XDROP_EINVAL
        res = dev.results()
    assert (res["status"][rcm] == X.XDROP_STATUS_INVALID).all()
    assert_same(res[~rcm], oracle_results(orc, w.subset(np.flatnonzero(~rcm))), "device forward")


def test_best_seeds_device(X, orc):
    """Several seeds per read pair: groups of 1-5 consecutive records with
    the same reads, half of them at random (usually worse) seed positions;
    the alignments and the device selection equal the oracle's."""
    base = W.template_pairs(n_pairs=40, len_lo=600, len_hi=1500, seed=44)
    rng = np.random.default_rng(45)
    recs = []
    for p in base.pairs:
        la, lb = int(base.read_len[p["a"]]), int(base.read_len[p["b"]])
        for _ in range(int(rng.integers(1, 6))):
            q = p.copy()
            if rng.random() < 0.5:  # another (random, usually worse) seed on the same reads
                q["seed_a"] = rng.integers(0, la - 17)
                q["seed_b"] = rng.integers(0, lb - 17)
            recs.append(q)
    w = base.subset(np.zeros(0, int))
    w = dataclasses.replace(w, pairs=np.array(recs, dtype=base.pairs.dtype))
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.align_device(dev, X.scoring(1, -1, -1, 50))
        best = al.best_seeds_device(dev, 1).cpu().numpy().view(np.uint32)
    res = dev.results()
    assert_same(res, oracle_results(orc, w), "multi-seed alignments")
    want = orc.best_seeds(w.pairs, res, match=1)
    assert np.array_equal(best, want)
    assert len(np.unique(want)) < len(want)  # groups of several seeds were reduced
