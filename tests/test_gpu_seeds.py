"""Seed discovery on the GPU (xdrop_find_candidates: reliable k-mers and
candidate read pairs) against the oracle (oracle/seeds.py), record for
record: the sort-based product here, the row-wise one (the default) in
test_gpu_seeds_rowwise.py, both at the paper's parameters (k = 31, stride
1, frequency window [20, 50], 29x coverage); and the candidates aligned
through xdrop_submit_pairs against the oracle's alignments."""
import ctypes

import numpy as np
import pytest

from oracle import seeds as S
from paper_2309_07270_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_07270_gb300 import build, xdrop
    build.build()
    return xdrop


def as_candidates(pairs, shared):
    out = np.zeros(len(pairs), S.CANDIDATE)
    for f in ("a", "b", "seed_a", "seed_b", "seed_len"):
        out[f] = pairs[f]
    out["shared"] = shared
    return out


def gpu(X, packed, off, lens, k, lo, hi, stride=1, rowwise=False, expect_product=None):
    """Candidates from the library; checks which product ran (the row-wise
    one unless a read overflows its table, or nothing to pair)."""
    with X.Aligner() as al:
        got = as_candidates(*al.find_candidates(packed, off, lens, k=k, lo=lo, hi=hi,
                                                stride=stride, rowwise=rowwise))
        st = X.xdrop_get_seed_stats(al.ctx)
    assert st["candidates"] == len(got)
    if expect_product is None:
        expect_product = X.XDROP_SEEDS_ROWWISE if rowwise else X.XDROP_SEEDS_SORT
    if st["runs"] > 0:
        assert st["product"] == expect_product
    return got


def same(got, want):
    assert len(got) == len(want)
    assert np.array_equal(got, want)


def pack(reads):
    return W.pack_reads([np.asarray(r, np.uint8) for r in reads])


def small_genome_reads(n_reads, seed, glen=400, lo=20, hi=160, rc_frac=0.4, err=True):
    rng = np.random.default_rng(seed)
    g = rng.integers(0, 4, glen).astype(np.uint8)
    reads = []
    for _ in range(n_reads):
        n = int(rng.integers(lo, hi + 1))
        s = int(rng.integers(0, glen - n + 1))
        r = W.mutate(g[s:s + n], rng)[0] if err else g[s:s + n].copy()
        reads.append(W.revcomp(r) if rng.random() < rc_frac else r)
    return reads


@pytest.mark.parametrize("k", [1, 3, 7, 16, 17, 31, 32])
@pytest.mark.parametrize("stride", [1, 3])
def test_small_sweep(X, k, stride):
    reads = small_genome_reads(9, seed=k * 10 + stride, err=k < 15)
    packed, off, lens = pack(reads)
    for lo, hi in ((1, 1024), (2, 5)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi, stride=stride)
        same(gpu(X, packed, off, lens, k, lo, hi, stride), want)


def repeat_reads():
    rng = np.random.default_rng(5)
    unit = rng.integers(0, 4, 7).astype(np.uint8)
    return [np.tile(unit, 12)[:80], np.zeros(0, np.uint8), np.tile(unit, 9)[3:60],
            W.revcomp(np.tile(unit, 10)[1:66]), rng.integers(0, 4, 90).astype(np.uint8),
            unit[:4].copy()]


def test_repeats_short_and_empty_reads(X):
    packed, off, lens = pack(repeat_reads())
    for k, lo, hi in ((5, 1, 1024), (9, 2, 30), (9, 20, 40), (4, 3, 1024)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi)
        same(gpu(X, packed, off, lens, k, lo, hi), want)


def test_medium_read_set(X):
    """Error-model reads of a 100 kb genome at 10x, both strands (1 Mb):
    many thread blocks in every kernel, thousands of candidates."""
    packed, off, lens = W.sequencing_reads(100_000, 10, 3_000, 1_500, 500, seed=8)
    for k, lo, hi in ((17, 2, 30), (15, 3, 12)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi)
        assert len(want) > 1000
        same(gpu(X, packed, off, lens, k, lo, hi), want)


def test_candidates_align_like_the_oracle(X, orc):
    """Seed discovery feeds seed-and-extend: the candidates, reverse-strand
    ones included, go to xdrop_submit_pairs as they are."""
    packed, off, lens = W.sequencing_reads(40_000, 8, 2_500, 1_000, 500, seed=21)
    sc = X.scoring(1, -1, -1, 30)
    with X.Aligner() as al:
        pairs, _ = al.find_candidates(packed, off, lens, k=17, lo=2, hi=20)
        assert len(pairs) > 100 and (pairs["b"] >> 31).sum() > 10
        out = np.zeros(len(pairs), X.RESULT_DTYPE)
        X.xdrop_sync(al.ctx, X.xdrop_submit_pairs(al.ctx, pairs, sc, out))
    want = orc.align_pairs(packed, off, lens, pairs, 1, -1, -1, 30)
    for f in X.RESULT_DTYPE.names:
        assert np.array_equal(out[f], want[f]), f


def test_result_cache_and_errors(X):
    reads = small_genome_reads(12, seed=4, err=False)
    packed, off, lens = pack(reads)
    want13 = S.candidate_pairs(packed, off, lens, k=13, lo=1, hi=1024)
    want9 = S.candidate_pairs(packed, off, lens, k=9, lo=2, hi=6)
    with X.Aligner() as al:
        X.xdrop_load_reads(al.ctx, packed, off, lens)
        same(as_candidates(*X.xdrop_find_candidates(al.ctx, 13, 1, 1024)), want13)
        same(as_candidates(*X.xdrop_find_candidates(al.ctx, 9, 2, 6)), want9)   # new params
        same(as_candidates(*X.xdrop_find_candidates(al.ctx, 13, 1, 1024)), want13)
        st = X.xdrop_get_seed_stats(al.ctx)
        assert st["product"] == X.XDROP_SEEDS_ROWWISE  # the default
        assert st["nonzeros"] > 0
        # a short output buffer gets the first records and the total
        prm = X.KmerParams(13, 1, 1, 1024, 0)
        buf = np.zeros(3, X.PAIR_DTYPE)
        n = ctypes.c_size_t()
        assert X.load().xdrop_find_candidates(al.ctx, ctypes.byref(prm), X._p(buf), None, 3,
                                              ctypes.byref(n)) == X.XDROP_OK
        assert n.value == len(want13) and len(want13) > 3
        for f in ("a", "b", "seed_a", "seed_b", "seed_len"):
            assert np.array_equal(buf[f], want13[f][:3])
        # a new read set replaces the cached result
        p2, o2, l2 = pack(reads[:5])
        X.xdrop_load_reads(al.ctx, p2, o2, l2)
        same(as_candidates(*X.xdrop_find_candidates(al.ctx, 13, 1, 1024)),
             S.candidate_pairs(p2, o2, l2, k=13, lo=1, hi=1024))
        for k, lo, hi, stride in ((0, 1, 10, 1), (33, 1, 10, 1), (13, 5, 4, 1), (13, 1, 1025, 1),
                                  (13, 0, 4, 1), (13, 1, 4, 0)):
            with pytest.raises(X.XdropError) as e:
                X.xdrop_find_candidates(al.ctx, k, lo, hi, stride)
            assert e.value.code == X.XDROP_EINVAL
        bad = X.KmerParams(13, 1, 1, 10, 2)   # unknown product flag
        assert X.load().xdrop_find_candidates(al.ctx, ctypes.byref(bad), None, None, 0,
                                              ctypes.byref(n)) == X.XDROP_EINVAL
    with X.Aligner() as al:  # no resident reads
        with pytest.raises(X.XdropError) as e:
            X.xdrop_find_candidates(al.ctx, 13, 1, 10)
        assert e.value.code == X.XDROP_EINVAL


@pytest.fixture(scope="module")
def paper29():
    """k = 31, window [20, 50], 29x coverage of a 100 kb genome with
    accurate reads (1% errors; at 12% almost no 31-mer reaches a count of
    20): about 3 Mb in 290 reads, and the oracle's candidates (about a
    minute on one core)."""
    packed, off, lens = W.sequencing_reads(100_000, 29, 10_000, 6_000, 1_000, seed=29,
                                           error_rate=0.01)
    packed = np.ascontiguousarray(packed, np.uint32)
    off = np.ascontiguousarray(off, np.uint64)
    lens = np.ascontiguousarray(lens, np.uint32)
    return packed, off, lens, S.candidate_pairs(packed, off, lens, k=31, lo=20, hi=50)


@pytest.mark.parametrize("rowwise", [False, True], ids=["sort", "rowwise"])
def test_paper_parameters_29x(X, paper29, rowwise):
    """The paper's seed parameters: both products equal the oracle record
    for record; every candidate is a pair a < b in (a, b) order and its
    seed is an exact k-mer match on the strand it names."""
    packed, off, lens, want = paper29
    assert len(want) > 1000 and (want["b"] >> 31).sum() > 100
    got = gpu(X, packed, off, lens, 31, 20, 50, rowwise=rowwise)
    same(got, want)
    key = got["a"].astype(np.int64) * len(lens) + (got["b"] & 0x7FFFFFFF)
    assert np.all(np.diff(key) > 0) and np.all(got["a"] < (got["b"] & 0x7FFFFFFF))
    assert np.all(got["seed_len"] == 31) and np.all(got["shared"] >= 1)
    w = W.Workload("reads", packed, off, lens, np.zeros(0, W.PAIR_DTYPE))
    for c in got:
        a = w.codes(int(c["a"]))
        b = w.codes(int(c["b"]) & 0x7FFFFFFF)
        if c["b"] >> 31:
            b = W.revcomp(b)
        sa, sb = int(c["seed_a"]), int(c["seed_b"])
        assert np.array_equal(a[sa:sa + 31], b[sb:sb + 31])
