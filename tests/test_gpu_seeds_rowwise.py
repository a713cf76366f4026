"""The row-wise product of seed discovery (XDROP_SEEDS_ROWWISE, the default)
on the GPU against the oracle, including the fallback to the sort-based
product when a read's shared-memory table overflows.  The paper's
parameters are tested for both products in test_gpu_seeds.py."""
import numpy as np
import pytest

from oracle import seeds as S
from paper_2309_07270_gb300 import workloads as W

from test_gpu_seeds import (X, as_candidates, gpu, pack, repeat_reads,  # noqa: F401
                               same, small_genome_reads)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 3, 7, 16, 17, 31, 32])
@pytest.mark.parametrize("stride", [1, 3])
def test_rowwise_small_sweep(X, k, stride):
    reads = small_genome_reads(9, seed=k * 10 + stride, err=k < 15)
    packed, off, lens = pack(reads)
    for lo, hi in ((1, 1024), (2, 5)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi, stride=stride)
        same(gpu(X, packed, off, lens, k, lo, hi, stride, rowwise=True), want)


def test_rowwise_repeats_short_and_empty_reads(X):
    packed, off, lens = pack(repeat_reads())
    for k, lo, hi in ((5, 1, 1024), (9, 2, 30), (9, 20, 40), (4, 3, 1024)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi)
        same(gpu(X, packed, off, lens, k, lo, hi, rowwise=True), want)


def test_rowwise_medium_read_set(X):
    packed, off, lens = W.sequencing_reads(100_000, 10, 3_000, 1_500, 500, seed=8)
    want = S.candidate_pairs(packed, off, lens, k=17, lo=2, hi=30)
    same(gpu(X, packed, off, lens, 17, 2, 30, rowwise=True), want)


def test_rowwise_result_cache(X):
    reads = small_genome_reads(12, seed=4, err=False)
    packed, off, lens = pack(reads)
    want13 = S.candidate_pairs(packed, off, lens, k=13, lo=1, hi=1024)
    with X.Aligner() as al:
        X.xdrop_load_reads(al.ctx, packed, off, lens)
        same(as_candidates(*X.xdrop_find_candidates(al.ctx, 13, 1, 1024, rowwise=True)), want13)
        assert X.xdrop_get_seed_stats(al.ctx)["product"] == X.XDROP_SEEDS_ROWWISE
        same(as_candidates(*X.xdrop_find_candidates(al.ctx, 13, 1, 1024, rowwise=False)), want13)
        assert X.xdrop_get_seed_stats(al.ctx)["product"] == X.XDROP_SEEDS_SORT


def star_reads(n_leaves, seed=12, k=8):
    """Read 0 holds many distinct k-mers; every other read is a copy of one
    of them, round robin: read 0 pairs with all n_leaves reads."""
    rng = np.random.default_rng(seed)
    while True:
        hub = rng.integers(0, 4, 160).astype(np.uint8)
        codes = S.occurrences([hub.tolist()], k)
        if len({c for c, *_ in codes}) == len(codes):
            break
    n_k = len(hub) - k + 1
    return [hub] + [hub[i % n_k:i % n_k + k].copy() for i in range(n_leaves)]


def test_rowwise_table_overflow_falls_back(X):
    """2,100 partners of one read overflow the 2,048-slot table: the call
    runs the sort-based product and still gives the oracle's candidates;
    2,000 partners fit."""
    for n_leaves, product in ((2100, X.XDROP_SEEDS_SORT), (2000, X.XDROP_SEEDS_ROWWISE)):
        packed, off, lens = pack(star_reads(n_leaves))
        want = S.candidate_pairs(packed, off, lens, k=8, lo=1, hi=1024)
        assert (want["a"] == 0).sum() == n_leaves
        same(gpu(X, packed, off, lens, 8, 1, 1024, rowwise=True, expect_product=product), want)
