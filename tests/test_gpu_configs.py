"""The uneven stress workload (config 3) and the 100x workload streamed in
device-memory-admitted chunks (config 4), against the oracle."""
import os

import numpy as np
import pytest

from paper_2309_07270_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SYNC_NS = int(300e9)


@pytest.fixture(scope="module")
def X():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_07270_gb300 import build, xdrop
    build.build()
    return xdrop


def fixed_bytes(X, w):
    """Device bytes a batched context holds with w's reads resident."""
    ctx = X.xdrop_init(0, 0, X.XDROP_MODE_BATCHED)
    try:
        X.xdrop_load_reads(ctx, w.packed, w.read_off, w.read_len)
        return X.xdrop_get_stats(ctx)["device_bytes"]
    finally:
        X.xdrop_free(ctx)


def submit_pairs(X, ctx, w, pairs):
    out = np.zeros(len(pairs), X.RESULT_DTYPE)
    t = X.xdrop_submit_pairs(ctx, pairs, X.scoring(w.match, w.mismatch, w.gap, w.x), out)
    X.xdrop_sync(ctx, t, SYNC_NS)
    return out


def test_chunked_equals_whole(X, orc):
    w = W.genome_overlaps(genome_len=1_500_000, seed=8)
    whole_ctx = X.xdrop_init(0, 0, X.XDROP_MODE_BATCHED)
    try:
        X.xdrop_load_reads(whole_ctx, w.packed, w.read_off, w.read_len)
        whole = submit_pairs(X, whole_ctx, w, w.pairs)
        assert X.xdrop_get_stats(whole_ctx)["graph_replays"] == 1
    finally:
        X.xdrop_free(whole_ctx)
    budget = fixed_bytes(X, w) + (w.n_pairs // 6) * 80 + (1 << 16)
    ctx = X.xdrop_init(0, budget, X.XDROP_MODE_BATCHED)
    try:
        X.xdrop_load_reads(ctx, w.packed, w.read_off, w.read_len)
        chunked = submit_pairs(X, ctx, w, w.pairs)
        st = X.xdrop_get_stats(ctx)
        assert st["graph_replays"] >= 5
        assert st["device_bytes"] <= budget
    finally:
        X.xdrop_free(ctx)
    assert np.array_equal(chunked.view(np.int32), whole.view(np.int32))
    idx = np.sort(np.random.default_rng(8).choice(w.n_pairs, 300, replace=False))
    want = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs[idx], 1, -1, -1, 50,
                           nthreads=os.cpu_count() or 1)
    assert np.array_equal(chunked[idx].view(np.int32), want.view(np.int32))


def test_uneven_stress(X, orc):
    """Pareto lengths (100 bp - 50 kb), 20 % unrelated pairs: autotuned
    batched form and plain form agree with each other and the oracle."""
    w = W.uneven_pairs(n_pairs=60_000, seed=3)
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        batched = al.align(w.packed, w.read_off, w.read_len, w.pairs, X.scoring(1, -1, -1, 50))
    with X.Aligner(mode=X.XDROP_MODE_PLAIN) as al:
        plain = al.align(w.packed, w.read_off, w.read_len, w.pairs, X.scoring(1, -1, -1, 50))
    assert np.array_equal(batched.view(np.int32), plain.view(np.int32))
    idx = np.sort(np.random.default_rng(3).choice(w.n_pairs, 2000, replace=False))
    want = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs[idx], 1, -1, -1, 50,
                           nthreads=os.cpu_count() or 1)
    assert np.array_equal(batched[idx].view(np.int32), want.view(np.int32))


def test_genome_100x_streamed(X, orc):
    """The full 100x workload (about 3.7M pairs) through a context whose
    budget holds the reads and about a fifth of the pair table; 50,000
    sampled pairs against the oracle."""
    w = W.genome_overlaps(coverage=100.0, seed=4)
    budget = fixed_bytes(X, w) + (w.n_pairs // 5) * 80 + (1 << 16)
    ctx = X.xdrop_init(0, budget, X.XDROP_MODE_BATCHED)
    try:
        X.xdrop_load_reads(ctx, w.packed, w.read_off, w.read_len)
        got = submit_pairs(X, ctx, w, w.pairs)
        st = X.xdrop_get_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    assert st["graph_replays"] >= 5
    assert (got["status"] == 0).all()
    idx = np.sort(np.random.default_rng(4).choice(w.n_pairs, 50_000, replace=False))
    want = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs[idx], 1, -1, -1, 50,
                           nthreads=os.cpu_count() or 1)
    assert np.array_equal(got[idx].view(np.int32), want.view(np.int32))
