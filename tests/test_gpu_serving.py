"""Serving (continuous batching) on the GPU.

Requests of read pairs from 25 producer threads go to one persistent
serving kernel.  Each request's results must be identical (integers,
tolerance 0) whether it runs alone or in the mix, and equal to the oracle.
Memory admission must queue requests that do not fit the budget and refuse
one that never can.  Extensions whose band outgrows the serving tile must
go through the wider tiers and stay exact.
"""
import threading
import time

import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def pool():
    """A small genome-overlap pool (1 Mbp genome, 29x)."""
    return W.genome_overlaps(genome_len=1_000_000, seed=5)


def requests_for(pool, n_producers=25, per_producer=3, lo=50, hi=600, seed=100):
    reqs = []
    for p in range(n_producers):
        rng = np.random.Generator(np.random.PCG64(seed + p))
        for _ in range(per_producer):
            k = int(rng.integers(lo, hi + 1))
            reqs.append((p, rng.integers(0, pool.n_pairs, size=k)))
    return reqs


def serve_ctx(X, pool, budget=0, tile=None):
    ctx = X.xdrop_init(0, budget, X.XDROP_MODE_SERVE)
    if tile:
        X.xdrop_set_tile(ctx, *tile)
    X.xdrop_load_reads(ctx, pool.packed, pool.read_off, pool.read_len)
    return ctx


SYNC_NS = int(60e9)  # a request that takes longer fails the test with the loop's counters


def sync(X, ctx, t):
    try:
        X.xdrop_sync(ctx, t, SYNC_NS)
    except X.XdropError as e:
        raise AssertionError(f"{e}; serving counters {X.xdrop_get_serve_stats(ctx)}") from e


def run_alone(X, ctx, pool, reqs, sc):
    outs = []
    for _, idx in reqs:
        out = np.zeros(len(idx), X.RESULT_DTYPE)
        t = X.xdrop_submit_pairs(ctx, pool.pairs[idx], sc, out)
        sync(X, ctx, t)
        outs.append(out)
    return outs


def run_mix(X, ctx, pool, reqs, sc, n_producers=25):
    """Every producer thread submits all its requests back to back, then
    syncs them; all producers run at once."""
    outs = [None] * len(reqs)
    errors = []
    by_prod = {}
    for i, (p, idx) in enumerate(reqs):
        by_prod.setdefault(p, []).append(i)

    def producer(items):
        try:
            tickets = []
            for i in items:
                out = np.zeros(len(reqs[i][1]), X.RESULT_DTYPE)
                outs[i] = out
                tickets.append(X.xdrop_submit_pairs(ctx, pool.pairs[reqs[i][1]], sc, out))
                time.sleep(0.001)
            for t in tickets:
                sync(X, ctx, t)
        except Exception as e:  # surfaced below
            errors.append(e)

    th = [threading.Thread(target=producer, args=(items,)) for items in by_prod.values()]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    assert all(not t.is_alive() for t in th)
    return outs


def test_alone_equals_mix_equals_oracle(X, orc, pool):
    reqs = requests_for(pool)
    sc = X.scoring(1, -1, -1, 50)
    ctx = serve_ctx(X, pool)
    try:
        alone = run_alone(X, ctx, pool, reqs, sc)
        mix = run_mix(X, ctx, pool, reqs, sc)
        st = X.xdrop_get_serve_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    for a, b in zip(alone, mix):
        assert np.array_equal(a.view(np.int32), b.view(np.int32))
    assert st["requests_done"] == 2 * len(reqs)
    assert st["max_in_flight"] > 1  # requests overlapped on the device
    # oracle on a sample of requests
    for k in range(0, len(reqs), 9):
        idx = reqs[k][1]
        want = orc.align_pairs(pool.packed, pool.read_off, pool.read_len, pool.pairs[idx],
                               1, -1, -1, 50, nthreads=8)
        assert np.array_equal(alone[k].view(np.int32), want.view(np.int32))


def test_memory_admission_queues_and_refuses(X, orc, pool):
    reqs = requests_for(pool, n_producers=6, per_producer=3, lo=200, hi=400, seed=300)
    sc = X.scoring(1, -1, -1, 50)
    budget = 64 * 1024  # two or three requests' buffers at a time
    ctx = serve_ctx(X, pool, budget=budget)
    try:
        mix = run_mix(X, ctx, pool, reqs, sc, n_producers=6)
        st = X.xdrop_get_serve_stats(ctx)
        big = pool.pairs[: 5000]
        out = np.zeros(len(big), X.RESULT_DTYPE)
        with pytest.raises(X.XdropError) as ei:
            X.xdrop_submit_pairs(ctx, big, sc, out)
        assert ei.value.code == X.XDROP_ENOMEM
    finally:
        X.xdrop_free(ctx)
    assert st["admission_waits"] > 0
    assert st["max_in_flight"] <= 3
    for k in (0, len(reqs) - 1):
        want = orc.align_pairs(pool.packed, pool.read_off, pool.read_len, pool.pairs[reqs[k][1]],
                               1, -1, -1, 50, nthreads=8)
        assert np.array_equal(mix[k].view(np.int32), want.view(np.int32))


def test_overflowing_bands_take_wider_tiers(X, orc, pool):
    """X = 400 makes bands wider than both in-kernel tiers (64 and 128
    slots): they finish on the 512-slot and unbounded tiers."""
    reqs = requests_for(pool, n_producers=4, per_producer=2, lo=20, hi=60, seed=500)
    sc = X.scoring(1, -1, -1, 400)
    ctx = serve_ctx(X, pool, tile=(4, 16))
    try:
        mix = run_mix(X, ctx, pool, reqs, sc, n_producers=4)
        st = X.xdrop_get_serve_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    assert st["wide_passes"] > 0
    for k, (_, idx) in enumerate(reqs):
        want = orc.align_pairs(pool.packed, pool.read_off, pool.read_len, pool.pairs[idx],
                               1, -1, -1, 400, nthreads=8)
        assert np.array_equal(mix[k].view(np.int32), want.view(np.int32))


def test_submit_pairs_outside_serving(X, orc, pool):
    """xdrop_submit_pairs in batched mode runs an ordinary ticket."""
    with X.Aligner() as al:
        X.xdrop_load_reads(al.ctx, pool.packed, pool.read_off, pool.read_len)
        idx = np.arange(0, pool.n_pairs, 37)
        out = np.zeros(len(idx), X.RESULT_DTYPE)
        t = X.xdrop_submit_pairs(al.ctx, pool.pairs[idx], X.scoring(1, -1, -1, 50), out)
        X.xdrop_sync(al.ctx, t, SYNC_NS)
    want = orc.align_pairs(pool.packed, pool.read_off, pool.read_len, pool.pairs[idx],
                           1, -1, -1, 50, nthreads=8)
    assert np.array_equal(out.view(np.int32), want.view(np.int32))


def test_mixed_scorings_packed_and_not(X, orc, pool):
    """Producers with different scorings share the serving kernel: one
    scoring fits the packed first tier, the other (mismatch -200) does
    not and runs on the 32-bit second tier.  Every request equals the
    oracle for its own scoring."""
    reqs = requests_for(pool, n_producers=8, per_producer=2, lo=40, hi=200, seed=700)
    scs = [(1, -1, -1, 50), (2, -200, -3, 60)]
    ctx = serve_ctx(X, pool)
    outs, errors = [None] * len(reqs), []

    def producer(items):
        try:
            tickets = []
            for i in items:
                p = reqs[i][0]
                out = np.zeros(len(reqs[i][1]), X.RESULT_DTYPE)
                outs[i] = out
                tickets.append(X.xdrop_submit_pairs(ctx, pool.pairs[reqs[i][1]],
                                                    X.scoring(*scs[p % 2]), out))
            for t in tickets:
                sync(X, ctx, t)
        except Exception as e:  # surfaced below
            errors.append(e)

    by_prod = {}
    for i, (p, _) in enumerate(reqs):
        by_prod.setdefault(p, []).append(i)
    try:
        th = [threading.Thread(target=producer, args=(items,)) for items in by_prod.values()]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=300)
        st = X.xdrop_get_serve_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    assert not errors, errors
    assert st["spill_taken"] > 0  # the second tier ran the unpacked scoring
    # no warp is reserved for the second tier: ring warps registered to serve it
    assert st["help_sessions"] > 0
    assert st["spill_taken"] == st["spill_reserved"]
    for i, (p, idx) in enumerate(reqs):
        want = orc.align_pairs(pool.packed, pool.read_off, pool.read_len, pool.pairs[idx],
                               *scs[p % 2], nthreads=8)
        assert np.array_equal(outs[i].view(np.int32), want.view(np.int32)), (i, scs[p % 2])


def test_reverse_strand_requests(X, orc):
    """Serving requests with reverse-strand pairs equal the oracle."""
    w = W.reverse_strand(W.template_pairs(n_pairs=120, len_lo=500, len_hi=3000, seed=43), 0.5, 5)
    sc = X.scoring(1, -1, -1, 50)
    ctx = serve_ctx(X, w)
    try:
        outs = run_alone(X, ctx, w, [(0, np.arange(0, 60)), (1, np.arange(60, 120))], sc)
    finally:
        X.xdrop_free(ctx)
    for k, idx in enumerate([np.arange(0, 60), np.arange(60, 120)]):
        want = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs[idx], 1, -1, -1, 50,
                               nthreads=8)
        assert np.array_equal(outs[k].view(np.int32), want.view(np.int32))


def test_idle_bound_ends_the_kernel_and_the_context_recovers(X, orc, pool):
    """The hang guard, without a fault: with a 2 ms idle bound the serving
    kernel's first-tier warps stop waiting for work on their own (counted in
    idle_exits, the status the host reads) well before the host's own idle
    stop, the kernel ends, and the next request launches it again and is
    exact."""
    sc = X.scoring(1, -1, -1, 50)
    ctx = X.xdrop_init(0, 0, X.XDROP_MODE_SERVE)
    try:
        X.xdrop_set_serve_idle(ctx, 2_000_000)
        X.xdrop_load_reads(ctx, pool.packed, pool.read_off, pool.read_len)
        first = run_alone(X, ctx, pool, [(0, np.arange(0, 300))], sc)[0]
        deadline = time.monotonic() + 5.0
        st = X.xdrop_get_serve_stats(ctx)
        while time.monotonic() < deadline and not (st["idle_exits"] > 0 and st["ring_warps"] == 0):
            time.sleep(0.002)
            st = X.xdrop_get_serve_stats(ctx)
        assert st["idle_exits"] > 0 and st["ring_warps"] == 0, st
        launches = st["relaunches"]
        second = run_alone(X, ctx, pool, [(0, np.arange(300, 600))], sc)[0]
        st2 = X.xdrop_get_serve_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    assert st2["relaunches"] > launches
    assert st2["requests_done"] == 2
    for out, idx in ((first, np.arange(0, 300)), (second, np.arange(300, 600))):
        want = orc.align_pairs(pool.packed, pool.read_off, pool.read_len, pool.pairs[idx],
                               1, -1, -1, 50, nthreads=8)
        assert np.array_equal(out.view(np.int32), want.view(np.int32))
