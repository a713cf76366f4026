"""Every pair of the benchmark workloads against the oracle.

The GPU path runs exactly as the benchmark times it (batched device submit,
autotuned first tile, one CUDA graph) and, beside it, the plain
per-10,000-pair form, every forced first tile, and the serving mode.  Each
result record (scores, coordinates, status) must equal the oracle's, pair
for pair: integer work, bit-exact.  The per-extension cell counts of the
library's counting pass, the numerator of the reported GCUPS, must equal
the oracle's counts of the cells it evaluates.

The oracle runs once per workload and X on every host core (about a
minute for the 29x workload at X = 50 on 16 cores).
"""
import threading

import numpy as np
import pytest

from paper_2309_07270_gb300 import workloads as W

pytestmark = pytest.mark.gpu
P16 = 0x100  # XDROP_TILE_PACKED16


@pytest.fixture(scope="module")
def X():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_07270_gb300 import build, xdrop
    build.build()
    return xdrop


def rows(res):
    return res.view(np.int32).reshape(-1, 7)


def assert_every_pair(got, want, what):
    g, e = rows(got), rows(want)
    assert g.shape == e.shape, what
    bad = np.flatnonzero((g != e).any(axis=1))
    assert bad.size == 0, (f"{what}: {bad.size} of {len(g)} pairs differ, first {bad[:5]}: "
                           f"gpu {g[bad[:3]]} oracle {e[bad[:3]]}")


@pytest.fixture(scope="module")
def uneven1m():
    return W.uneven_pairs(n_pairs=1_000_000, seed=3)


@pytest.mark.parametrize("x", [50, 100])
def test_genome_29x_every_pair(X, oracle_full, genome29, x):
    """The 29x overlap workload (313,859 pairs): the benchmarked batched
    form, the plain form and the cell counts, every pair."""
    w = genome29.with_x(x)
    want, want_cells = oracle_full(("genome29x", x), w)
    sc = X.scoring(1, -1, -1, x)
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.align_device(dev, sc)
        assert_every_pair(dev.results(), want, f"29x x={x} batched")
        cells = al.count_cells_device(dev, sc).cpu().numpy().reshape(-1, 2)
        host = al.align(w.packed, w.read_off, w.read_len, w.pairs, sc)
    assert np.array_equal(cells, want_cells), "cell counts differ from the oracle's"
    assert int(cells.sum()) == int(want_cells.sum())
    assert_every_pair(host, want, f"29x x={x} host submit")
    with X.Aligner(mode=X.XDROP_MODE_PLAIN) as al:
        al.align_device(dev, sc)
        assert_every_pair(dev.results(), want, f"29x x={x} plain")


TILES = [(4, 16), (4, 16 | P16), (8, 8 | P16), (8, 16 | P16), (16, 8 | P16), (4, 8 | P16),
         (2, 16 | P16), (2, 32 | P16), (4, 32 | P16)]


@pytest.mark.parametrize("x", [50, 100])
def test_genome_29x_every_tile_every_pair(X, oracle_full, genome29, x):
    """Each forced first tile (packed and 32-bit) on every pair of the 29x
    workload, against the oracle."""
    w = genome29.with_x(x)
    want, _ = oracle_full(("genome29x", x), w)
    dev = X.DeviceInputs.from_workload(w)
    sc = X.scoring(1, -1, -1, x)
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        for t in TILES:
            al.set_tile(*t)
            al.align_device(dev, sc)
            assert al.tile() == t
            assert_every_pair(dev.results(), want, f"29x x={x} tile {t[0]}x{t[1] & 0xff}"
                              + ("p" if t[1] & P16 else ""))


def test_genome_29x_served_every_pair(X, oracle_full, genome29):
    """The serving configuration: 25 producer threads, each submitting
    batches of U[1k, 20k] pairs drawn from the 29x pool (seeds 100 + p) to
    one serving context at once; every returned record equals the
    oracle's record of its pool pair."""
    w = genome29.with_x(50)
    want, _ = oracle_full(("genome29x", 50), w)
    sched = W.serving_schedule(w.n_pairs, n_producers=25, rate_pairs_per_s=2e6, duration_s=0.5,
                               seed_base=100)
    reqs = [idx for items in sched for _, idx in items]
    assert len(reqs) >= 25
    sc = X.scoring(1, -1, -1, 50)
    ctx = X.xdrop_init(0, 0, X.XDROP_MODE_SERVE)
    outs = [np.zeros(len(idx), X.RESULT_DTYPE) for idx in reqs]
    errors = []
    try:
        X.xdrop_load_reads(ctx, w.packed, w.read_off, w.read_len)

        def producer(items):
            try:
                tickets = [X.xdrop_submit_pairs(ctx, w.pairs[reqs[i]], sc, outs[i]) for i in items]
                for t in tickets:
                    X.xdrop_sync(ctx, t, int(300e9))
            except Exception as e:  # reported below
                errors.append(e)

        per = {}
        k = 0
        for p, items in enumerate(sched):
            per[p] = list(range(k, k + len(items)))
            k += len(items)
        th = [threading.Thread(target=producer, args=(v,)) for v in per.values() if v]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=600)
        st = X.xdrop_get_serve_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    assert not errors, errors
    assert st["requests_done"] == len(reqs)
    assert st["max_in_flight"] > 1
    # every published extension was claimed (per block, with this backlog), and the
    # overflowed ones were served by warps that left the first tier to help
    assert st["consumed"] == st["published"]
    assert st["spill_taken"] == st["spill_reserved"] > 0
    assert st["help_sessions"] > 0
    assert st["surplus_counts"] == 0
    for idx, out in zip(reqs, outs):
        assert_every_pair(out, want[idx], "served request")


def test_ring_reuse_under_a_deep_backlog(X, oracle_full, genome29):
    """Requests whose extensions outnumber the serving task ring (2^21
    entries) several times, submitted at once by 8 producers: the ring is
    reused while a deep backlog of claimed and unclaimed entries is in
    flight, and requests finish out of order.  Every record equals the
    oracle's, every extension is counted exactly once, and no slot reuse
    loses or repeats a task."""
    w = genome29.with_x(50)
    want, _ = oracle_full(("genome29x", 50), w)
    rng = np.random.default_rng(909)
    reqs = [rng.choice(w.n_pairs, size=int(rng.integers(15_000, 20_001)), replace=False)
            for _ in range(160)]
    assert 2 * sum(len(r) for r in reqs) > 2.5 * (1 << 21)
    sc = X.scoring(1, -1, -1, 50)
    ctx = X.xdrop_init(0, 0, X.XDROP_MODE_SERVE)
    outs = [np.zeros(len(idx), X.RESULT_DTYPE) for idx in reqs]
    errors = []
    try:
        X.xdrop_load_reads(ctx, w.packed, w.read_off, w.read_len)

        def producer(items):
            try:
                tickets = [X.xdrop_submit_pairs(ctx, w.pairs[reqs[i]], sc, outs[i]) for i in items]
                for t in tickets:
                    X.xdrop_sync(ctx, t, int(300e9))
            except Exception as e:  # reported below
                errors.append(e)

        th = [threading.Thread(target=producer, args=(list(range(p, len(reqs), 8)),))
              for p in range(8)]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=900)
        st = X.xdrop_get_serve_stats(ctx)
    finally:
        X.xdrop_free(ctx)
    assert not errors, errors
    assert st["requests_done"] == len(reqs)
    assert st["published"] == st["consumed"] == 2 * sum(len(r) for r in reqs)
    assert st["surplus_counts"] == 0
    assert st["spill_taken"] == st["spill_reserved"]
    for idx, out in zip(reqs, outs):
        assert_every_pair(out, want[idx], "request after ring reuse")


def test_uneven_1m_every_pair(X, oracle_full, uneven1m):
    """The uneven stress workload (1M pairs, Pareto lengths 100 bp - 50 kb,
    20 % unrelated pairs): batched (autotuned, graph) and plain forms and
    the cell counts, every pair."""
    w = uneven1m
    want, want_cells = oracle_full(("uneven1m", 50), w)
    sc = X.scoring(1, -1, -1, 50)
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        al.align_device(dev, sc)
        assert_every_pair(dev.results(), want, "uneven batched")
        cells = al.count_cells_device(dev, sc).cpu().numpy().reshape(-1, 2)
    assert np.array_equal(cells, want_cells), "cell counts differ from the oracle's"
    with X.Aligner(mode=X.XDROP_MODE_PLAIN) as al:
        al.align_device(dev, sc)
        assert_every_pair(dev.results(), want, "uneven plain")
