"""The round-robin token of the paper's schedulers (Alg. 1), on CPU threads.

Invariants from the algorithm's description: at most one rank holds the
token (no two ranks use the GPU at once), ranks with unequal numbers of
batches never deadlock (finished ranks are skipped), every unit runs
exactly once, and the token visits waiting ranks in ring order.
"""
import threading
import time

from paper_2309_07270_gb300.serving import TokenRing


def run_ring(counts, hold_s=0.0005):
    ring = TokenRing(len(counts))
    log = []
    inside = [0]
    peak = [0]
    lk = threading.Lock()

    def rank(r):
        for u in range(counts[r]):
            assert ring.acquire(r, timeout=10)
            with lk:
                inside[0] += 1
                peak[0] = max(peak[0], inside[0])
                log.append((r, u))
            time.sleep(hold_s)
            with lk:
                inside[0] -= 1
            ring.release(r)

    th = [threading.Thread(target=rank, args=(r,)) for r in range(len(counts))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=30)
    assert not any(t.is_alive() for t in th), "deadlock"
    return log, peak[0], ring


def test_mutual_exclusion_and_completeness():
    counts = [3, 0, 7, 1, 4, 2]
    log, peak, ring = run_ring(counts)
    assert peak == 1 and ring.max_holders == 1
    assert sorted(log) == sorted((r, u) for r in range(len(counts)) for u in range(counts[r]))
    assert ring.units == sum(counts)
    for r in range(len(counts)):  # each rank's units in its own order
        assert [u for rr, u in log if rr == r] == list(range(counts[r]))


def test_round_robin_skips_idle_ranks():
    counts = [4, 4, 0, 4]
    # ranks wait before the first grant so the order is deterministic
    ring = TokenRing(len(counts))
    order = []
    ready = threading.Barrier(3)

    def rank(r):
        ready.wait()
        for _ in range(counts[r]):
            ring.acquire(r, timeout=10)
            order.append(r)
            time.sleep(0.002)
            ring.release(r)

    th = [threading.Thread(target=rank, args=(r,)) for r in (0, 1, 3)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=30)
    assert len(order) == 12
    # after the first grant every turn goes to the next waiting rank in ring order
    for a, b in zip(order[2:], order[3:]):
        assert b == {0: 1, 1: 3, 3: 0}[a]


def test_acquire_timeout_leaves_ring_usable():
    ring = TokenRing(2)
    assert ring.acquire(0, timeout=1)
    got = ring.acquire(1, timeout=0.05)  # held by rank 0
    assert not got
    ring.release(0)
    assert ring.acquire(1, timeout=1)
    ring.release(1)
