"""Serving driver: many producer threads sending alignment requests to one GPU.

Producers stand in for the paper's MPI ranks (Section "Method"): each one
submits batches of read pairs with Poisson arrivals.  Four launch policies
are compared on the same arrivals:

* ``device-loop``: the library's serving mode (continuous batching: a
  persistent kernel takes requests as memory and slots free up, so work of
  requests that arrive while others run overlaps on the device);
* ``per-producer-streams``: each producer owns a batched context (its own
  CUDA stream and launches);
* ``ring-subbatch``: the paper's One-to-all / One-to-one schedulers on one
  GPU (Alg. 1): a token passes among producers that have work; the holder
  runs one sub-batch of at most 10,000 pairs, waits for it, and passes the
  token on;
* ``ring-batch``: the Opt-one-to-one scheduler: the holder runs all
  sub-batches of one batch before passing the token.

Latency of a request = time its results are back on the host minus its
arrival time.  This module is host logic only; every alignment runs in the
library's kernels.
"""
from __future__ import annotations

import queue
import statistics
import threading
import time

import numpy as np

from . import xdrop as X

SUB_BATCH = 10_000  # the paper's batch size (Section "Baseline")
POLICIES = ("device-loop", "per-producer-streams", "ring-subbatch", "ring-batch")


class TokenRing:
    """Round-robin token among ranks that have work (Alg. 1 on one GPU).

    A rank calls ``acquire(r)`` when it has a unit of work ready and
    ``release(r)`` when the unit is done.  The token goes to the next rank in ring order that is waiting,
    so finished or idle ranks are skipped (Alg. 1's search for the nearest
    unfinished rank, which keeps the ring from waiting on completed ranks)."""

    def __init__(self, n_ranks: int):
        self.n = n_ranks
        self.cv = threading.Condition()
        self.holder = None
        self.waiting = [False] * n_ranks
        self.last = n_ranks - 1
        self.units = 0
        self.max_holders = 0
        self._inside = 0

    def acquire(self, r: int, timeout: float | None = None) -> bool:
        with self.cv:
            self.waiting[r] = True
            if self.holder is None:
                self._grant()
            ok = self.cv.wait_for(lambda: self.holder == r, timeout=timeout)
            if not ok:
                self.waiting[r] = False
                return False
            self.waiting[r] = False
            self._inside += 1
            self.max_holders = max(self.max_holders, self._inside)
            return True

    def release(self, r: int) -> None:
        with self.cv:
            assert self.holder == r
            self._inside -= 1
            self.units += 1
            self.last = r
            self.holder = None
            self._grant()
            self.cv.notify_all()

    def _grant(self):
        for k in range(1, self.n + 1):
            cand = (self.last + k) % self.n
            if self.waiting[cand]:
                self.holder = cand
                self.cv.notify_all()
                return


def _percentile(v, q):
    if not v:
        return None
    return float(np.percentile(np.asarray(v), q))


class Result:
    def __init__(self, policy, rho, offered_pairs_s):
        self.policy = policy
        self.rho = rho
        self.offered_pairs_s = offered_pairs_s
        self.latencies = []
        self.pairs = 0
        self.requests = 0
        self.wall_s = 0.0
        self.errors = []
        self.outputs = {}
        self.serve_stats = None  # device-loop: the serving loop's counters

    def summary(self):
        return {"policy": self.policy, "rho": self.rho,
                "offered_pairs_per_s": self.offered_pairs_s,
                "requests": self.requests, "pairs": self.pairs,
                "pairs_per_s": self.pairs / self.wall_s if self.wall_s else None,
                "p50_ms": _percentile(self.latencies, 50) * 1e3 if self.latencies else None,
                "p99_ms": _percentile(self.latencies, 99) * 1e3 if self.latencies else None,
                "mean_ms": statistics.mean(self.latencies) * 1e3 if self.latencies else None,
                "errors": len(self.errors),
                "first_errors": self.errors[:3],
                "serve_stats": self.serve_stats}


def run_policy(policy, pool, schedule, sc, device=0, budget=0, tile=None, keep_outputs=False,
               rho=None, offered=None, sync_timeout_s=120.0):
    """Replay ``schedule`` (per producer: [(arrival_s, pair_indices)], from
    workloads.serving_schedule) under ``policy``.  Returns a Result."""
    if policy not in POLICIES:
        raise ValueError(policy)
    n_prod = len(schedule)
    res = Result(policy, rho, offered)
    lock = threading.Lock()
    ctxs = []
    if policy == "device-loop":
        ctx = X.xdrop_init(device, budget, X.XDROP_MODE_SERVE)
        if tile:
            X.xdrop_set_tile(ctx, *tile)
        X.xdrop_load_reads(ctx, pool.packed, pool.read_off, pool.read_len)
        ctxs = [ctx] * n_prod
    elif policy == "per-producer-streams":
        for _ in range(n_prod):
            c = X.xdrop_init(device, 0, X.XDROP_MODE_BATCHED)
            if tile:
                X.xdrop_set_tile(c, *tile)
            X.xdrop_load_reads(c, pool.packed, pool.read_off, pool.read_len)
            ctxs.append(c)
    else:
        c = X.xdrop_init(device, 0, X.XDROP_MODE_BATCHED)
        if tile:
            X.xdrop_set_tile(c, *tile)
        X.xdrop_load_reads(c, pool.packed, pool.read_off, pool.read_len)
        ctxs = [c] * n_prod
    ring = TokenRing(n_prod) if policy.startswith("ring") else None
    # warm the contexts (autotuning and graph capture happen outside timing)
    warm = pool.pairs[: min(2048, pool.n_pairs)]
    for c in {id(c): c for c in ctxs}.values():
        out = np.zeros(len(warm), X.RESULT_DTYPE)
        X.xdrop_sync(c, X.xdrop_submit_pairs(c, warm, sc, out))

    done_q = queue.Queue()
    t0 = time.perf_counter() + 0.05

    def record(p, k, arrival, n, out):
        lat = time.perf_counter() - (t0 + arrival)
        with lock:
            res.latencies.append(lat)
            res.pairs += n
            res.requests += 1
            if keep_outputs:
                res.outputs[(p, k)] = out

    def waiter():
        while True:
            item = done_q.get()
            if item is None:
                return
            c, t, p, k, arrival, n, out = item
            try:
                X.xdrop_sync(c, t, int(sync_timeout_s * 1e9))
                record(p, k, arrival, n, out)
            except Exception as e:
                with lock:
                    res.errors.append(repr(e))

    def producer(p):
        c = ctxs[p]
        for k, (arrival, idx) in enumerate(schedule[p]):
            delay = t0 + arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            pairs = pool.pairs[idx]
            try:
                if policy in ("device-loop", "per-producer-streams"):
                    out = np.zeros(len(idx), X.RESULT_DTYPE)
                    t = X.xdrop_submit_pairs(c, pairs, sc, out)
                    done_q.put((c, t, p, k, arrival, len(idx), out))
                else:
                    out = np.zeros(len(idx), X.RESULT_DTYPE)
                    chunks = [slice(s, min(s + SUB_BATCH, len(idx)))
                              for s in range(0, len(idx), SUB_BATCH)]
                    if policy == "ring-batch":
                        ring.acquire(p)
                        try:
                            for sl in chunks:
                                X.xdrop_sync(c, X.xdrop_submit_pairs(c, pairs[sl], sc, out[sl]))
                        finally:
                            ring.release(p)
                    else:
                        for sl in chunks:
                            ring.acquire(p)
                            try:
                                X.xdrop_sync(c, X.xdrop_submit_pairs(c, pairs[sl], sc, out[sl]))
                            finally:
                                ring.release(p)
                    record(p, k, arrival, len(idx), out)
            except Exception as e:
                with lock:
                    res.errors.append(repr(e))

    waiters = [threading.Thread(target=waiter, daemon=True) for _ in range(32)]
    for w in waiters:
        w.start()
    prods = [threading.Thread(target=producer, args=(p,)) for p in range(n_prod)]
    for th in prods:
        th.start()
    for th in prods:
        th.join()
    for _ in waiters:
        done_q.put(None)
    for w in waiters:
        w.join()
    res.wall_s = time.perf_counter() - t0
    if policy == "device-loop":
        res.serve_stats = X.xdrop_get_serve_stats(ctxs[0])
    for c in {id(c): c for c in ctxs}.values():
        X.xdrop_free(c)
    if ring is not None:
        assert ring.max_holders <= 1
    return res
