"""Host logic of the serving driver (serving.run_policy) against a fake
library: every request of a schedule is delivered whole, into the right
output rows, under each of the four launch policies; the token-ring
policies run at most one sub-batch of 10,000 pairs (or one whole batch, for
the batch variant) at a time; every context opened is freed once.  No GPU:
the fake records calls and answers each pair with its own indices."""
import threading
import time
import types

import numpy as np
import pytest

from paper_2309_07270_gb300 import serving
from paper_2309_07270_gb300 import xdrop as X

N_POOL = 60_000


class FakeLib:
    XDROP_MODE_BATCHED = X.XDROP_MODE_BATCHED
    XDROP_MODE_SERVE = X.XDROP_MODE_SERVE
    RESULT_DTYPE = X.RESULT_DTYPE

    def __init__(self, fail_ticket=None, sync_s=0.0):
        self.sync_s = sync_s
        self.lock = threading.Lock()
        self.modes = {}          # ctx -> mode
        self.loaded = set()
        self.freed = []
        self.submits = []        # (ctx, n_pairs)
        self.pending = {}        # ticket -> (ctx, pairs, out)
        self.open_max = {}       # ctx -> largest number of tickets open at once
        self.next_ticket = 1
        self.fail_ticket = fail_ticket

    def xdrop_init(self, device=0, budget=0, mode=X.XDROP_MODE_BATCHED):
        with self.lock:
            ctx = object()
            self.modes[ctx] = mode
            self.open_max[ctx] = 0
            return ctx

    def xdrop_set_tile(self, ctx, lanes, cells):
        assert ctx in self.modes

    def xdrop_load_reads(self, ctx, packed, read_off, read_len):
        assert ctx in self.modes
        self.loaded.add(ctx)

    def xdrop_submit_pairs(self, ctx, pairs, sc, out):
        assert ctx in self.loaded and ctx not in self.freed
        assert len(out) == len(pairs) and out.dtype == X.RESULT_DTYPE
        with self.lock:
            t = self.next_ticket
            self.next_ticket += 1
            self.pending[t] = (ctx, pairs.copy(), out)
            self.submits.append((ctx, len(pairs)))
            n_open = sum(1 for c, _, _ in self.pending.values() if c is ctx)
            self.open_max[ctx] = max(self.open_max[ctx], n_open)
            return t

    def xdrop_sync(self, ctx, ticket, timeout_ns=-1):
        with self.lock:
            c, pairs, out = self.pending.pop(ticket)
        assert c is ctx
        if self.sync_s:
            time.sleep(self.sync_s)
        if ticket == self.fail_ticket:
            raise RuntimeError("fake sync failure")
        out["left_score"] = pairs["a"]
        out["right_score"] = pairs["seed_a"]
        out["status"] = 0

    def xdrop_get_serve_stats(self, ctx):
        assert self.modes[ctx] == X.XDROP_MODE_SERVE
        return {"requests": 0}

    def xdrop_free(self, ctx):
        with self.lock:
            self.freed.append(ctx)


def pool():
    pairs = np.zeros(N_POOL, X.PAIR_DTYPE)
    pairs["a"] = np.arange(N_POOL)
    pairs["seed_a"] = 7 * np.arange(N_POOL)
    return types.SimpleNamespace(packed=np.zeros(4, np.uint32),
                                 read_off=np.zeros(1, np.uint64),
                                 read_len=np.zeros(1, np.uint32),
                                 pairs=pairs, n_pairs=N_POOL)


def schedule(n_prod=4):
    """Sizes around the 10,000-pair sub-batch bound, arrivals within 40 ms."""
    rng = np.random.default_rng(3)
    sizes = [1, 9_999, 10_000, 10_001, 25_000, 333]
    out = []
    for p in range(n_prod):
        items = []
        for k, n in enumerate(sizes[p % 2:]):
            items.append((0.005 * k + 0.001 * p, rng.integers(0, N_POOL, n)))
        out.append(items)
    return out


def warm_size():
    return min(2048, N_POOL)


@pytest.mark.parametrize("policy", serving.POLICIES)
def test_every_request_delivered_into_its_rows(monkeypatch, policy):
    fake = FakeLib()
    monkeypatch.setattr(serving, "X", fake)
    sched = schedule()
    res = serving.run_policy(policy, pool(), sched, sc=None, keep_outputs=True,
                             sync_timeout_s=5.0)
    assert res.errors == []
    n_req = sum(len(s) for s in sched)
    n_pairs = sum(len(idx) for s in sched for _, idx in s)
    assert (res.requests, res.pairs, len(res.latencies)) == (n_req, n_pairs, n_req)
    assert all(lat > 0 for lat in res.latencies)
    for p, items in enumerate(sched):
        for k, (_, idx) in enumerate(items):
            out = res.outputs[(p, k)]
            assert np.array_equal(out["left_score"], idx)
            assert np.array_equal(out["right_score"], 7 * idx)
    assert fake.pending == {}
    s = res.summary()
    assert s["policy"] == policy and s["requests"] == n_req and s["errors"] == 0
    assert s["p50_ms"] <= s["p99_ms"]


@pytest.mark.parametrize("policy", serving.POLICIES)
def test_contexts_and_launch_granularity(monkeypatch, policy):
    fake = FakeLib()
    monkeypatch.setattr(serving, "X", fake)
    sched = schedule()
    res = serving.run_policy(policy, pool(), sched, sc=None)
    ctxs = list(fake.modes)
    # one serving context, one per producer, or one shared batched context
    want_ctx = {"device-loop": 1, "per-producer-streams": len(sched)}.get(policy, 1)
    assert len(ctxs) == want_ctx
    want_mode = X.XDROP_MODE_SERVE if policy == "device-loop" else X.XDROP_MODE_BATCHED
    assert all(m == want_mode for m in fake.modes.values())
    assert sorted(map(id, fake.freed)) == sorted(map(id, ctxs))  # each freed once
    assert (res.serve_stats is not None) == (policy == "device-loop")
    # each context first takes one warm-up batch
    sizes = [n for _, n in fake.submits]
    assert sizes[:want_ctx] == [warm_size()] * want_ctx
    sizes = sorted(sizes[want_ctx:])
    req = [len(idx) for s in sched for _, idx in s]
    if policy.startswith("ring"):
        sub = [min(serving.SUB_BATCH, n - s) for n in req for s in range(0, n, serving.SUB_BATCH)]
        assert sizes == sorted(sub)
        assert max(sizes) <= serving.SUB_BATCH
        # the token holder waits for its launch before passing the token on
        assert fake.open_max[ctxs[0]] == 1
    else:
        assert sizes == sorted(req)


def ring_order(monkeypatch, policy):
    """Which producer made each submit, two producers each sending one
    30,000-pair request (three sub-batches) at the same time; every sync
    takes 20 ms so that both wait for the token."""
    fake = FakeLib(sync_s=0.02)
    owner = {}
    order = []
    real_submit = fake.xdrop_submit_pairs

    def submit(ctx, pairs, sc, out):
        order.append(owner.get(threading.get_ident()))
        return real_submit(ctx, pairs, sc, out)

    class Tagged(threading.Thread):
        def run(self):
            if self._args:  # producer threads get their index as the one argument
                owner[threading.get_ident()] = self._args[0]
            super().run()

    monkeypatch.setattr(fake, "xdrop_submit_pairs", submit)
    monkeypatch.setattr(serving, "X", fake)
    monkeypatch.setattr(serving.threading, "Thread", Tagged)
    idx = np.arange(30_000)
    res = serving.run_policy(policy, pool(), [[(0.0, idx)], [(0.0, idx)]], sc=None)
    assert res.errors == [] and res.requests == 2
    return [p for p in order if p is not None]


def test_ring_batch_holds_the_token_for_a_whole_batch(monkeypatch):
    """Opt-one-to-one: the holder runs all sub-batches of its batch."""
    assert ring_order(monkeypatch, "ring-batch") in ([0, 0, 0, 1, 1, 1], [1, 1, 1, 0, 0, 0])


def test_ring_subbatch_passes_the_token_after_each_sub_batch(monkeypatch):
    """One-to-all / one-to-one: the token moves on after every sub-batch,
    to the next producer that waits, so the two alternate."""
    runs = ring_order(monkeypatch, "ring-subbatch")
    assert sorted(runs) == [0, 0, 0, 1, 1, 1]
    assert all(a != b for a, b in zip(runs, runs[1:]))


def test_sync_failure_is_reported_and_the_rest_delivered(monkeypatch):
    fake = FakeLib(fail_ticket=5)   # ticket 1 is the warm-up batch
    monkeypatch.setattr(serving, "X", fake)
    sched = schedule(n_prod=2)
    res = serving.run_policy("device-loop", pool(), sched, sc=None, sync_timeout_s=5.0)
    n_req = sum(len(s) for s in sched)
    assert len(res.errors) == 1 and "fake sync failure" in res.errors[0]
    assert res.requests == n_req - 1


def test_unknown_policy_is_rejected(monkeypatch):
    monkeypatch.setattr(serving, "X", FakeLib())
    with pytest.raises(ValueError):
        serving.run_policy("round-robin", pool(), schedule(), sc=None)
