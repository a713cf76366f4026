"""The allocation-free entry point (xdrop_align_static).

Some callers cannot allocate device memory when they align: a process whose
device memory belongs to another allocator, a latency-critical path that
cannot pay for cudaMalloc and its implicit synchronisation, or work issued
while a stream is being captured.  xdrop_align_static keeps its scratch in
a static array of the library and allocates nothing.  Its results must equal
the context-based entry point's (xdrop_submit_device) and the oracle's,
bit for bit, on two calls in a row, with more extensions than the kernel has
CTAs, so that each CTA reuses its scratch slice within a call.  Extensions
longer than the scratch allows get XDROP_STATUS_TOO_LONG and zero fields;
invalid pairs get XDROP_STATUS_INVALID and zero scores.

This file is collected last, so that a run stopping at its first failure
has already run every other test.
"""
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


def _workload():
    # 300 pairs = 600 extensions of uneven lengths: more than the kernel's
    # 128 CTAs, so every CTA runs several extensions in one call
    return W.template_pairs(n_pairs=300, len_lo=100, len_hi=2500, seed=31, x=40)


def _oracle(orc, w, pairs=None):
    return orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs if pairs is None else pairs,
                           w.match, w.mismatch, w.gap, w.x, nthreads=8)


def _call(X, dev, w, sc, max_read_len, out, stream):
    X.xdrop_align_static(dev.packed.data_ptr(), dev.packed.numel(), dev.read_off.data_ptr(),
                         dev.read_len.data_ptr(), dev.read_len.numel(), dev.pairs.data_ptr(),
                         w.n_pairs, sc, max_read_len, out.data_ptr(), stream)


def test_static_entry_matches_device_entry_and_oracle_two_calls(X, orc):
    import torch
    w = _workload()
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner() as al:
        al.align_device(dev, sc)
        want = dev.results().copy()
    oracle = _oracle(orc, w)
    assert np.array_equal(want.view(np.int32), oracle.view(np.int32))
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((w.n_pairs * 7,), -7, dtype=torch.int32, device="cuda:0")
        _call(X, dev, w, sc, int(w.read_len.max()), out, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(X.RESULT_DTYPE)
        assert np.array_equal(got.view(np.int32), want.view(np.int32)), f"call {call}"


def test_static_entry_too_long_and_invalid(X, orc):
    """A max_read_len below some extensions' lengths, and two invalid pairs
    (a read id past the last read, a seed past its read's end)."""
    import torch
    w = _workload()
    pairs = w.pairs.copy()
    pairs[7]["b"] = w.n_reads + 5
    pairs[11]["seed_a"] = w.read_len[pairs[11]["a"]]
    bad = np.zeros(w.n_pairs, bool)
    bad[[7, 11]] = True
    dev = X.DeviceInputs(w.packed, w.read_off, w.read_len, pairs)
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    limit = 1000
    out = torch.full((w.n_pairs * 7,), -7, dtype=torch.int32, device="cuda:0")
    _call(X, dev, w, sc, limit, out, 0)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(-1, 7)
    assert (got[bad, 6] == X.XDROP_STATUS_INVALID).all()
    assert (got[bad, :6] == 0).all()
    want = _oracle(orc, w, pairs[~bad]).view(np.int32).reshape(-1, 7)
    ok = pairs[~bad]
    la = w.read_len[ok["a"]].astype(np.int64)
    m = np.stack([ok["seed_a"].astype(np.int64), la - ok["seed_a"] - ok["seed_len"]], axis=1)
    g = got[~bad]
    # each CTA's slice holds 3*(limit+1) words rounded up to 64: an
    # extension with m <= limit always fits, one with m > limit + 21 never
    fits, over = m <= limit, m > limit + 21
    assert over.any() and fits.all(axis=1).any()
    for side in (0, 1):
        f = slice(3 * side, 3 * side + 3)
        assert (g[over[:, side], f] == 0).all()
        assert (g[over[:, side], 6] & X.XDROP_STATUS_TOO_LONG).all()
        assert np.array_equal(g[fits[:, side], f], want[fits[:, side], f])
    both = fits.all(axis=1)
    assert (g[both, 6] == 0).all()


def test_static_entry_rejects_oversized_reads(X):
    import torch
    w = _workload()
    dev = X.DeviceInputs.from_workload(w)
    out = torch.zeros(w.n_pairs * 7, dtype=torch.int32, device="cuda:0")
    with pytest.raises(X.XdropError) as ei:
        _call(X, dev, w, X.scoring(1, -1, -1, 40), 3_000_000, out, 0)
    assert ei.value.code == X.XDROP_EINVAL
    assert "max_read_len" in str(ei.value)
