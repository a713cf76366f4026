"""The allocation-free entry point (xdrop_align_static) against the
context-based device entry point.

Callers that cannot allocate device memory at alignment time (a process
whose device memory belongs to another allocator, a latency-critical path,
work issued during stream capture) use xdrop_align_static, which keeps its
scratch in a static array of the library.  This file is collected last so
that a run stopping at the first failure has already run every other test.
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
    a = W.template_pairs(n_pairs=40, len_lo=300, len_hi=2500, seed=31, x=40)
    return a


def test_static_entry_matches_device_entry_two_calls(X):
    import torch
    w = _workload()
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner() as al:
        al.align_device(dev, sc)
        want = dev.results().copy()
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((w.n_pairs * 7,), -7, dtype=torch.int32, device="cuda:0")
        X.xdrop_align_static(dev.packed.data_ptr(), dev.packed.numel(), dev.read_off.data_ptr(),
                             dev.read_len.data_ptr(), dev.read_len.numel(), dev.pairs.data_ptr(),
                             w.n_pairs, sc, int(w.read_len.max()), out.data_ptr(),
                             stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(X.RESULT_DTYPE)
        assert np.array_equal(got.view(np.int32), want.view(np.int32)), f"call {call}"


def test_static_entry_rejects_oversized_reads(X):
    import torch
    w = _workload()
    dev = X.DeviceInputs.from_workload(w)
    out = torch.zeros(w.n_pairs * 7, dtype=torch.int32, device="cuda:0")
    with pytest.raises(X.XdropError) as ei:
        X.xdrop_align_static(dev.packed.data_ptr(), dev.packed.numel(), dev.read_off.data_ptr(),
                             dev.read_len.data_ptr(), dev.read_len.numel(), dev.pairs.data_ptr(),
                             w.n_pairs, X.scoring(1, -1, -1, 40), 3_000_000, out.data_ptr(), 0)
    assert ei.value.code == X.XDROP_EINVAL
    assert "max_read_len" in str(ei.value)
