"""Adaptive acceptance on the GPU (xdrop_accept_device) against the oracle
(oracle.accept): the kernel gets the oracle's own alignment results, so
the comparison isolates the acceptance step; reverse-strand pairs, failed
alignments and several error rates and slacks.  Collected last: this
entry point has the least GPU history."""
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


@pytest.mark.parametrize("e4,d4", [(1500, 1000), (0, 0), (600, 2500), (10000, 10000)])
def test_accept_matches_oracle(X, orc, e4, d4):
    import torch
    # 80 % true overlaps, 20 % unrelated reads sharing only a planted seed
    w = W.reverse_strand(W.uneven_pairs(n_pairs=400, seed=3, x=30), 0.5, seed=2)
    res = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs, w.match, w.mismatch, w.gap,
                          w.x)
    res["status"][::37] = 1   # some failed alignments
    dev = X.DeviceInputs.from_workload(w)
    dev.out[: 7 * w.n_pairs].copy_(torch.from_numpy(res.view(np.int32).reshape(-1).copy()))
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    with X.Aligner() as al:
        got = al.accept_device(dev, sc, e4, d4).cpu().numpy()
    want = orc.accept(w.pairs, res, w.read_len, w.match, w.mismatch, e4, d4)
    assert np.array_equal(got, want)
    if (e4, d4) == (1500, 1000):
        assert w.n_pairs // 2 < want.sum() < w.n_pairs - w.n_pairs // 10


def test_accept_after_device_alignment(X, orc):
    """The usual chain: align on the device, then accept from the results
    in place; equal to the oracle's acceptance of the oracle's alignments."""
    w = W.template_pairs(n_pairs=200, len_lo=300, len_hi=2500, seed=8, x=40)
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner() as al:
        al.align_device(dev, sc)
        got = al.accept_device(dev, sc, 1500, 1000).cpu().numpy()
    res = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs, w.match, w.mismatch, w.gap,
                          w.x)
    assert np.array_equal(got, orc.accept(w.pairs, res, w.read_len, w.match, w.mismatch, 1500, 1000))


def test_accept_rejects_bad_parameters(X):
    import torch
    dev = X.DeviceInputs.from_workload(W.template_pairs(n_pairs=4, seed=1))
    acc = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with X.Aligner() as al:
        for e4, d4 in ((10001, 0), (0, 10001)):
            with pytest.raises(X.XdropError) as e:
                X.xdrop_accept_device(al.ctx, dev.pairs.data_ptr(), dev.out.data_ptr(), 4,
                                      dev.read_len.data_ptr(), dev.read_len.numel(), 1, -1, e4, d4,
                                      acc.data_ptr())
            assert e.value.code == X.XDROP_EINVAL
