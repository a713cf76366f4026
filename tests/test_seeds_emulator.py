"""Seed discovery's per-element steps (csrc/xd_seeds.cuh), run on the CPU in
the device pipeline's order by tests/seeds_emulator.cpp for both products
(sort-based and row-wise), against the oracle (oracle/seeds.py) record for
record: k from 1 to 32 (windows over one, two
and three packed words), strides, repeats inside a read, reads shorter
than k, empty reads, read counts around the key-width boundaries."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import seeds as S
from paper_2309_07270_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    so = tmp_path_factory.mktemp("seeds_emu") / "libseeds_emu.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-Wall", "-Werror", "-shared", "-fPIC", "-o", str(so),
                    os.path.join(HERE, "seeds_emulator.cpp")], check=True)
    lib = ctypes.CDLL(str(so))
    vp, u32, i64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int64
    lib.emulate_candidates.restype = i64
    lib.emulate_candidates.argtypes = [vp, vp, vp, u32, u32, u32, u32, u32, vp, i64]
    lib.emulate_candidates_rowwise.restype = i64
    lib.emulate_candidates_rowwise.argtypes = [vp, vp, vp, u32, u32, u32, u32, u32, u32, vp, i64]
    return lib


def run_emu(lib, product, packed, off, lens, k, lo, hi, stride=1, table_lg=11):
    """Candidates of the emulated product ("sort" or "rows"); None when the
    row-wise tables overflow."""
    packed = np.ascontiguousarray(packed, np.uint32)
    off = np.ascontiguousarray(off, np.uint64)
    lens = np.ascontiguousarray(lens, np.uint32)
    args = [packed.ctypes.data, off.ctypes.data, lens.ctypes.data, len(lens), k, stride, lo, hi]
    if product == "rows":
        fn = lambda o, c: lib.emulate_candidates_rowwise(*args, table_lg, o, c)  # noqa: E731
    else:
        fn = lambda o, c: lib.emulate_candidates(*args, o, c)  # noqa: E731
    n = fn(None, 0)
    if n < 0:
        return None
    out = np.zeros(6 * max(n, 1), np.uint32)
    assert fn(out.ctypes.data, n) == n
    return out[:6 * n].view(S.CANDIDATE)


@pytest.fixture(scope="module", params=["sort", "rows"])
def emu(lib, request):
    def run(packed, off, lens, k, lo, hi, stride=1):
        got = run_emu(lib, request.param, packed, off, lens, k, lo, hi, stride)
        assert got is not None
        return got
    return run


def same(got, want):
    assert got.dtype == want.dtype and len(got) == len(want)
    assert np.array_equal(got, want)


def pack(reads):
    return W.pack_reads([np.asarray(r, np.uint8) for r in reads])


def small_genome_reads(n_reads, seed, glen=400, lo=20, hi=160, rc_frac=0.4, err=True):
    """Overlapping reads of a short genome, some reverse-complemented."""
    rng = np.random.default_rng(seed)
    g = rng.integers(0, 4, glen).astype(np.uint8)
    reads = []
    for _ in range(n_reads):
        n = int(rng.integers(lo, hi + 1))
        s = int(rng.integers(0, glen - n + 1))
        r = W.mutate(g[s:s + n], rng)[0] if err else g[s:s + n].copy()
        reads.append(W.revcomp(r) if rng.random() < rc_frac else r)
    return reads


@pytest.mark.parametrize("k", [1, 2, 3, 7, 15, 16, 17, 24, 31, 32])
@pytest.mark.parametrize("stride", [1, 3])
def test_k_and_stride_sweep(emu, k, stride):
    reads = small_genome_reads(9, seed=k * 10 + stride, err=k < 15)
    packed, off, lens = pack(reads)
    for lo, hi in ((1, 1024), (2, 5)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi, stride=stride)
        same(emu(packed, off, lens, k, lo, hi, stride), want)
    if k >= 7:
        assert len(S.candidate_pairs(packed, off, lens, k=k, lo=1, hi=1024, stride=stride)) > 0


def test_repeats_inside_reads(emu):
    """A periodic read has each k-mer many times: it counts every time
    toward the frequency, but only its first occurrence pairs reads."""
    rng = np.random.default_rng(5)
    unit = rng.integers(0, 4, 7).astype(np.uint8)
    reads = [np.tile(unit, 12)[:80], np.tile(unit, 9)[3:60], W.revcomp(np.tile(unit, 10)[1:66]),
             rng.integers(0, 4, 90).astype(np.uint8)]
    packed, off, lens = pack(reads)
    for k, lo, hi in ((5, 1, 1024), (9, 2, 30), (9, 20, 40), (4, 3, 1024)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi)
        same(emu(packed, off, lens, k, lo, hi), want)
    assert len(S.candidate_pairs(packed, off, lens, k=9, lo=20, hi=40)) == 3


def test_short_and_empty_reads(emu):
    reads = small_genome_reads(8, seed=9, err=False)
    reads[2] = reads[2][:5]
    reads[5] = np.zeros(0, np.uint8)
    reads.insert(0, np.zeros(0, np.uint8))
    packed, off, lens = pack(reads)
    for k in (6, 11):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=1, hi=1024)
        same(emu(packed, off, lens, k, 1, 1024), want)


@pytest.mark.parametrize("n_reads", [1, 2, 3, 4, 5, 17, 33])
def test_read_count_key_widths(emu, n_reads):
    reads = small_genome_reads(n_reads, seed=100 + n_reads, glen=300, lo=40, hi=120, err=False)
    packed, off, lens = pack(reads)
    want = S.candidate_pairs(packed, off, lens, k=13, lo=1, hi=1024)
    same(emu(packed, off, lens, 13, 1, 1024), want)
    if n_reads == 1:
        assert len(want) == 0


def test_nothing_to_pair(emu):
    packed, off, lens = pack([np.zeros(0, np.uint8), np.array([1, 2, 3], np.uint8)])
    assert len(emu(packed, off, lens, 5, 1, 10)) == 0
    packed, off, lens = pack([np.array([0, 1, 2, 3] * 5, np.uint8)])
    assert len(emu(packed, off, lens, 3, 1, 10)) == 0     # one read: no pairs


def test_sequencing_reads_medium(emu):
    """Error-model reads of a 20 kb genome at 5x, both strands: about 100 kb."""
    packed, off, lens = W.sequencing_reads(20_000, 5, 2_000, 1_000, 500, seed=3)
    for k, lo, hi in ((17, 2, 8), (13, 2, 12)):
        want = S.candidate_pairs(packed, off, lens, k=k, lo=lo, hi=hi)
        assert len(want) > 100 and (want["b"] >> 31).sum() > 20
        same(emu(packed, off, lens, k, lo, hi), want)


def star_reads(n_leaves, seed=12, k=8):
    """Read 0 holds many distinct k-mers; every other read is a copy of one
    of them, round robin: read 0 pairs with all n_leaves reads while no
    k-mer is held by more than a few reads."""
    rng = np.random.default_rng(seed)
    while True:
        hub = rng.integers(0, 4, 160).astype(np.uint8)
        codes = S.occurrences([hub.tolist()], k)
        if len({c for c, *_ in codes}) == len(codes):   # distinct canonical k-mers
            break
    n_k = len(hub) - k + 1
    reads = [hub] + [hub[i % n_k:i % n_k + k].copy() for i in range(n_leaves)]
    return reads


def test_row_tables_overflow_and_fit(lib):
    """A read with more partners than its table has slots makes the
    row-wise product give up (the library then runs the sort-based one);
    with room to spare both products equal the oracle."""
    packed, off, lens = pack(star_reads(40))
    want = S.candidate_pairs(packed, off, lens, k=8, lo=1, hi=1024)
    assert (want["a"] == 0).sum() == 40
    assert run_emu(lib, "rows", packed, off, lens, 8, 1, 1024, table_lg=5) is None   # 32 slots
    for lg in (6, 11):
        same(run_emu(lib, "rows", packed, off, lens, 8, 1, 1024, table_lg=lg), want)
    same(run_emu(lib, "sort", packed, off, lens, 8, 1, 1024), want)


def test_row_tables_full_size_overflow(lib):
    """2,100 partners of one read overflow the library's 2,048-slot table;
    2,000 fit."""
    packed, off, lens = pack(star_reads(2100))
    assert run_emu(lib, "rows", packed, off, lens, 8, 1, 1024) is None
    want = S.candidate_pairs(packed, off, lens, k=8, lo=1, hi=1024)
    assert (want["a"] == 0).sum() == 2100
    same(run_emu(lib, "sort", packed, off, lens, 8, 1, 1024), want)
    packed, off, lens = pack(star_reads(2000))    # 2,000 partners fit (98% full)
    want = S.candidate_pairs(packed, off, lens, k=8, lo=1, hi=1024)
    same(run_emu(lib, "rows", packed, off, lens, 8, 1, 1024), want)


def test_rows_with_small_tables_and_heavy_probing(lib):
    """Tables just large enough (many collisions, long probe chains) still
    give the oracle's candidates."""
    reads = small_genome_reads(33, seed=77, glen=300, lo=40, hi=120, err=False)
    packed, off, lens = pack(reads)
    want = S.candidate_pairs(packed, off, lens, k=13, lo=1, hi=1024)
    max_partners = max(np.bincount(want["a"], minlength=len(reads)))
    lg = int(np.ceil(np.log2(max_partners)))
    same(run_emu(lib, "rows", packed, off, lens, 13, 1, 1024, table_lg=lg), want)
