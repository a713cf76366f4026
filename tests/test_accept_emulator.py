"""The acceptance kernel's per-pair arithmetic (csrc/xd_accept.cuh), run on
the CPU by tests/accept_emulator.cpp, against the oracle (oracle.accept) on
random and extreme inputs: scores near the threshold, error rates and slack
at 0 and 100%, heavy mismatch penalties, either strand."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    so = tmp_path_factory.mktemp("accept_emu") / "libaccept_emu.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-Wall", "-Werror", "-shared", "-fPIC", "-o", str(so),
                    os.path.join(HERE, "accept_emulator.cpp")], check=True)
    lib = ctypes.CDLL(str(so))
    vp, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32
    lib.emulate_accept.restype = None
    lib.emulate_accept.argtypes = [vp, vp, vp, u32, ctypes.c_uint64, i32, i32, u32, u32, vp]

    def run(pairs, res, lens, match, mismatch, e4, d4):
        pairs = np.ascontiguousarray(pairs)
        res = np.ascontiguousarray(res)
        lens = np.ascontiguousarray(lens, np.uint32)
        out = np.zeros(max(len(pairs), 1), np.uint8)
        lib.emulate_accept(pairs.ctypes.data, res.ctypes.data, lens.ctypes.data, len(lens),
                           len(pairs), match, mismatch, e4, d4, out.ctypes.data)
        return out[:len(pairs)]

    return run


def random_case(orc, rng, n=3000):
    n_reads = 50
    lens = rng.integers(0, 30000, n_reads).astype(np.uint32)
    pairs = np.zeros(n, orc.ORC_PAIR)
    pairs["a"] = rng.integers(0, n_reads, n)
    pairs["b"] = rng.integers(0, n_reads, n) | np.where(rng.random(n) < 0.5, 0x80000000, 0)
    pairs["seed_len"] = rng.integers(0, 40, n)
    la = lens[pairs["a"]].astype(np.int64)
    lb = lens[pairs["b"] & 0x7FFFFFFF].astype(np.int64)
    pairs["seed_a"] = (rng.random(n) * np.maximum(la - pairs["seed_len"], 0)).astype(np.uint32)
    pairs["seed_b"] = (rng.random(n) * np.maximum(lb - pairs["seed_len"], 0)).astype(np.uint32)
    res = np.zeros(n, orc.ORC_RESULT)
    res["left_score"] = rng.integers(-200, 20000, n)
    res["right_score"] = rng.integers(-200, 20000, n)
    res["status"] = np.where(rng.random(n) < 0.05, rng.integers(1, 3, n), 0)
    return pairs, res, lens


@pytest.mark.parametrize("match,mismatch", [(1, -1), (2, -3), (5, -4), (1, -1000), (3, 0)])
@pytest.mark.parametrize("e4,d4", [(0, 0), (1500, 1000), (10000, 0), (0, 10000), (333, 77),
                                   (9999, 1)])
def test_matches_oracle(orc, emu, match, mismatch, e4, d4):
    rng = np.random.default_rng(match * 1000 + e4 + d4)
    pairs, res, lens = random_case(orc, rng)
    want = orc.accept(pairs, res, lens, match, mismatch, e4, d4)
    got = emu(pairs, res, lens, match, mismatch, e4, d4)
    assert np.array_equal(got, want)


def test_scores_on_the_threshold(orc, emu):
    """Totals placed at the threshold and one either side: every pair sits
    exactly where integer rounding would go wrong."""
    rng = np.random.default_rng(9)
    pairs, res, lens = random_case(orc, rng, 2000)
    res["status"] = 0
    res["left_score"] = 0
    e4, d4 = 1500, 1000
    q = 10 ** 4
    for shift in (-1, 0, 1):
        for p in range(len(pairs)):
            a, b = int(pairs["a"][p]), int(pairs["b"][p]) & 0x7FFFFFFF
            sa, sb = int(pairs["seed_a"][p]), int(pairs["seed_b"][p])
            L = min(sa, sb) + min(int(lens[a]) - sa, int(lens[b]) - sb)
            phi = (q - e4) ** 2
            thr_num = (q - d4) * L * (phi - (q * q - phi))       # match 1, mismatch -1, x 10^12
            need = -(-thr_num // q ** 3)                          # smallest accepted total
            res["right_score"][p] = need + shift - int(pairs["seed_len"][p])
        want = orc.accept(pairs, res, lens, 1, -1, e4, d4)
        assert np.array_equal(emu(pairs, res, lens, 1, -1, e4, d4), want)
        assert want.all() if shift >= 0 else not want.any()
