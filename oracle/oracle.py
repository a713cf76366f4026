"""ctypes loader for the C oracle (TEST INFRASTRUCTURE ONLY).

``build()`` compiles ``xdrop_oracle.c`` with the host C compiler into
``liborc.so`` beside it; ``load()`` opens it.  The wrappers take numpy arrays
in the library's input layout (2-bit packed reads, read offsets in bases,
read lengths, 20-byte pair records) and return numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xdrop_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

# Record layouts of xdrop_oracle.h (declared here, not borrowed from the
# library's binding).
ORC_PAIR = np.dtype([("a", "<u4"), ("b", "<u4"), ("seed_a", "<u4"),
                     ("seed_b", "<u4"), ("seed_len", "<u4")])
ORC_RESULT = np.dtype([("left_score", "<i4"), ("left_begin_a", "<i4"),
                       ("left_begin_b", "<i4"), ("right_score", "<i4"),
                       ("right_end_a", "<i4"), ("right_end_b", "<i4"),
                       ("status", "<i4")])


class _Scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap", ctypes.c_int32), ("x", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no intrinsics) if it is stale."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-pthread",
               "-Wall", "-Wextra", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        lib.orc_extend.argtypes = [p, ctypes.c_int64, p, ctypes.c_int64,
                                   ctypes.POINTER(_Scoring),
                                   ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]
        lib.orc_extend.restype = ctypes.c_int
        lib.orc_unpack.argtypes = [p, ctypes.c_uint64, ctypes.c_uint64, p]
        lib.orc_unpack.restype = None
        lib.orc_align_pairs.argtypes = [p, p, p, ctypes.c_uint32, p,
                                        ctypes.c_size_t,
                                        ctypes.POINTER(_Scoring), p, p,
                                        ctypes.c_int]
        lib.orc_align_pairs.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _scoring(match, mismatch, gap, x):
    return _Scoring(int(match), int(mismatch), int(gap), int(x))


def extend(a, b, match=1, mismatch=-1, gap=-1, x=50):
    """One extension over code sequences a, b (0..3 per base).

    Returns (score, best_i, best_j, cells)."""
    lib = load()
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint8))
    s = _scoring(match, mismatch, gap, x)
    sc = ctypes.c_int32()
    bi, bj, cells = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = lib.orc_extend(_ptr(a if a.size else np.zeros(1, np.uint8)), a.size,
                        _ptr(b if b.size else np.zeros(1, np.uint8)), b.size,
                        ctypes.byref(s), ctypes.byref(sc), ctypes.byref(bi),
                        ctypes.byref(bj), ctypes.byref(cells))
    if rc != 0:
        raise ValueError("orc_extend rejected its arguments")
    return sc.value, bi.value, bj.value, cells.value


def unpack(packed, off, length):
    lib = load()
    packed = np.ascontiguousarray(packed, dtype=np.uint32)
    out = np.empty(max(int(length), 1), np.uint8)
    lib.orc_unpack(_ptr(packed), int(off), int(length), _ptr(out))
    return out[:int(length)]


def align_pairs(packed, read_off, read_len, pairs, match=1, mismatch=-1,
                gap=-1, x=50, nthreads=1, with_cells=False):
    """Seed-and-extend of every pair; returns a structured result array
    (and the per-extension cell counts, shape (n_pairs, 2), if asked)."""
    lib = load()
    packed = np.ascontiguousarray(packed, dtype=np.uint32)
    read_off = np.ascontiguousarray(read_off, dtype=np.uint64)
    read_len = np.ascontiguousarray(read_len, dtype=np.uint32)
    pairs = np.ascontiguousarray(pairs)
    if pairs.dtype.itemsize != ORC_PAIR.itemsize:
        raise TypeError("pair records must be 5 x uint32")
    n = pairs.shape[0]
    out = np.zeros(max(n, 1), ORC_RESULT)
    cells = np.zeros((max(n, 1), 2), np.int64) if with_cells else None
    s = _scoring(match, mismatch, gap, x)
    lib.orc_align_pairs(_ptr(packed), _ptr(read_off), _ptr(read_len),
                        len(read_len), _ptr(pairs), n, ctypes.byref(s),
                        _ptr(out), _ptr(cells) if cells is not None else None,
                        int(nthreads))
    out = out[:n]
    if with_cells:
        return out, cells[:n]
    return out


NO_BEST = 0xFFFFFFFF


def best_seeds(pairs, results, match=1):
    """Several seeds per read pair, keeping the best extension.

    Consecutive pair records with the same (a, b) (b with its strand flag)
    are the seeds of one read pair, a group.  The total score of a record
    is left_score + seed_len * match + right_score (seed-and-extend: the
    exact seed scores seed_len matches; Section "Related works", BELLA
    paragraph).  For every record p the result holds the index of the
    record of p's group with the highest total score among records with
    status 0; ties go to the lowest index; a group without such a record
    gives NO_BEST.  Plain loops over the definition."""
    pairs = np.asarray(pairs)
    results = np.asarray(results)
    n = len(pairs)
    best = np.full(n, NO_BEST, np.uint32)
    start = 0
    while start < n:
        end = start + 1
        while (end < n and pairs["a"][end] == pairs["a"][start]
               and pairs["b"][end] == pairs["b"][start]):
            end += 1
        winner, top = NO_BEST, None
        for p in range(start, end):
            if int(results["status"][p]) != 0:
                continue
            total = (int(results["left_score"][p]) + int(pairs["seed_len"][p]) * int(match)
                     + int(results["right_score"][p]))
            if top is None or total > top:
                winner, top = p, total
        best[start:end] = winner
        start = end
    return best


def accept(pairs, results, read_len, match=1, mismatch=-1, error_e4=1500, delta_e4=1000):
    """BELLA-style adaptive acceptance of each aligned pair (Section "Related
    works", BELLA paragraph: an adaptive threshold decides which X-drop
    alignments are kept; the paper gives no formula, so this is the reading
    fixed here, with every quantity an exact integer or rational):

      - total = left_score + seed_len * match + right_score;
      - L = the overlap the seed implies: min(seed_a, seed_b)
        + min(len_a - seed_a, len_b - seed_b) (positions and length of b on
        the strand the pair names);
      - with error rate e = error_e4 / 10^4 per read, a column of the
        overlap pairs two correct bases with probability phi = (1 - e)^2 and
        scores match then, mismatch otherwise: the expected score is
        L * (phi * match + (1 - phi) * mismatch);
      - accepted iff status is 0 and total >= (1 - delta) * expected, with
        delta = delta_e4 / 10^4.

    Returns uint8 flags.  Python integers throughout (no rounding)."""
    pairs = np.asarray(pairs)
    results = np.asarray(results)
    out = np.zeros(len(pairs), np.uint8)
    q = 10 ** 4
    for p in range(len(pairs)):
        if int(results["status"][p]) != 0:
            continue
        a, b = int(pairs["a"][p]), int(pairs["b"][p]) & 0x7FFFFFFF
        sa, sb = int(pairs["seed_a"][p]), int(pairs["seed_b"][p])
        la, lb = int(read_len[a]), int(read_len[b])
        L = min(sa, sb) + min(la - sa, lb - sb)
        total = (int(results["left_score"][p]) + int(pairs["seed_len"][p]) * int(match)
                 + int(results["right_score"][p]))
        phi_q2 = (q - int(error_e4)) ** 2                    # phi * 10^8
        exp_q2 = phi_q2 * int(match) + (q * q - phi_q2) * int(mismatch)
        # total >= (1 - delta) * L * expected, scaled by 10^12
        out[p] = 1 if total * q ** 3 >= (q - int(delta_e4)) * L * exp_q2 else 0
    return out
