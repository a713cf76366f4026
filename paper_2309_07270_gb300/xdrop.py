"""ctypes binding of libxdrop.so (argument marshalling only).

The functions carry the C ABI's names (include/xdrop.h).  Every step of the
alignment runs inside the library's CUDA kernels; if the library is
missing, or no GPU is visible, calls raise instead of computing anything
on the CPU.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libxdrop.so")

XDROP_OK = 0
XDROP_EINVAL = -1
XDROP_ENOMEM = -2
XDROP_ECUDA = -3
XDROP_ETIMEDOUT = -4
XDROP_EBUSY = -5
XDROP_MODE_BATCHED = 0
XDROP_MODE_PLAIN = 1
XDROP_MODE_SERVE = 2
XDROP_SEEDS_ROWWISE = 0
XDROP_SEEDS_SORT = 1
XDROP_STATUS_OK = 0
XDROP_STATUS_INVALID = 1
XDROP_STATUS_TOO_LONG = 2
XDROP_TILE_PACKED16 = 0x100  # xdrop_set_tile: 16-bit packed tile
XDROP_PAIR_RC = 0x80000000   # in a pair's b: the reverse strand of read b

PAIR_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("seed_a", "<u4"),
                       ("seed_b", "<u4"), ("seed_len", "<u4")])
RESULT_DTYPE = np.dtype([("left_score", "<i4"), ("left_begin_a", "<i4"),
                         ("left_begin_b", "<i4"), ("right_score", "<i4"),
                         ("right_end_a", "<i4"), ("right_end_b", "<i4"),
                         ("status", "<i4")])

EXPORTS = ["xdrop_init", "xdrop_submit", "xdrop_submit_device", "xdrop_sync",
           "xdrop_free", "xdrop_last_error", "xdrop_stream", "xdrop_get_stats",
           "xdrop_count_cells_device", "xdrop_last_spills", "xdrop_set_tile",
           "xdrop_align_static", "xdrop_static_last_error", "xdrop_load_reads",
           "xdrop_submit_pairs", "xdrop_get_serve_stats", "xdrop_best_seeds_device",
           "xdrop_find_candidates", "xdrop_get_seed_stats", "xdrop_accept_device",
           "xdrop_set_serve_idle"]


class XdropError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"xdrop error {code}: {msg}")
        self.code = code


class Scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap", ctypes.c_int32), ("x", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_double), ("main_kernel_ms", ctypes.c_double),
                ("tasks", ctypes.c_uint64),
                ("overflow_tasks", ctypes.c_uint64), ("wide_tasks", ctypes.c_uint64),
                ("launches", ctypes.c_uint32), ("graph_replays", ctypes.c_uint32),
                ("tile_lanes", ctypes.c_uint32), ("tile_cells", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_uint64), ("wide_passes", ctypes.c_uint64),
                ("relaunches", ctypes.c_uint64), ("max_in_flight", ctypes.c_uint64),
                ("admission_waits", ctypes.c_uint64), ("published", ctypes.c_uint64),
                ("consumed", ctypes.c_uint64), ("spill_reserved", ctypes.c_uint64),
                ("spill_taken", ctypes.c_uint64), ("ring_warps", ctypes.c_uint64),
                ("idle_exits", ctypes.c_uint64),
                ("help_sessions", ctypes.c_uint64),
                ("surplus_counts", ctypes.c_uint64)]


class KmerParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("stride", ctypes.c_uint32),
                ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class AcceptParams(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("error_e4", ctypes.c_uint32), ("delta_e4", ctypes.c_uint32)]


class SeedStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("occurrences", ctypes.c_uint64),
                ("runs", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("product", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("nonzeros", ctypes.c_uint64)]


_lib = None


def load():
    """Open libxdrop.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_2309_07270_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    lib.xdrop_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int, sz, u32]
    lib.xdrop_submit.argtypes = [vp, vp, vp, vp, u32, vp, sz, ctypes.POINTER(Scoring), vp,
                                 ctypes.POINTER(u64)]
    lib.xdrop_submit_device.argtypes = [vp, vp, u64, vp, vp, u32, vp, sz,
                                        ctypes.POINTER(Scoring), vp, ctypes.POINTER(u64)]
    lib.xdrop_sync.argtypes = [vp, u64, ctypes.c_int64]
    lib.xdrop_free.argtypes = [vp]
    lib.xdrop_free.restype = None
    lib.xdrop_last_error.argtypes = [vp]
    lib.xdrop_last_error.restype = ctypes.c_char_p
    lib.xdrop_stream.argtypes = [vp]
    lib.xdrop_stream.restype = vp
    lib.xdrop_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.xdrop_count_cells_device.argtypes = [vp, vp, u64, vp, vp, u32, vp, sz,
                                             ctypes.POINTER(Scoring), vp]
    lib.xdrop_last_spills.argtypes = [vp, vp, sz, ctypes.POINTER(sz)]
    lib.xdrop_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.xdrop_best_seeds_device.argtypes = [vp, vp, vp, sz, ctypes.c_int32, vp]
    lib.xdrop_load_reads.argtypes = [vp, vp, vp, vp, u32]
    lib.xdrop_submit_pairs.argtypes = [vp, vp, sz, ctypes.POINTER(Scoring), vp,
                                       ctypes.POINTER(u64)]
    lib.xdrop_get_serve_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
    lib.xdrop_set_serve_idle.argtypes = [vp, u64]
    lib.xdrop_find_candidates.argtypes = [vp, ctypes.POINTER(KmerParams), vp, vp, sz,
                                          ctypes.POINTER(sz)]
    lib.xdrop_get_seed_stats.argtypes = [vp, ctypes.POINTER(SeedStats)]
    lib.xdrop_accept_device.argtypes = [vp, vp, vp, sz, vp, u32, ctypes.POINTER(AcceptParams), vp]
    for name in ("xdrop_load_reads", "xdrop_submit_pairs", "xdrop_get_serve_stats",
                 "xdrop_best_seeds_device", "xdrop_find_candidates", "xdrop_get_seed_stats",
                 "xdrop_accept_device", "xdrop_set_serve_idle"):
        getattr(lib, name).restype = ctypes.c_int
    lib.xdrop_align_static.argtypes = [vp, u64, vp, vp, u32, vp, sz, ctypes.POINTER(Scoring),
                                       u32, vp, vp]
    lib.xdrop_align_static.restype = ctypes.c_int
    lib.xdrop_static_last_error.argtypes = []
    lib.xdrop_static_last_error.restype = ctypes.c_char_p
    for name in ("xdrop_set_tile", "xdrop_last_spills", "xdrop_init", "xdrop_submit", "xdrop_submit_device", "xdrop_sync",
                 "xdrop_get_stats", "xdrop_count_cells_device"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != XDROP_OK:
        msg = load().xdrop_last_error(ctx).decode()
        raise XdropError(rc, msg)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else ctypes.c_void_p(0)


def scoring(match=1, mismatch=-1, gap=-1, x=50) -> Scoring:
    return Scoring(int(match), int(mismatch), int(gap), int(x))


def xdrop_init(device=0, device_mem_budget=0, flags=XDROP_MODE_BATCHED):
    ctx = ctypes.c_void_p()
    _check(load().xdrop_init(ctypes.byref(ctx), int(device), int(device_mem_budget),
                             int(flags)))
    return ctx


def xdrop_submit(ctx, packed, read_off, read_len, pairs, sc: Scoring, out):
    """Host arrays (numpy).  ``out`` is a RESULT_DTYPE array the caller
    keeps alive until xdrop_sync returns."""
    packed = np.ascontiguousarray(packed, dtype=np.uint32)
    read_off = np.ascontiguousarray(read_off, dtype=np.uint64)
    read_len = np.ascontiguousarray(read_len, dtype=np.uint32)
    pairs = np.ascontiguousarray(pairs)
    if pairs.dtype.itemsize != 20 or out.dtype.itemsize != 28 or not out.flags.c_contiguous:
        raise TypeError("pairs must be 20-byte records and out a contiguous 28-byte-record array")
    t = ctypes.c_uint64()
    _check(load().xdrop_submit(ctx, _p(packed), _p(read_off), _p(read_len), len(read_len),
                               _p(pairs), len(pairs), ctypes.byref(sc), _p(out),
                               ctypes.byref(t)), ctx)
    return t.value


def xdrop_submit_device(ctx, packed_ptr, n_words, read_off_ptr, read_len_ptr, n_reads,
                        pairs_ptr, n_pairs, sc: Scoring, out_ptr):
    """Device pointers (ints, e.g. torch.Tensor.data_ptr())."""
    t = ctypes.c_uint64()
    _check(load().xdrop_submit_device(ctx, ctypes.c_void_p(packed_ptr), int(n_words),
                                      ctypes.c_void_p(read_off_ptr),
                                      ctypes.c_void_p(read_len_ptr), int(n_reads),
                                      ctypes.c_void_p(pairs_ptr), int(n_pairs),
                                      ctypes.byref(sc), ctypes.c_void_p(out_ptr),
                                      ctypes.byref(t)), ctx)
    return t.value


def xdrop_sync(ctx, ticket, timeout_ns=-1):
    _check(load().xdrop_sync(ctx, int(ticket), int(timeout_ns)), ctx)


def xdrop_free(ctx):
    load().xdrop_free(ctx)


def xdrop_last_error(ctx=None) -> str:
    return load().xdrop_last_error(ctx).decode()


def xdrop_stream(ctx) -> int:
    return int(load().xdrop_stream(ctx) or 0)


def xdrop_get_stats(ctx) -> dict:
    st = Stats()
    _check(load().xdrop_get_stats(ctx, ctypes.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in Stats._fields_}


def xdrop_count_cells_device(ctx, packed_ptr, n_words, read_off_ptr, read_len_ptr, n_reads,
                             pairs_ptr, n_pairs, sc: Scoring, cells_ptr):
    _check(load().xdrop_count_cells_device(ctx, ctypes.c_void_p(packed_ptr), int(n_words),
                                           ctypes.c_void_p(read_off_ptr),
                                           ctypes.c_void_p(read_len_ptr), int(n_reads),
                                           ctypes.c_void_p(pairs_ptr), int(n_pairs),
                                           ctypes.byref(sc), ctypes.c_void_p(cells_ptr)), ctx)


def xdrop_align_static(packed_ptr, n_words, read_off_ptr, read_len_ptr, n_reads, pairs_ptr,
                       n_pairs, sc: Scoring, max_read_len, out_ptr, stream=0):
    """Allocation-free alignment: device pointers (ints), enqueued on
    ``stream`` (a raw cudaStream_t value, 0 for the default stream)."""
    lib = load()
    rc = lib.xdrop_align_static(ctypes.c_void_p(packed_ptr), int(n_words),
                                ctypes.c_void_p(read_off_ptr), ctypes.c_void_p(read_len_ptr),
                                int(n_reads), ctypes.c_void_p(pairs_ptr), int(n_pairs),
                                ctypes.byref(sc), int(max_read_len), ctypes.c_void_p(out_ptr),
                                ctypes.c_void_p(stream))
    if rc != XDROP_OK:
        raise XdropError(rc, lib.xdrop_static_last_error().decode())


def xdrop_static_last_error() -> str:
    return load().xdrop_static_last_error().decode()


def xdrop_load_reads(ctx, packed, read_off, read_len):
    packed = np.ascontiguousarray(packed, dtype=np.uint32)
    read_off = np.ascontiguousarray(read_off, dtype=np.uint64)
    read_len = np.ascontiguousarray(read_len, dtype=np.uint32)
    _check(load().xdrop_load_reads(ctx, _p(packed), _p(read_off), _p(read_len), len(read_len)),
           ctx)


def xdrop_submit_pairs(ctx, pairs, sc: Scoring, out):
    """Host pairs against the resident reads; ``out`` (RESULT_DTYPE) must
    stay alive until xdrop_sync returns."""
    pairs = np.ascontiguousarray(pairs)
    if pairs.dtype.itemsize != 20 or out.dtype.itemsize != 28 or not out.flags.c_contiguous:
        raise TypeError("pairs must be 20-byte records and out a contiguous 28-byte-record array")
    t = ctypes.c_uint64()
    _check(load().xdrop_submit_pairs(ctx, _p(pairs), len(pairs), ctypes.byref(sc), _p(out),
                                     ctypes.byref(t)), ctx)
    return t.value


def xdrop_get_serve_stats(ctx) -> dict:
    st = ServeStats()
    _check(load().xdrop_get_serve_stats(ctx, ctypes.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in ServeStats._fields_}


def xdrop_set_serve_idle(ctx, idle_ns):
    """Serving hang guard: bound (ns) of a group's wait for work."""
    _check(load().xdrop_set_serve_idle(ctx, ctypes.c_uint64(int(idle_ns))), ctx)


def xdrop_set_tile(ctx, lanes, cells):
    _check(load().xdrop_set_tile(ctx, int(lanes), int(cells)), ctx)


def xdrop_best_seeds_device(ctx, pairs_ptr, results_ptr, n, match, best_ptr):
    _check(load().xdrop_best_seeds_device(ctx, pairs_ptr, results_ptr, int(n), int(match),
                                          best_ptr), ctx)


def xdrop_find_candidates(ctx, k=31, lo=20, hi=30, stride=1, rowwise=True):
    """Candidate pairs of the resident reads (pairs as PAIR_DTYPE, ready for
    xdrop_submit_pairs) and their shared reliable k-mer counts; ``rowwise``
    (the default) runs the row-wise product, False the sort-based one (same
    result)."""
    prm = KmerParams(int(k), int(stride), int(lo), int(hi),
                     XDROP_SEEDS_ROWWISE if rowwise else XDROP_SEEDS_SORT)
    n = ctypes.c_size_t()
    _check(load().xdrop_find_candidates(ctx, ctypes.byref(prm), None, None, 0, ctypes.byref(n)),
           ctx)
    pairs = np.zeros(n.value, PAIR_DTYPE)
    shared = np.zeros(n.value, np.uint32)
    if n.value:  # the context kept the result: this call only copies it
        _check(load().xdrop_find_candidates(ctx, ctypes.byref(prm), _p(pairs), _p(shared),
                                            n.value, ctypes.byref(n)), ctx)
    return pairs, shared


def xdrop_accept_device(ctx, pairs_ptr, results_ptr, n, read_len_ptr, n_reads, match, mismatch,
                        error_e4, delta_e4, accept_ptr):
    prm = AcceptParams(int(match), int(mismatch), int(error_e4), int(delta_e4))
    _check(load().xdrop_accept_device(ctx, pairs_ptr, results_ptr, int(n), read_len_ptr,
                                      int(n_reads), ctypes.byref(prm), accept_ptr), ctx)


def xdrop_get_seed_stats(ctx) -> dict:
    st = SeedStats()
    _check(load().xdrop_get_seed_stats(ctx, ctypes.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in SeedStats._fields_ if k != "pad"}


def xdrop_last_spills(ctx, cap=1 << 24) -> np.ndarray:
    n = ctypes.c_size_t()
    buf = np.zeros(max(int(cap), 1), np.uint32)
    _check(load().xdrop_last_spills(ctx, _p(buf), int(cap), ctypes.byref(n)), ctx)
    return buf[: min(int(n.value), int(cap))]


# ---------------------------------------------------------------------------
# Convenience layer over the C calls (still marshalling only).
# ---------------------------------------------------------------------------

class Aligner:
    """One library context.  ``align`` takes a workload in host memory,
    ``align_device`` one already resident on the GPU (see DeviceInputs)."""

    def __init__(self, device=0, mode=XDROP_MODE_BATCHED, budget=0):
        self.ctx = xdrop_init(device, budget, mode)
        self.mode = mode

    def close(self):
        if self.ctx is not None:
            xdrop_free(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def align(self, packed, read_off, read_len, pairs, sc: Scoring):
        out = np.zeros(len(pairs), RESULT_DTYPE)
        t = xdrop_submit(self.ctx, packed, read_off, read_len, pairs, sc, out)
        xdrop_sync(self.ctx, t)
        return out

    def submit_device(self, dev, sc: Scoring):
        return xdrop_submit_device(self.ctx, dev.packed.data_ptr(), dev.packed.numel(),
                                   dev.read_off.data_ptr(), dev.read_len.data_ptr(),
                                   dev.read_len.numel(), dev.pairs.data_ptr(),
                                   dev.n_pairs, sc, dev.out.data_ptr())

    def align_device(self, dev, sc: Scoring):
        t = self.submit_device(dev, sc)
        xdrop_sync(self.ctx, t)
        return dev.out

    def best_seeds_device(self, dev, match):
        """Best seed of every read pair of `dev` (see xdrop_best_seeds_device);
        returns a uint32 torch tensor, one index per pair record."""
        import torch
        best = torch.zeros(max(dev.n_pairs, 1), dtype=torch.int32, device=dev.packed.device)
        xdrop_best_seeds_device(self.ctx, dev.pairs.data_ptr(), dev.out.data_ptr(), dev.n_pairs,
                                match, best.data_ptr())
        torch.cuda.synchronize(dev.packed.device)
        return best[: dev.n_pairs]

    def find_candidates(self, packed, read_off, read_len, k=31, lo=20, hi=30, stride=1,
                        rowwise=True):
        """Load a read set and return its candidate pairs and shared counts
        (xdrop_find_candidates); the reads stay resident for submit_pairs."""
        xdrop_load_reads(self.ctx, packed, read_off, read_len)
        return xdrop_find_candidates(self.ctx, k, lo, hi, stride, rowwise)

    def accept_device(self, dev, sc: Scoring, error_e4=1500, delta_e4=1000):
        """Adaptive acceptance flag of every pair of `dev` from the results
        in dev.out (see xdrop_accept_device); returns a uint8 torch tensor."""
        import torch
        acc = torch.zeros(max(dev.n_pairs, 1), dtype=torch.uint8, device=dev.packed.device)
        xdrop_accept_device(self.ctx, dev.pairs.data_ptr(), dev.out.data_ptr(), dev.n_pairs,
                            dev.read_len.data_ptr(), dev.read_len.numel(), sc.match, sc.mismatch,
                            error_e4, delta_e4, acc.data_ptr())
        torch.cuda.synchronize(dev.packed.device)
        return acc[: dev.n_pairs]

    def count_cells_device(self, dev, sc: Scoring):
        import torch
        cells = torch.zeros(2 * max(dev.n_pairs, 1), dtype=torch.int64, device=dev.packed.device)
        xdrop_count_cells_device(self.ctx, dev.packed.data_ptr(), dev.packed.numel(),
                                 dev.read_off.data_ptr(), dev.read_len.data_ptr(),
                                 dev.read_len.numel(), dev.pairs.data_ptr(), dev.n_pairs, sc,
                                 cells.data_ptr())
        return cells[: 2 * dev.n_pairs]

    def stats(self):
        return xdrop_get_stats(self.ctx)

    def set_tile(self, lanes, cells):
        xdrop_set_tile(self.ctx, lanes, cells)

    def tile(self):
        st = self.stats()
        return int(st["tile_lanes"]), int(st["tile_cells"])

    def stream(self):
        return xdrop_stream(self.ctx)


class DeviceInputs:
    """Workload arrays in torch CUDA tensors (torch is the allocator only)."""

    def __init__(self, packed, read_off, read_len, pairs, device="cuda:0"):
        import torch
        self.packed = torch.from_numpy(np.ascontiguousarray(packed, np.uint32).view(np.int32)).to(device)
        self.read_off = torch.from_numpy(np.ascontiguousarray(read_off, np.uint64).view(np.int64)).to(device)
        self.read_len = torch.from_numpy(np.ascontiguousarray(read_len, np.uint32).view(np.int32)).to(device)
        pr = np.ascontiguousarray(pairs).view(np.int32).reshape(-1)
        self.pairs = torch.from_numpy(pr.copy()).to(device)
        self.n_pairs = len(pairs)
        self.out = torch.zeros(max(self.n_pairs, 1) * 7, dtype=torch.int32, device=device)

    def results(self) -> np.ndarray:
        a = self.out[: self.n_pairs * 7].cpu().numpy()
        return a.view(RESULT_DTYPE).reshape(-1)

    @classmethod
    def from_workload(cls, w, device="cuda:0"):
        return cls(w.packed, w.read_off, w.read_len, w.pairs, device)
