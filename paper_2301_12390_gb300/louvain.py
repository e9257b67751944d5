"""ctypes binding of the engine's C ABI (include/louvain.h).

Argument marshalling only: every step of the method runs in the CUDA library
libgblouvain.so.  If that library is missing this module raises; there is no
CPU fallback.  Function names are the C names; :class:`Louvain` is a small
convenience wrapper over them.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgblouvain.so")

SYNC, ASYNC = 0, 1
PTR_HOST, PTR_DEVICE = 0, 1

ERRORS = {
    -1: "INVALID_ARG", -2: "NOT_SYMMETRIC", -3: "BAD_CSR", -4: "OOM", -5: "CUDA", -6: "TIMEOUT", -7: "STATE",
    -8: "OVERFLOW", -9: "INTERNAL", -10: "CAPACITY",
}
STATIC_MAX_VERTICES = 1 << 20   # LOUVAIN_STATIC_MAX_VERTICES


class LouvainError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tolerance", ctypes.c_double), ("tolerance_decline", ctypes.c_double),
                ("pass_tolerance", ctypes.c_double), ("max_iterations", ctypes.c_int32),
                ("max_passes", ctypes.c_int32), ("prune", ctypes.c_int32), ("singleton_guard", ctypes.c_int32),
                ("subrounds", ctypes.c_int32), ("validate", ctypes.c_int32), ("record_levels", ctypes.c_int32),
                ("cuda_graphs", ctypes.c_int32), ("reclass", ctypes.c_int32), ("bucket_streams", ctypes.c_int32),
                ("colour_classes", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("reserved_d", ctypes.c_double * 4)]


class Stats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("iterations", ctypes.c_int32), ("moves", ctypes.c_int64),
                ("lm_edges", ctypes.c_int64), ("communities", ctypes.c_int64), ("q", ctypes.c_double),
                ("lm_ms", ctypes.c_double), ("agg_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("lm_vertices", ctypes.c_int64), ("lm_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("lm_candidates", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


class PassInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("k", ctypes.c_int64), ("moves", ctypes.c_int64),
                ("iterations", ctypes.c_int32), ("level_recorded", ctypes.c_int32), ("coarse_built", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("coarse_nnz", ctypes.c_int64), ("n_before_hi", ctypes.c_int64),
                ("n_before_lo", ctypes.c_uint64), ("n_after_hi", ctypes.c_int64), ("n_after_lo", ctypes.c_uint64),
                ("lm_ms", ctypes.c_double), ("agg_ms", ctypes.c_double)]


_lib = None

# (name, restype, argtypes) of every exported function
_VP, _I64, _I32, _U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
SIGNATURES = [
    ("louvain_default_options", _I32, [ctypes.POINTER(Options)]),
    ("louvain_create", _I32, [ctypes.POINTER(_VP), ctypes.POINTER(Options), _I32, _VP]),
    ("louvain_set_options", _I32, [_VP, ctypes.POINTER(Options)]),
    ("louvain_load_csr", _I32, [_VP, _I64, _I64, _VP, _VP, _VP, _I32]),
    ("louvain_run", _I32, [_VP]),
    ("louvain_get_membership", _I32, [_VP, _VP, _I64, _I32]),
    ("louvain_get_modularity", _I32, [_VP, ctypes.POINTER(ctypes.c_double)]),
    ("louvain_get_modularity_exact", _I32, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_U64), ctypes.POINTER(_I64)]),
    ("louvain_modularity", _I32, [_VP, _VP, _I64, _I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64),
                                  ctypes.POINTER(_U64), ctypes.POINTER(_I64)]),
    ("louvain_modularity_static", _I32, [_I64, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(_I64), ctypes.POINTER(_U64), ctypes.POINTER(_I64)]),
    ("louvain_load_batch", _I32, [_VP, _I64, _VP, _I64, _I64, _VP, _VP, _VP, _I32]),
    ("louvain_get_num_graphs", _I32, [_VP, ctypes.POINTER(_I64)]),
    ("louvain_batch_get_modularity", _I32, [_VP, _VP, _VP, _VP, _VP]),
    ("louvain_batch_get_graph_info", _I32, [_VP, _I64, _VP]),
    ("louvain_batch_get_iterations", _I32, [_VP, _I64, _VP, _I64, ctypes.POINTER(_I64)]),
    ("louvain_get_stats", _I32, [_VP, ctypes.POINTER(Stats)]),
    ("louvain_get_pass_info", _I32, [_VP, _I32, ctypes.POINTER(PassInfo)]),
    ("louvain_get_iteration", _I32, [_VP, _I64, _VP]),
    ("louvain_get_level", _I32, [_VP, _I32, _VP, _I64]),
    ("louvain_get_coarse", _I32, [_VP, _I32, _VP, _I64, _VP, _VP, _I64]),
    ("louvain_get_device_bytes", _I32, [_VP, ctypes.POINTER(_I64)]),
    ("louvain_destroy", None, [_VP]),
    ("louvain_last_error", ctypes.c_char_p, [_VP]),
    ("louvain_version", ctypes.c_char_p, []),
]


def load_library(path: str = LIB_PATH):
    """Load libgblouvain.so and declare its functions; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA engine library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_options(**kw) -> Options:
    o = Options()
    load_library().louvain_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


@dataclass
class PassRecord:
    n: int
    nnz: int
    k: int
    moves: int
    iterations: int
    n_before: int
    n_after: int
    coarse_built: bool
    coarse_nnz: int
    lm_ms: float
    agg_ms: float


def _i128(hi, lo) -> int:
    return (int(hi) << 64) + (int(lo) & ((1 << 64) - 1))


class Louvain:
    """One engine context on a CUDA device.

    Inputs may be numpy arrays (host) or CUDA torch tensors (device); the
    engine copies them.  `stream` is a cudaStream_t handle (int) or None.
    """

    def __init__(self, device: int = 0, stream: Optional[int] = None, **options):
        self.lib = load_library()
        self.opt = default_options(**options)
        h = ctypes.c_void_p()
        rc = self.lib.louvain_create(ctypes.byref(h), ctypes.byref(self.opt), device, stream or None)
        if rc:
            raise LouvainError(rc, "louvain_create failed")
        self.h = h
        self.n = None

    def _check(self, rc):
        if rc:
            raise LouvainError(rc, self.lib.louvain_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.louvain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **options):
        for k, v in options.items():
            if not hasattr(self.opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(self.opt, k, v)
        self._check(self.lib.louvain_set_options(self.h, ctypes.byref(self.opt)))

    def load_csr(self, off, col, w):
        dev = _is_device(off)
        if not dev:
            off = np.ascontiguousarray(off, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            w = np.ascontiguousarray(w, dtype=np.int32)
        n = len(off) - 1
        nnz = len(col)
        self._keep = (off, col, w)
        self._check(self.lib.louvain_load_csr(self.h, n, nnz, _ptr(off), _ptr(col), _ptr(w),
                                              PTR_DEVICE if dev else PTR_HOST))
        self._keep = None
        self.n = n

    def load_batch(self, graph_offsets, off, col, w):
        """Load graphs g = 0..G-1 owning vertices [graph_offsets[g], graph_offsets[g+1]) of one CSR."""
        dev = _is_device(off)
        if not dev:
            off = np.ascontiguousarray(off, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            w = np.ascontiguousarray(w, dtype=np.int32)
            graph_offsets = np.ascontiguousarray(graph_offsets, dtype=np.int64)
        n = len(off) - 1
        G = len(graph_offsets) - 1
        self._keep = (graph_offsets, off, col, w)
        self._check(self.lib.louvain_load_batch(self.h, G, _ptr(graph_offsets), n, len(col), _ptr(off), _ptr(col),
                                                _ptr(w), PTR_DEVICE if dev else PTR_HOST))
        self._keep = None
        self.n = n
        self.G = G

    def num_graphs(self) -> int:
        g = ctypes.c_int64()
        self._check(self.lib.louvain_get_num_graphs(self.h, ctypes.byref(g)))
        return g.value

    def load_parts(self, graphs):
        """Load graphs [(off, col, w), ...] (host arrays, ids local to each graph) as one batch, copied graph by
        graph to the device (no host-side concatenation)."""
        G = len(graphs)
        arrs = [(np.ascontiguousarray(o, np.int64), np.ascontiguousarray(c, np.int32), np.ascontiguousarray(w, np.int32))
                for o, c, w in graphs]
        ns = np.array([len(o) - 1 for o, _, _ in arrs], np.int64)
        nnzs = np.array([len(c) for _, c, _ in arrs], np.int64)
        P = ctypes.c_void_p * G
        offs = P(*[o.ctypes.data for o, _, _ in arrs])
        cols = P(*[c.ctypes.data for _, c, _ in arrs])
        ws = P(*[w.ctypes.data for _, _, w in arrs])
        self._check(self.lib.louvain_load_parts(self.h, G, ns.ctypes.data, nnzs.ctypes.data, offs, cols, ws))
        self.n = int(ns.sum())

    def batch_modularity(self):
        """(q[G] float64, exact numerators [G] python ints, M[G])."""
        G = self.num_graphs()
        q = np.empty(G, np.float64)
        hi = np.empty(G, np.int64)
        lo = np.empty(G, np.uint64)
        M = np.empty(G, np.int64)
        self._check(self.lib.louvain_batch_get_modularity(self.h, q.ctypes.data, hi.ctypes.data, lo.ctypes.data,
                                                          M.ctypes.data))
        return q, [_i128(a, b) for a, b in zip(hi.tolist(), lo.tolist())], M

    def batch_graph_info(self, g: int):
        out = np.zeros(4, np.int64)
        self._check(self.lib.louvain_batch_get_graph_info(self.h, g, out.ctypes.data))
        return {"passes": int(out[0]), "iterations": int(out[1]), "communities": int(out[2]), "moves": int(out[3])}

    def batch_iterations(self, g: int):
        cnt = ctypes.c_int64()
        self._check(self.lib.louvain_batch_get_iterations(self.h, g, None, 0, ctypes.byref(cnt)))
        buf = np.zeros(4 * max(cnt.value, 1), np.int64)
        self._check(self.lib.louvain_batch_get_iterations(self.h, g, buf.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return [(int(buf[4 * t]), int(buf[4 * t + 1]), _i128(buf[4 * t + 2], buf[4 * t + 3])) for t in range(cnt.value)]

    def run(self):
        self._check(self.lib.louvain_run(self.h))

    def run_partitioned(self, parts: int) -> float:
        """Partition, then merge: parts' induced subgraphs run as one batch, then the whole graph from their
        communities. Returns the parts' run time in ms."""
        ms = ctypes.c_double()
        self._check(self.lib.louvain_run_partitioned(self.h, parts, ctypes.byref(ms)))
        return ms.value

    def run_from(self, memb):
        """Incremental re-run: pass 0 starts from membership memb (host array or device tensor, n entries)."""
        if not _is_device(memb):
            memb = np.ascontiguousarray(memb, dtype=np.int32)
        self._check(self.lib.louvain_run_from(self.h, _ptr(memb), self.n,
                                              PTR_DEVICE if _is_device(memb) else PTR_HOST))

    def membership(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n, np.int32)
        self._check(self.lib.louvain_get_membership(self.h, _ptr(out), self.n,
                                                    PTR_DEVICE if _is_device(out) else PTR_HOST))
        return out

    def modularity(self) -> float:
        q = ctypes.c_double()
        self._check(self.lib.louvain_get_modularity(self.h, ctypes.byref(q)))
        return q.value

    def modularity_exact(self):
        hi, lo, M = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
        self._check(self.lib.louvain_get_modularity_exact(self.h, ctypes.byref(hi), ctypes.byref(lo), ctypes.byref(M)))
        return _i128(hi.value, lo.value), M.value

    def modularity_of(self, memb):
        """(Q, exact numerator, M) of an arbitrary membership of the loaded graph, on the device."""
        dev = _is_device(memb)
        if not dev:
            memb = np.ascontiguousarray(memb, dtype=np.int32)
        q, hi, lo, M = ctypes.c_double(), ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
        self._check(self.lib.louvain_modularity(self.h, _ptr(memb), self.n, PTR_DEVICE if dev else PTR_HOST,
                                                ctypes.byref(q), ctypes.byref(hi), ctypes.byref(lo), ctypes.byref(M)))
        return q.value, _i128(hi.value, lo.value), M.value

    def stats(self) -> Stats:
        s = Stats()
        self._check(self.lib.louvain_get_stats(self.h, ctypes.byref(s)))
        return s

    def passes(self) -> List[PassRecord]:
        out = []
        st = self.stats()
        for p in range(st.passes):
            pi = PassInfo()
            self._check(self.lib.louvain_get_pass_info(self.h, p, ctypes.byref(pi)))
            out.append(PassRecord(pi.n, pi.nnz, pi.k, pi.moves, pi.iterations, _i128(pi.n_before_hi, pi.n_before_lo),
                                  _i128(pi.n_after_hi, pi.n_after_lo), bool(pi.coarse_built), pi.coarse_nnz,
                                  pi.lm_ms, pi.agg_ms))
        return out

    def set_mapping(self, thresholds=None):
        """Local-moving degree thresholds (5 increasing ints within the kernels' capacities; None = defaults)."""
        if thresholds is None:
            self._check(self.lib.louvain_set_mapping(self.h, None))
            return
        t = np.ascontiguousarray(thresholds, dtype=np.int32)
        if t.shape != (5,):
            raise ValueError("five thresholds")
        self._check(self.lib.louvain_set_mapping(self.h, t.ctypes.data))

    def mapping(self):
        t = np.zeros(5, np.int32)
        self._check(self.lib.louvain_get_mapping(self.h, t.ctypes.data))
        return t.tolist()

    def autotune(self):
        """Pick the fastest local-moving mapping for the loaded graph; returns (thresholds, best trial ms)."""
        t = np.zeros(5, np.int32)
        ms = ctypes.c_double()
        self._check(self.lib.louvain_autotune(self.h, t.ctypes.data, ctypes.byref(ms)))
        return t.tolist(), ms.value

    def iterations(self):
        """[(pass, moves, S exact)] of every local-moving iteration of the last run."""
        st = self.stats()
        buf = np.zeros(4, np.int64)
        out = []
        for t in range(st.iterations):
            self._check(self.lib.louvain_get_iteration(self.h, t, buf.ctypes.data))
            out.append((int(buf[0]), int(buf[1]), _i128(buf[2], buf[3])))
        return out

    def level(self, p: int, n: int) -> np.ndarray:
        out = np.empty(n, np.int32)
        self._check(self.lib.louvain_get_level(self.h, p, out.ctypes.data, n))
        return out

    def coarse(self, p: int, k: int, nnz: int):
        off = np.empty(k + 1, np.int64)
        col = np.empty(max(nnz, 1), np.int32)
        w = np.empty(max(nnz, 1), np.int64)
        self._check(self.lib.louvain_get_coarse(self.h, p, off.ctypes.data, k, col.ctypes.data, w.ctypes.data, nnz))
        return off, col[:nnz], w[:nnz]

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.louvain_get_device_bytes(self.h, ctypes.byref(b)))
        return b.value


def modularity_static(off, col, w, memb, stream=None):
    """louvain_modularity_static on CUDA tensors (device pointers): (Q, exact numerator, M).

    offsets int64 (n + 1), cols / weights / memb int32, contiguous, on the
    device that is current.  `stream` is a torch.cuda.Stream, a raw
    cudaStream_t handle (int) or None (the default stream).  Allocates no
    device memory; include/louvain.h says who needs that and gives the limits
    (fixed capacity, calls must not overlap on the GPU)."""
    lib = load_library()
    want = (("offsets", off, "torch.int64"), ("cols", col, "torch.int32"), ("weights", w, "torch.int32"),
            ("memb", memb, "torch.int32"))
    dev = None
    for name, t, dt in want:
        if not hasattr(t, "is_cuda") or not t.is_cuda:
            raise TypeError(f"modularity_static: {name} must be a CUDA tensor")
        if str(t.dtype) != dt:
            raise TypeError(f"modularity_static: {name} must be {dt}, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"modularity_static: {name} must be contiguous")
        if dev is not None and t.device != dev:
            raise ValueError("modularity_static: all tensors must be on one device")
        dev = t.device
    n = len(off) - 1
    if len(memb) != n:
        raise ValueError("modularity_static: memb must have one entry per vertex")
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream   # a torch.cuda.Stream
    q, hi, lo, M = ctypes.c_double(), ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
    rc = lib.louvain_modularity_static(n, _ptr(off), _ptr(col), _ptr(w), _ptr(memb), stream or None,
                                       ctypes.byref(q), ctypes.byref(hi), ctypes.byref(lo), ctypes.byref(M))
    if rc:
        raise LouvainError(rc, "louvain_modularity_static failed")
    return q.value, _i128(hi.value, lo.value), M.value


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("batch_max_graphs", ctypes.c_int32), ("batch_max_entries", ctypes.c_int64),
                ("hbm_budget_bytes", ctypes.c_int64), ("borrow_inputs", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


class ServerResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("n", ctypes.c_int64), ("communities", ctypes.c_int64), ("q", ctypes.c_double),
                ("num_hi", ctypes.c_int64), ("num_lo", ctypes.c_uint64), ("M", ctypes.c_int64),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


SIGNATURES += [
    ("louvain_set_mapping", _I32, [_VP, _VP]),
    ("louvain_get_mapping", _I32, [_VP, _VP]),
    ("louvain_autotune", _I32, [_VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("louvain_run_from", _I32, [_VP, _VP, _I64, _I32]),
    ("louvain_load_parts", _I32, [_VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    ("louvain_run_partitioned", _I32, [_VP, _I64, ctypes.POINTER(ctypes.c_double)]),
]


SIGNATURES += [
    ("louvain_arena_bytes", _I32, [_I64, _I64, ctypes.POINTER(_I64)]),
    ("louvain_server_default_config", _I32, [ctypes.POINTER(ServerConfig)]),
    ("louvain_server_create", _I32, [ctypes.POINTER(_VP), ctypes.POINTER(Options), ctypes.POINTER(ServerConfig), _I32]),
    ("louvain_server_submit", _I32, [_VP, _I64, _I64, _I64, _VP, _VP, _VP]),
    ("louvain_server_poll", _I32, [_VP, ctypes.POINTER(ServerResult), _I64, ctypes.POINTER(_I64), _I32]),
    ("louvain_server_membership", _I32, [_VP, _I64, _VP, _I64]),
    ("louvain_server_stats", _I32, [_VP, _VP]),
    ("louvain_server_destroy", None, [_VP]),
    ("louvain_server_timings", _I32, [_VP, _VP]),
]


class Server:
    """Continuous-batching request server (louvain_server_*): submit host CSR graphs at any
    time, poll finished results; each result equals the graph's result alone."""

    def __init__(self, device: int = 0, slots: int = 2, batch_max_entries=None, batch_max_graphs=None,
                 hbm_budget_bytes=None, borrow_inputs=False, **options):
        self.lib = load_library()
        self.opt = default_options(**options)
        cfg = ServerConfig()
        self.lib.louvain_server_default_config(ctypes.byref(cfg))
        cfg.slots = slots
        if batch_max_entries is not None:
            cfg.batch_max_entries = batch_max_entries
        if batch_max_graphs is not None:
            cfg.batch_max_graphs = batch_max_graphs
        if hbm_budget_bytes is not None:
            cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.borrow_inputs = 1 if borrow_inputs else 0
        self.cfg_borrow = bool(borrow_inputs)
        self._borrowed = {}   # borrowed inputs stay referenced until their result is polled
        h = ctypes.c_void_p()
        rc = self.lib.louvain_server_create(ctypes.byref(h), ctypes.byref(self.opt), ctypes.byref(cfg), device)
        if rc:
            raise LouvainError(rc, "louvain_server_create failed")
        self.h = h
        self._n = {}

    def submit(self, request_id: int, off, col, w):
        off = np.ascontiguousarray(off, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int32)
        rc = self.lib.louvain_server_submit(self.h, request_id, len(off) - 1, len(col), off.ctypes.data,
                                            col.ctypes.data, w.ctypes.data)
        if rc:
            raise LouvainError(rc, f"submit of request {request_id} failed")
        self._n[request_id] = len(off) - 1
        if self.cfg_borrow:
            self._borrowed[request_id] = (off, col, w)

    def poll(self, wait_ms: int = 0, cap: int = 1024):
        buf = (ServerResult * cap)()
        cnt = ctypes.c_int64()
        self.lib.louvain_server_poll(self.h, buf, cap, ctypes.byref(cnt), wait_ms)
        out = []
        for r in buf[:cnt.value]:
            self._borrowed.pop(r.request_id, None)
            out.append({"id": r.request_id, "status": r.status, "batch_size": r.batch_size, "n": r.n,
                        "communities": r.communities, "q": r.q, "num": _i128(r.num_hi, r.num_lo), "M": r.M,
                        "submit_s": r.submit_s, "start_s": r.start_s, "done_s": r.done_s})
        return out

    def membership(self, request_id: int) -> np.ndarray:
        n = self._n.pop(request_id)
        out = np.empty(n, np.int32)
        rc = self.lib.louvain_server_membership(self.h, request_id, out.ctypes.data, n)
        if rc:
            raise LouvainError(rc, f"no membership for request {request_id}")
        return out

    def stats(self):
        out = np.zeros(8, np.int64)
        self.lib.louvain_server_stats(self.h, out.ctypes.data)
        keys = ["submitted", "finished", "runs", "queued", "reserved_bytes", "peak_reserved_bytes", "budget_bytes",
                "slots"]
        return dict(zip(keys, out.tolist()))

    def timings(self):
        """Seconds summed over all runs: host batch assembly, load, run, result fetch."""
        out = np.zeros(4, np.float64)
        self.lib.louvain_server_timings(self.h, out.ctypes.data)
        return dict(zip(["assemble_s", "load_s", "run_s", "fetch_s"], out.tolist()))

    def close(self):
        if getattr(self, "h", None):
            self.lib.louvain_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def arena_bytes(n: int, nnz: int) -> int:
    b = ctypes.c_int64()
    load_library().louvain_arena_bytes(n, nnz, ctypes.byref(b))
    return b.value
