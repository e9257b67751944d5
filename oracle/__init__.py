"""Oracle: plain single-threaded Louvain (louvain_oracle.c) and exact helpers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  It
shares no code with the CUDA engine and never imports it.

The method follows Section 3.2 of the paper (local-moving and aggregation
phases, passes, threshold scaling with tolerance 0.01 and decline factor 10,
synchronous and asynchronous variants); see the header of louvain_oracle.c for
the formulas (Newman-Girvan modularity; the paper writes none) and the
readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "louvain_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

SYNC, ASYNC = 0, 1


_MT_SRC = os.path.join(_HERE, "louvain_mt.c")
_MT_LIB = os.path.join(_HERE, "liblouvain_mt.so")
_mt_lib = None


def build(force: bool = False) -> str:
    """Compile louvain_oracle.c into liboracle.so (gcc; no FMA contraction), and
    the multi-threaded CPU baseline louvain_mt.c into liblouvain_mt.so (OpenMP
    where the compiler has it, else one thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    if force or not os.path.exists(_MT_LIB) or os.path.getmtime(_MT_LIB) < os.path.getmtime(_MT_SRC):
        tmp = _MT_LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _MT_SRC]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _MT_LIB)
    return _LIB


class Options(ctypes.Structure):
    """Run options; defaults are the paper's (tolerance 0.01, decline 10, pass tolerance 0)."""
    _fields_ = [("mode", ctypes.c_int), ("tolerance", ctypes.c_double), ("tolerance_decline", ctypes.c_double),
                ("pass_tolerance", ctypes.c_double), ("max_iterations", ctypes.c_int),
                ("max_passes", ctypes.c_int), ("prune", ctypes.c_int), ("singleton_guard", ctypes.c_int),
                ("subrounds", ctypes.c_int), ("colour_classes", ctypes.c_int), ("stop_rule", ctypes.c_int)]

    @classmethod
    def make(cls, mode=SYNC, tolerance=0.01, tolerance_decline=10.0, pass_tolerance=0.0, max_iterations=20,
             max_passes=10, prune=0, singleton_guard=1, subrounds=1, colour_classes=0, stop_rule=0):
        return cls(mode, tolerance, tolerance_decline, pass_tolerance, max_iterations, max_passes, prune,
                   singleton_guard, subrounds, colour_classes, stop_rule)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.or_modularity.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.or_modularity.restype = i32
        lib.or_vertex_gains.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp, i64]
        lib.or_vertex_gains.restype = i64
        lib.or_louvain.argtypes = [i64, vp, vp, vp, ctypes.POINTER(Options), i32]
        lib.or_louvain.restype = vp
        lib.or_louvain_from.argtypes = [i64, vp, vp, vp, ctypes.POINTER(Options), i32, vp]
        lib.or_louvain_from.restype = vp
        lib.or_free.argtypes = [vp]
        lib.or_result_summary.argtypes = [vp, vp, vp]
        lib.or_result_top.argtypes = [vp, vp]
        lib.or_result_pass.argtypes = [vp, i32, vp]
        lib.or_result_iter.argtypes = [vp, i64, vp]
        lib.or_result_level.argtypes = [vp, i32, vp]
        lib.or_result_coarse.argtypes = [vp, i32, vp, vp, vp]
        lib.or_aggregate.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp, i64, vp]
        lib.or_aggregate.restype = i32
        lib.or_brute_best.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        lib.or_brute_best.restype = i32
        lib.or_colour_classes.argtypes = [i64, vp, vp, i32, vp]
        lib.or_colour_classes.restype = i32
        _lib = lib
    return _lib


def _i128(hi: int, lo: int) -> int:
    return (int(hi) << 64) + (int(lo) & ((1 << 64) - 1))


def _arrs(off, col, w):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int64)
    return off, col, w


@dataclass
class Pass:
    n: int
    nnz: int
    k: int
    moves: int
    iterations: int
    n_before: int   # exact Q numerator before the pass (singletons of the pass graph)
    n_after: int    # exact Q numerator after local-moving
    level: Optional[np.ndarray] = None          # renumbered membership of the pass graph
    coarse: Optional[tuple] = None               # (off, col, w int64) built from this pass


@dataclass
class Result:
    top: np.ndarray
    M: int
    q_num: int
    Q: float
    passes: List[Pass] = field(default_factory=list)
    iterations: List[tuple] = field(default_factory=list)   # (pass, moves, S exact)


def louvain(off, col, w, mode=SYNC, tolerance=0.01, tolerance_decline=10.0, pass_tolerance=0.0,
            max_iterations=20, max_passes=10, prune=0, singleton_guard=1, subrounds=1,
            record_levels=False, initial=None, colour_classes=0, stop_rule=0) -> Result:
    """Run the oracle Louvain; exact integers for every recorded quantity.

    singleton_guard, subrounds and colour_classes apply to the synchronous
    mode only (colour_classes: the classes are colour_classes() of every pass
    graph instead of i mod subrounds).
    initial: a membership of the input (values in [0, n)) that pass 0 starts
    from instead of singletons (an incremental re-run).
    stop_rule: what an iteration's "total change in modularity" (Section 3.2)
    is: 0 = 2S/M^2, S the sum of the movers' gains; 1 = the exact change of
    the Q numerator over the iteration, recomputed from the membership, / M^2."""
    lib = _load()
    off, col, w = _arrs(off, col, w)
    n = len(off) - 1
    opt = Options.make(mode, tolerance, tolerance_decline, pass_tolerance, max_iterations, max_passes, prune,
                       singleton_guard, subrounds, int(colour_classes), int(stop_rule))
    init = None
    if initial is not None:
        init = np.ascontiguousarray(initial, dtype=np.int32)
        if init.shape != (n,):
            raise ValueError("initial membership must have n entries")
    h = lib.or_louvain_from(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, ctypes.byref(opt),
                            int(record_levels), None if init is None else init.ctypes.data)
    if not h:
        raise ValueError("oracle: invalid options")
    try:
        s = np.zeros(8, np.int64)
        q = ctypes.c_double()
        lib.or_result_summary(h, s.ctypes.data, ctypes.byref(q))
        top = np.empty(n, np.int32)
        lib.or_result_top(h, top.ctypes.data)
        res = Result(top=top, M=int(s[1]), q_num=_i128(s[2], s[3]), Q=q.value)
        for p in range(int(s[4])):
            a = np.zeros(12, np.int64)
            lib.or_result_pass(h, p, a.ctypes.data)
            ps = Pass(n=int(a[0]), nnz=int(a[1]), k=int(a[2]), moves=int(a[3]), iterations=int(a[4]),
                      n_before=_i128(a[8], a[9]), n_after=_i128(a[10], a[11]))
            if a[5]:
                lv = np.empty(ps.n, np.int32)
                lib.or_result_level(h, p, lv.ctypes.data)
                ps.level = lv
            if a[6]:
                co = np.empty(ps.k + 1, np.int64)
                cc = np.empty(max(int(a[7]), 1), np.int32)
                cw = np.empty(max(int(a[7]), 1), np.int64)
                lib.or_result_coarse(h, p, co.ctypes.data, cc.ctypes.data, cw.ctypes.data)
                ps.coarse = (co, cc[:int(a[7])], cw[:int(a[7])])
            res.passes.append(ps)
        for t in range(int(s[5])):
            a = np.zeros(4, np.int64)
            lib.or_result_iter(h, t, a.ctypes.data)
            res.iterations.append((int(a[0]), int(a[1]), _i128(a[2], a[3])))
        return res
    finally:
        lib.or_free(h)


def colour_classes(off, col, pass_index=0):
    """(classes, count): the capped greedy colouring of a graph that the
    colour-class mode uses in pass `pass_index` (see or_colour_classes)."""
    lib = _load()
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(off) - 1
    cls = np.empty(max(n, 1), np.int32)
    k = lib.or_colour_classes(n, off.ctypes.data, col.ctypes.data, int(pass_index), cls.ctypes.data)
    if k < 0:
        raise ValueError("oracle: bad graph")
    return cls[:n], int(k)


def modularity(off, col, w, memb):
    """(Q as float64, exact numerator N, M): Q = N / M^2 with N = M sum L_c - sum Sigma_c^2."""
    lib = _load()
    off, col, w = _arrs(off, col, w)
    memb = np.ascontiguousarray(memb, dtype=np.int32)
    n = len(off) - 1
    hi, lo, M, q = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64(), ctypes.c_double()
    rc = lib.or_modularity(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, memb.ctypes.data,
                           ctypes.byref(hi), ctypes.byref(lo), ctypes.byref(M), ctypes.byref(q))
    if rc != 0:
        raise ValueError("oracle.modularity: membership out of range")
    return q.value, _i128(hi.value, lo.value), M.value


def vertex_gains(off, col, w, memb, i):
    """{community: exact gain} for moving vertex i to each neighbouring community != memb[i]."""
    lib = _load()
    off, col, w = _arrs(off, col, w)
    memb = np.ascontiguousarray(memb, dtype=np.int32)
    n = len(off) - 1
    cap = n
    cs = np.empty(max(cap, 1), np.int32)
    hi = np.empty(max(cap, 1), np.int64)
    lo = np.empty(max(cap, 1), np.uint64)
    cnt = lib.or_vertex_gains(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, memb.ctypes.data, i,
                              cs.ctypes.data, hi.ctypes.data, lo.ctypes.data, cap)
    return {int(cs[t]): _i128(hi[t], lo[t]) for t in range(cnt)}


def aggregate(off, col, w, level, k):
    """Coarse CSR (off, col, w int64) over k communities, rows sorted by column."""
    lib = _load()
    off, col, w = _arrs(off, col, w)
    level = np.ascontiguousarray(level, dtype=np.int32)
    n = len(off) - 1
    cap = max(int(off[-1]), 1)
    oo = np.empty(k + 1, np.int64)
    oc = np.empty(cap, np.int32)
    ow = np.empty(cap, np.int64)
    nnz = ctypes.c_int64()
    rc = lib.or_aggregate(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, level.ctypes.data, k,
                          oo.ctypes.data, oc.ctypes.data, ow.ctypes.data, cap, ctypes.byref(nnz))
    if rc != 0:
        raise ValueError(f"oracle.aggregate failed ({rc})")
    return oo, oc[:nnz.value].copy(), ow[:nnz.value].copy()


def brute_best(off, col, w):
    """(best exact numerator, first best membership, partitions enumerated) over all set partitions."""
    lib = _load()
    off, col, w = _arrs(off, col, w)
    n = len(off) - 1
    memb = np.empty(max(n, 1), np.int32)
    hi, lo, cnt = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
    rc = lib.or_brute_best(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, memb.ctypes.data,
                           ctypes.byref(hi), ctypes.byref(lo), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError("oracle.brute_best: n must be in [1, 12]")
    return _i128(hi.value, lo.value), memb[:n].copy(), cnt.value


# ------------------------------------------------ multi-threaded baseline

class _MTOptions(ctypes.Structure):
    _fields_ = [("tolerance", ctypes.c_double), ("tolerance_decline", ctypes.c_double),
                ("pass_tolerance", ctypes.c_double), ("max_iterations", ctypes.c_int),
                ("max_passes", ctypes.c_int), ("threads", ctypes.c_int)]


@dataclass
class MTResult:
    top: np.ndarray
    M: int
    q_num: int
    Q: float
    passes: int
    iterations: int
    moves: int
    scanned: int     # CSR entries scanned by local moving (every vertex every iteration)
    threads: int


def _load_mt():
    global _mt_lib
    if _mt_lib is None:
        build()
        lib = ctypes.CDLL(_MT_LIB)
        lib.mt_louvain.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(_MTOptions), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.mt_louvain.restype = ctypes.c_int
        lib.mt_threads_available.restype = ctypes.c_int
        _mt_lib = lib
    return _mt_lib


def threads_available() -> int:
    """Threads the multi-threaded baseline can use (1 without OpenMP)."""
    return int(_load_mt().mt_threads_available())


def louvain_mt(off, col, w, threads=None, tolerance=0.01, tolerance_decline=10.0, pass_tolerance=0.0,
               max_iterations=20, max_passes=10) -> MTResult:
    """Multi-threaded CPU Louvain (louvain_mt.c): the paper's shared-memory
    asynchronous design with a hashtable per thread.  A CPU baseline for the
    benchmark, not the oracle; with one thread it is the oracle's sequential
    asynchronous run without pruning."""
    lib = _load_mt()
    off, col, w = _arrs(off, col, w)
    n = len(off) - 1
    t = threads_available() if threads is None else int(threads)
    opt = _MTOptions(tolerance, tolerance_decline, pass_tolerance, max_iterations, max_passes, t)
    top = np.empty(n, np.int32)
    out = np.zeros(8, np.int64)
    q = ctypes.c_double()
    used = lib.mt_louvain(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, ctypes.byref(opt), top.ctypes.data,
                          out.ctypes.data, ctypes.byref(q))
    if used < 0:
        raise ValueError("louvain_mt: invalid options")
    return MTResult(top=top, M=int(out[6]), q_num=_i128(out[4], out[5]), Q=q.value, passes=int(out[0]),
                    iterations=int(out[1]), moves=int(out[2]), scanned=int(out[3]), threads=int(used))
