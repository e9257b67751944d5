"""Seeded synthetic graph generators (symmetric CSR) shared by tests, bench and server.

The graphs stand in for the SuiteSparse graphs of the paper's Table 1 (Section
3.1.2), which are not available offline: R-MAT for the heavy-tailed web and
social graphs, a perturbed 2D grid for the road networks, and a planted-
partition SBM for graphs with known community structure.  The module holds
no community-detection arithmetic; it only draws graphs.

The C source (graphgen.c) is compiled by :func:`build` into ``libgraphgen.so``
beside it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so (gcc, no libm, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("off", ctypes.POINTER(ctypes.c_int64)), ("col", ctypes.POINTER(ctypes.c_int32)),
                ("w", ctypes.POINTER(ctypes.c_int32)), ("truth", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_CSR)
        u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.gg_sbm.argtypes = [u64, i64, i64, dbl, dbl, i32, i32, P]
        lib.gg_rmat.argtypes = [u64, ctypes.c_int, i64, dbl, dbl, dbl, dbl, i32, i32, P]
        lib.gg_grid_road.argtypes = [u64, i64, dbl, dbl, i32, i32, P]
        lib.gg_from_edges.argtypes = [i64, i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, u64, i32, i32, P]
        lib.gg_free.argtypes = [P]
        lib.gg_sbm_batch.argtypes = [i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, i32, i32, P, ctypes.c_void_p]
        lib.gg_sbm_batch.restype = ctypes.c_int
        lib.gg_uniform.argtypes = [u64, u64, u64]
        lib.gg_uniform.restype = dbl
        for f in (lib.gg_sbm, lib.gg_rmat, lib.gg_grid_road, lib.gg_from_edges):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class CSR:
    """Symmetric CSR graph: int64 offsets, int32 columns, int32 weights (> 0)."""
    n: int
    off: np.ndarray
    col: np.ndarray
    w: np.ndarray
    truth: Optional[np.ndarray] = None

    @property
    def nnz(self) -> int:
        return int(self.off[-1]) if self.n >= 0 and len(self.off) else 0

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)


def _take(c: _CSR, lib) -> CSR:
    n, nnz = int(c.n), int(c.nnz)
    off = np.ctypeslib.as_array(c.off, shape=(n + 1,)).copy() if n >= 0 else np.zeros(1, np.int64)
    col = np.ctypeslib.as_array(c.col, shape=(max(nnz, 1),))[:nnz].copy()
    w = np.ctypeslib.as_array(c.w, shape=(max(nnz, 1),))[:nnz].copy()
    truth = np.ctypeslib.as_array(c.truth, shape=(max(n, 1),))[:n].copy() if bool(c.truth) else None
    lib.gg_free(ctypes.byref(c))
    return CSR(n, off, col, w, truth)


def _check(rc: int, what: str):
    if rc == -2:
        raise ValueError(f"{what}: invalid arguments")
    if rc != 0:
        raise MemoryError(f"{what}: out of host memory")


def sbm(seed: int, n: int, k: int, p_in: float, p_out: float, wmin: int = 1, wmax: int = 1) -> CSR:
    """Planted-partition SBM: k near-equal blocks, edge probability p_in inside, p_out across."""
    lib = _load()
    c = _CSR()
    _check(lib.gg_sbm(seed, n, k, p_in, p_out, wmin, wmax, ctypes.byref(c)), "sbm")
    return _take(c, lib)


def rmat(seed: int, scale: int, edge_factor: float = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         wmin: int = 1, wmax: int = 1, n: int = 0) -> CSR:
    """R-MAT graph, self-loops removed, duplicates merged, symmetrised, ids permuted."""
    lib = _load()
    s = _CSR()
    _check(lib.gg_rmat(seed, scale, n, edge_factor, a, b, c, wmin, wmax, ctypes.byref(s)), "rmat")
    return _take(s, lib)


def grid_road(seed: int, side: int, drop: float = 0.1, shortcut_frac: float = 0.001, wmin: int = 1,
              wmax: int = 100) -> CSR:
    """side x side grid, `drop` of the grid edges removed, plus random long-range shortcuts."""
    lib = _load()
    s = _CSR()
    _check(lib.gg_grid_road(seed, side, drop, shortcut_frac, wmin, wmax, ctypes.byref(s)), "grid_road")
    return _take(s, lib)


def from_edges(n: int, edges: Sequence[Tuple[int, int]], keep_loops: bool = True, seed: int = 0, wmin: int = 1,
               wmax: int = 1) -> CSR:
    """Canonical symmetric CSR from an undirected edge list (weights hashed per pair)."""
    lib = _load()
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    u = np.ascontiguousarray(e[:, 0])
    v = np.ascontiguousarray(e[:, 1])
    s = _CSR()
    _check(lib.gg_from_edges(n, len(u), u.ctypes.data, v.ctypes.data, int(keep_loops), seed, wmin, wmax,
                             ctypes.byref(s)), "from_edges")
    return _take(s, lib)


def from_weighted_edges(n: int, edges: Sequence[Tuple[int, int, int]]) -> CSR:
    """Symmetric CSR from explicit (u, v, w) undirected edges; duplicate pairs have weights summed.

    Pure numpy, for small hand-made test graphs with chosen weights.
    """
    rows: List[Tuple[int, int, int]] = []
    for (u, v, w) in edges:
        rows.append((u, v, w))
        if u != v:
            rows.append((v, u, w))
    acc = {}
    for (u, v, w) in rows:
        acc[(u, v)] = acc.get((u, v), 0) + w
    keys = sorted(acc)
    off = np.zeros(n + 1, np.int64)
    for (u, _v) in keys:
        off[u + 1] += 1
    off = np.cumsum(off).astype(np.int64)
    col = np.array([k[1] for k in keys], np.int32)
    w = np.array([acc[k] for k in keys], np.int32)
    return CSR(n, off, col, w)


def uniform(seed: int, stream: int, i: int) -> float:
    """Counter-based U[0,1) draw i of a stream (same generator as the graphs)."""
    return float(_load().gg_uniform(seed, stream, i))


def batch_sbm_specs(seed: int, count: int, nmin: int = 256, nmax: int = 16384, kmin: int = 4, kmax: int = 64,
                    pin_lo: float = 0.05, pin_hi: float = 0.2, p_out: float = 1e-3):
    """Per-graph (seed, n, k, p_in, p_out) of a batch of SBM graphs: n log-uniform in
    [nmin, nmax], k uniform in {kmin..kmax} (capped at n), p_in uniform in [pin_lo, pin_hi]."""
    specs = []
    ln_lo, ln_hi = math.log(nmin), math.log(nmax)
    for g in range(count):
        un = uniform(seed, 20, g)
        n = int(round(math.exp(ln_lo + (ln_hi - ln_lo) * un)))
        n = max(nmin, min(nmax, n))
        k = kmin + int(uniform(seed, 21, g) * (kmax - kmin + 1))
        k = max(1, min(k, n))
        p_in = pin_lo + (pin_hi - pin_lo) * uniform(seed, 22, g)
        specs.append((seed * 1000003 + g, n, k, p_in, p_out))
    return specs


def sbm_batch(specs, wmin: int = 1, wmax: int = 1) -> Tuple[CSR, np.ndarray]:
    """Build many SBM graphs (specs from batch_sbm_specs) on all host cores and pack them into one
    block-diagonal CSR; returns it with the per-graph vertex offsets (int64, len(specs) + 1).
    The graphs are identical to sbm(*spec) one by one."""
    lib = _load()
    cnt = len(specs)
    seed = np.array([s[0] for s in specs], np.uint64)
    n = np.array([s[1] for s in specs], np.int64)
    k = np.array([s[2] for s in specs], np.int64)
    pin = np.array([s[3] for s in specs], np.float64)
    pout = np.array([s[4] for s in specs], np.float64)
    vo = np.zeros(cnt + 1, np.int64)
    c = _CSR()
    _check(lib.gg_sbm_batch(cnt, seed.ctypes.data, n.ctypes.data, k.ctypes.data, pin.ctypes.data, pout.ctypes.data,
                            wmin, wmax, ctypes.byref(c), vo.ctypes.data), "sbm_batch")
    return _take(c, lib), vo


def split(big: CSR, vo: np.ndarray) -> List[CSR]:
    """The graphs of a block-diagonal CSR, each with its own ids."""
    out = []
    for g in range(len(vo) - 1):
        v0, v1 = int(vo[g]), int(vo[g + 1])
        e0, e1 = int(big.off[v0]), int(big.off[v1])
        out.append(CSR(v1 - v0, big.off[v0:v1 + 1] - e0, big.col[e0:e1] - v0, big.w[e0:e1]))
    return out


def concat(graphs: Sequence[CSR]) -> Tuple[CSR, np.ndarray]:
    """Pack graphs into one block-diagonal CSR; returns it with per-graph vertex offsets (int64)."""
    vo = np.zeros(len(graphs) + 1, np.int64)
    for i, g in enumerate(graphs):
        vo[i + 1] = vo[i] + g.n
    total_n = int(vo[-1])
    total_nnz = sum(g.nnz for g in graphs)
    off = np.zeros(total_n + 1, np.int64)
    col = np.empty(total_nnz, np.int32)
    w = np.empty(total_nnz, np.int32)
    e0 = 0
    for i, g in enumerate(graphs):
        v0 = int(vo[i])
        off[v0:v0 + g.n + 1] = g.off + e0
        col[e0:e0 + g.nnz] = g.col + v0
        w[e0:e0 + g.nnz] = g.w
        e0 += g.nnz
    return CSR(total_n, off, col, w), vo
