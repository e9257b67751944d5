"""The multi-threaded CPU baseline (oracle/louvain_mt.c, the paper's OpenMP
design: asynchronous, a hashtable per thread, Section 3.2).  It is a
benchmark baseline, not the oracle: these CPU tests pin it to the oracle.
With one thread it is the sequential asynchronous method, so it must equal
the oracle's asynchronous run (pruning off) exactly; with several threads its
order is the scheduler's, so its modularity must be the exact modularity of
its membership and stay near the oracle's."""
import random

import numpy as np
import pytest

import graphgen as gg
import oracle


def _graphs():
    rng = random.Random(31)
    gs = [gg.sbm(41, 1200, 12, 0.12, 0.01, wmin=1, wmax=6), gg.rmat(42, 12, 10, wmin=1, wmax=8),
          gg.grid_road(43, 40, 0.1, 0.01, wmin=1, wmax=9)]
    for _ in range(8):
        n = rng.randint(3, 12)
        edges = [(u, v, rng.randint(1, 5)) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.4]
        if rng.random() < 0.5:
            edges.append((0, 0, 2))
        gs.append(gg.from_weighted_edges(n, edges))
    return gs


@pytest.mark.parametrize("tol", [0.01, 1e-6])
def test_one_thread_equals_the_oracle_sequential_run(tol):
    for g in _graphs():
        a = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=0, tolerance=tol)
        b = oracle.louvain_mt(g.off, g.col, g.w, threads=1, tolerance=tol)
        assert np.array_equal(a.top, b.top)
        assert (a.q_num, a.M) == (b.q_num, b.M) and a.Q == b.Q
        assert b.passes == len(a.passes) and b.iterations == len(a.iterations)


def test_threads_keep_exact_modularity_and_quality():
    for g in _graphs()[:3]:
        ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=0)
        r = oracle.louvain_mt(g.off, g.col, g.w, threads=max(2, oracle.threads_available()))
        _, num, M = oracle.modularity(g.off, g.col, g.w, r.top)
        assert (num, M) == (r.q_num, r.M)
        assert r.Q >= ref.Q - 0.02, (r.Q, ref.Q)
