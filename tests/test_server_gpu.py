"""The request server: requests arriving while others run are admitted as
slots and memory free up, batched with whatever waits, and each result equals
the graph's result alone (synchronous: bit for bit; asynchronous: within 0.01
of the oracle)."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from engine_util import async_within_tolerance, assert_async_quality_over_graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def request_graphs():
    out = []
    for i in range(40):
        if i % 2 == 0:
            n = 200 + 37 * i
            out.append(gg.sbm(1000 + i, n, 2 + i % 9, 0.15, 0.01, wmin=1, wmax=8))
        else:
            out.append(gg.rmat(2000 + i, 9 + i % 5, 8 + i % 9, wmin=1, wmax=8))
    return out


GRAPHS = request_graphs()


def alone(g, mode):
    from paper_2301_12390_gb300 import Louvain
    with Louvain(device=0, mode=mode, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        lv.run()
        return lv.membership(), lv.modularity_exact()


def serve(graphs, mode, gap_s=0.0, **cfg):
    from paper_2301_12390_gb300 import Server
    results = {}
    with Server(device=0, mode=mode, prune=1, **cfg) as srv:
        for i, g in enumerate(graphs):
            srv.submit(i, g.off, g.col, g.w)
            if gap_s:
                time.sleep(gap_s)
            for r in srv.poll():
                results[r["id"]] = r
        while len(results) < len(graphs):
            for r in srv.poll(wait_ms=200):
                results[r["id"]] = r
        membs = {i: srv.membership(i) for i in results if results[i]["status"] == 0}
        stats = srv.stats()
    return results, membs, stats


@pytest.mark.parametrize("cfg", [dict(slots=2), dict(slots=3, batch_max_entries=50_000),
                                 dict(slots=1, batch_max_entries=0), dict(slots=4, borrow_inputs=True)])
def test_sync_results_equal_alone(cfg):
    results, membs, stats = serve(GRAPHS, mode=0, gap_s=0.002, **cfg)
    assert stats["finished"] == len(GRAPHS)
    for i, g in enumerate(GRAPHS):
        m, (num, M) = alone(g, 0)
        assert results[i]["status"] == 0
        assert np.array_equal(membs[i], m), i
        assert (results[i]["num"], results[i]["M"]) == (num, M), i
    if cfg.get("batch_max_entries", 1) != 0:
        assert stats["runs"] <= len(GRAPHS)


def test_async_results_within_tolerance():
    results, membs, stats = serve(GRAPHS, mode=1)
    assert_async_quality_over_graphs(
        [(async_within_tolerance(g.off, g.col, g.w, results[i]["q"]), results[i]["q"]) for i, g in enumerate(GRAPHS)])


def test_admission_by_memory_budget():
    from paper_2301_12390_gb300 import arena_bytes
    big = max(arena_bytes(g.n, g.nnz) for g in GRAPHS)
    # room for about one graph at a time: slots must wait for each other's memory
    results, membs, stats = serve(GRAPHS[:12], mode=0, slots=3, hbm_budget_bytes=int(1.5 * big))
    assert all(results[i]["status"] == 0 for i in range(12))
    assert stats["peak_reserved_bytes"] <= int(1.5 * big)
    for i, g in enumerate(GRAPHS[:12]):
        m, _ = alone(g, 0)
        assert np.array_equal(membs[i], m)
    # a request larger than the whole budget is answered with OOM, the others still run
    tiny = arena_bytes(300, 3000)
    results, membs, stats = serve([GRAPHS[0], GRAPHS[1]], mode=0, slots=1,
                                  hbm_budget_bytes=max(arena_bytes(GRAPHS[0].n, GRAPHS[0].nnz), tiny))
    assert results[0]["status"] == 0
    assert results[1]["status"] == -4 or arena_bytes(GRAPHS[1].n, GRAPHS[1].nnz) <= arena_bytes(GRAPHS[0].n,
                                                                                                GRAPHS[0].nnz)
