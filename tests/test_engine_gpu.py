"""GPU parity of the CUDA engine against the oracle, through the C ABI.

Synchronous mode: bit-exact (top membership, exact modularity numerator,
every iteration's move count and gain sum S, every pass's level and coarse
CSR).  Asynchronous mode: final modularity no lower than the oracle's minus
0.01.  Inputs are the seeded synthetic graphs of the benchmark configurations
at sizes the oracle finishes in seconds, chosen so that every degree class of
the local-moving phase (thread, warp, block, hub) and of the aggregation
phase is used, plus edge cases.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from engine_util import assert_sync_parity, engine_run
from paper_2301_12390_gb300 import Louvain, LouvainError

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_runs.json")


@pytest.fixture(scope="module", autouse=True)
def _engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def graphs():
    return {
        "sbm600": gg.sbm(11, 600, 12, 0.15, 0.01, wmin=1, wmax=9),
        "sbm8192": gg.sbm(0x5EED, 8192, 64, 0.1, 0.0005),          # the small benchmark configuration
        "rmat14": gg.rmat(0x5EED + 1, 14, 16, wmin=1, wmax=8),
        "rmat16": gg.rmat(0x5EED + 1, 16, 16, wmin=1, wmax=8),     # hubs of degree > 4096
        "road128": gg.grid_road(0x5EED + 2, 128),
    }


G = graphs()


# ------------------------------------------------------------- hand runs

def test_hand_worked_runs_on_gpu():
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        if case["options"] is None:
            continue
        g = gg.from_weighted_edges(case["n"], [tuple(e) for e in case["edges"]])
        o = dict(case["options"])
        mode = 0 if o.pop("mode") == "sync" else 1
        ex = case["expect"]
        for prune in ([o.pop("prune")] if "prune" in o else (0, 1)):
            got = engine_run(g, mode=mode, prune=prune, **o)
            if mode == 0:
                assert list(got["top"]) == ex["top"], case["name"]
                assert got["exact"] == (ex["q_num"], ex["M"]), case["name"]
                assert [list(t) for t in got["iters"]] == ex["iterations"], case["name"]
            else:
                assert got["q"] >= ex["Q"] - 0.01, case["name"]


# --------------------------------------------------------- sync parity

@pytest.mark.parametrize("name", list(G))
@pytest.mark.parametrize("prune", [0, 1])
def test_sync_parity(name, prune):
    assert_sync_parity(G[name], prune=prune)


@pytest.mark.parametrize("name", ["sbm8192", "rmat16", "road128"])
@pytest.mark.parametrize("subrounds", [4, 16])
def test_sync_parity_subrounds(name, subrounds):
    assert_sync_parity(G[name], prune=1, subrounds=subrounds)


@pytest.mark.parametrize("name", list(G))
@pytest.mark.parametrize("prune", [0, 1])
def test_sync_parity_recomputed_stop_rule(name, prune):
    """stop_rule 1: an iteration's change is the exact change of the Q
    numerator over it (recomputed on the device after every iteration);
    bit-exact with the oracle's same reading."""
    assert_sync_parity(G[name], prune=prune, stop_rule=1)


@pytest.mark.parametrize("name", ["sbm600", "rmat16", "road128"])
def test_async_quality_recomputed_stop_rule(name):
    g = G[name]
    got = engine_run(g, mode=1, prune=1, stop_rule=1)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
    _, num, M = oracle.modularity(g.off, g.col, g.w, got["top"])
    assert got["exact"] == (num, M)


@pytest.mark.parametrize("name", ["road128", "sbm8192"])
@pytest.mark.parametrize("graphs", [0, 1])
def test_sync_parity_with_and_without_cuda_graphs(name, graphs):
    """From the third iteration of a pass the engine replays a captured CUDA
    graph; the result must not depend on it."""
    assert_sync_parity(G[name], prune=1, subrounds=4, cuda_graphs=graphs)


@pytest.mark.parametrize("name", ["sbm600", "rmat14"])
def test_sync_parity_plain_jacobi(name):
    assert_sync_parity(G[name], singleton_guard=0)


def test_sync_parity_wide_arithmetic():
    """Weights near the int32 maximum: M >= 2^31, so gains need 128 bits and
    coarse weights 64 bits."""
    base = gg.sbm(5, 700, 10, 0.12, 0.01)
    # weights from the unordered pair keep the CSR symmetric
    rows = np.repeat(np.arange(base.n), np.diff(base.off))
    lo, hi = np.minimum(rows, base.col), np.maximum(rows, base.col)
    w = (2**31 - 1 - ((lo.astype(np.int64) * 131 + hi) % 1000)).astype(np.int32)
    g = gg.CSR(base.n, base.off, base.col, w)
    got, ref = assert_sync_parity(g, prune=1)
    assert ref.M >= 2**31


def test_sync_parity_wide_arithmetic_large_communities():
    """Wide sums with communities above 4,096 member entries: the aggregation
    takes its global-table path with 64-bit shared sums (three blocks of
    1,000 vertices, about 22,000 entries each)."""
    base = gg.sbm(11, 3000, 3, 0.02, 0.0007)
    rows = np.repeat(np.arange(base.n), np.diff(base.off))
    lo, hi = np.minimum(rows, base.col), np.maximum(rows, base.col)
    w = (2**31 - 1 - ((lo.astype(np.int64) * 131 + hi) % 1000)).astype(np.int32)
    g = gg.CSR(base.n, base.off, base.col, w)
    got, ref = assert_sync_parity(g, prune=1)
    assert ref.M >= 2**31
    dsum = np.bincount(ref.passes[0].level, weights=np.diff(g.off))   # member entries per pass-0 community
    assert dsum.max() > 4096


@pytest.mark.parametrize("opt", [dict(prune=1), dict(prune=0, subrounds=4), dict(prune=1, singleton_guard=0)])
def test_sync_parity_graph_of_block_vertices(opt):
    """A graph whose every vertex has degree 129-1,024 (checked below), so
    that all of pass 0 runs in the block-per-vertex kernel with its
    2,048-slot table: bit-exact with the oracle under pruning, four classes
    and no singleton guard."""
    g = gg.sbm(21, 3000, 4, 0.3, 0.01, wmin=1, wmax=9)
    deg = np.diff(g.off)
    assert deg.min() > 128 and deg.max() <= 1024
    assert_sync_parity(g, **opt)


def test_async_quality_graph_of_block_vertices():
    g = gg.sbm(21, 3000, 4, 0.3, 0.01, wmin=1, wmax=9)
    got = engine_run(g, mode=1, prune=1)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
    _, num, M = oracle.modularity(g.off, g.col, g.w, got["top"])
    assert got["exact"] == (num, M)


def test_sync_parity_max_iterations_and_passes():
    g = G["sbm8192"]
    assert_sync_parity(g, max_iterations=1)
    assert_sync_parity(g, max_passes=1)
    assert_sync_parity(g, max_passes=2, tolerance=0.0)


# ------------------------------------------------- vertex mapping, autotuner

@pytest.mark.parametrize("name", ["rmat16", "sbm8192"])
@pytest.mark.parametrize("thresholds", [[4, 16, 64, 256, 2048], [8, 32, 128, 1024, 4096], [1, 2, 3, 4, 5],
                                        [1, 32, 128, 1024, 4096]])
def test_sync_parity_under_any_mapping(name, thresholds):
    """Which kernel handles a vertex never changes the result: bit-exact sync
    parity with the oracle under non-default degree thresholds (the third
    sends almost every vertex to the hub path, the fourth every vertex of
    degree 2-32 to the lane-per-vertex sorting kernel)."""
    g = G[name]
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.set_mapping(thresholds)
        assert lv.mapping() == thresholds
        lv.load_csr(g.off, g.col, g.w)
        lv.run()
        top, exact = lv.membership(), lv.modularity_exact()
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.SYNC, prune=1)
    assert np.array_equal(top, ref.top)
    assert exact == (ref.q_num, ref.M)


def test_mapping_rejects_bad_thresholds():
    with Louvain(device=0) as lv:
        for bad in ([8, 32, 128, 1024, 5000], [8, 8, 128, 1024, 4096], [0, 32, 128, 1024, 4096], [9, 32, 128, 1024, 4096]):
            with pytest.raises(LouvainError):
                lv.set_mapping(bad)
        lv.set_mapping(None)
        assert lv.mapping() == [8, 32, 128, 1024, 4096]


def test_autotune_keeps_results():
    """The autotuner picks a valid mapping; runs after it still match the oracle (sync) bit for bit."""
    g = G["rmat16"]
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        th, ms = lv.autotune()
        assert ms > 0 and len(th) == 5 and all(a < b for a, b in zip(th, th[1:]))
        assert all(1 <= t <= cap for t, cap in zip(th, [8, 32, 128, 1024, 4096]))
        lv.run()
        top, exact = lv.membership(), lv.modularity_exact()
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.SYNC, prune=1)
    assert np.array_equal(top, ref.top)
    assert exact == (ref.q_num, ref.M)


# ------------------------------------------ incremental re-runs (warm start)

@pytest.mark.parametrize("name", ["sbm600", "rmat16", "road128"])
def test_sync_run_from_matches_oracle(name):
    """Pass 0 from a given membership: bit-exact sync parity with the oracle
    started from the same membership (a random one, the identity, and the
    graph's own previous result)."""
    g = G[name]
    rng = np.random.default_rng(5)
    inits = [rng.integers(0, g.n, g.n).astype(np.int32), np.arange(g.n, dtype=np.int32)]
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        lv.run()
        inits.append(lv.membership())
        for init in inits:
            lv.run_from(init)
            top, exact = lv.membership(), lv.modularity_exact()
            its = lv.iterations()
            ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.SYNC, prune=1, initial=init)
            assert np.array_equal(top, ref.top)
            assert exact == (ref.q_num, ref.M)
            assert its == list(ref.iterations)


def test_async_run_from_keeps_quality_and_rejects_bad_ids():
    g = G["sbm8192"]
    with Louvain(device=0, mode=1, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        lv.run()
        prev = lv.membership()
        q_prev = lv.modularity()
        lv.run_from(prev)
        assert lv.modularity() >= q_prev - 0.01
        bad = prev.copy()
        bad[3] = g.n
        with pytest.raises(LouvainError):
            lv.run_from(bad)
        lv.run()   # the graph stays loaded after a rejected membership
        assert lv.modularity() > 0.5


def test_batch_run_from_equals_each_graph_alone():
    """Several graphs: a run from per-graph memberships (global ids) gives,
    in sync mode, each graph's result from its own membership alone."""
    gs = [G["sbm600"], G["road128"], gg.sbm(3, 300, 6, 0.2, 0.02)]
    big, vo = gg.concat(gs)
    rng = np.random.default_rng(9)
    init = np.concatenate([vo[k] + rng.integers(0, g.n, g.n) for k, g in enumerate(gs)]).astype(np.int32)
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.load_batch(vo, big.off, big.col, big.w)
        lv.run_from(init)
        memb = lv.membership()
        q, nums, Ms = lv.batch_modularity()
    for k, g in enumerate(gs):
        ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.SYNC, prune=1,
                             initial=init[vo[k]:vo[k + 1]] - vo[k])
        assert np.array_equal(memb[vo[k]:vo[k + 1]], ref.top), k
        assert nums[k] == ref.q_num, k


# ------------------------------------------------ partition, then merge

def oracle_partitioned(g, parts, **kw):
    """The same steps with the oracle: each part's induced subgraph alone,
    then the whole graph from their communities (global ids)."""
    n = g.n
    vo = [(p * n + parts - 1) // parts for p in range(parts + 1)]
    init = np.empty(n, np.int32)
    for p in range(parts):
        a, b = vo[p], vo[p + 1]
        edges = []
        for u in range(a, b):
            for x in range(int(g.off[u]), int(g.off[u + 1])):
                v = int(g.col[x])
                if a <= v < b and u <= v:
                    edges.append((u - a, v - a, int(g.w[x])))
        sub = gg.from_weighted_edges(b - a, edges)
        r = oracle.louvain(sub.off, sub.col, sub.w, **kw)
        init[a:b] = a + r.top
    return oracle.louvain(g.off, g.col, g.w, initial=init, **kw)


@pytest.mark.parametrize("name", ["sbm600", "rmat14", "road128"])
@pytest.mark.parametrize("parts", [2, 7])
def test_sync_partitioned_matches_oracle(name, parts):
    g = G[name]
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        ms = lv.run_partitioned(parts)
        top, exact = lv.membership(), lv.modularity_exact()
    ref = oracle_partitioned(g, parts, mode=oracle.SYNC, prune=1)
    assert ms > 0
    assert np.array_equal(top, ref.top)
    assert exact == (ref.q_num, ref.M)


@pytest.mark.parametrize("name", ["road128", "rmat14"])
def test_async_partitioned_quality(name):
    """Asynchronous partition-then-merge ends within 0.01 of the oracle
    running the same method (the partition by id ranges is only as good as
    the ids' locality: on the grid, whose ids are spatial, it matches or beats
    a plain run; on R-MAT, whose ids are random, most entries are cut)."""
    g = G[name]
    ref = oracle_partitioned(g, 8, mode=oracle.ASYNC, prune=1)
    plain = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    with Louvain(device=0, mode=1, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        lv.run_partitioned(8)
        assert lv.modularity() >= ref.Q - 0.01, (lv.modularity(), ref.Q)
        lv.run_partitioned(1)   # one part: a plain run
        assert lv.modularity() >= plain.Q - 0.01


# ------------------------------------------------------- async quality

@pytest.mark.parametrize("name", ["sbm600", "rmat16", "road128"])
@pytest.mark.parametrize("reclass", [0, 1, 2, 3])
def test_async_class_modes(name, reclass):
    """Every way of drawing the asynchronous classes (id mod P, hashed per
    iteration, hashed per pass, automatic) keeps Q within 0.01 of the oracle."""
    g = G[name]
    got = engine_run(g, mode=1, prune=1, reclass=reclass)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
    _, num, M = oracle.modularity(g.off, g.col, g.w, got["top"])
    assert got["exact"] == (num, M)


@pytest.mark.parametrize("reclass", [1, 2])
def test_sync_ignores_class_mode(reclass):
    """Synchronous classes are always id mod P (the oracle's), whatever reclass says."""
    assert_sync_parity(G["rmat14"], prune=1, subrounds=4, reclass=reclass)


@pytest.mark.parametrize("name", list(G))
@pytest.mark.parametrize("prune,subrounds", [(0, 0), (1, 0), (1, 32)])
def test_async_quality(name, prune, subrounds):
    g = G[name]
    got = engine_run(g, mode=1, prune=prune, subrounds=subrounds)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=prune)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
    # the reported modularity is that of the reported membership, exactly
    _, num, M = oracle.modularity(g.off, g.col, g.w, got["top"])
    assert got["exact"] == (num, M)


@pytest.mark.parametrize("name", ["sbm600", "rmat16", "road128", "sbm8192"])
@pytest.mark.parametrize("prune", [0, 1])
def test_sync_parity_colour_classes(name, prune):
    """Colour classes (a greedy colouring of every pass graph) in synchronous
    mode: bit-exact with the oracle's colour-class mode at every pass."""
    assert_sync_parity(G[name], prune=prune, colour_classes=1)


@pytest.mark.parametrize("name", ["rmat16", "road128"])
def test_async_quality_colour_classes(name):
    g = G[name]
    got = engine_run(g, mode=1, prune=1, colour_classes=1)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
    _, num, M = oracle.modularity(g.off, g.col, g.w, got["top"])
    assert got["exact"] == (num, M)


# ---------------------------------------------------------- edge cases

@pytest.mark.parametrize("mode", [0, 1])
def test_edge_cases(mode):
    cases = [
        gg.from_weighted_edges(1, []),
        gg.from_weighted_edges(5, []),
        gg.from_weighted_edges(3, [(1, 1, 4)]),
        gg.from_weighted_edges(6, [(0, 1, 1), (2, 2, 3), (4, 5, 2)]),
        gg.from_weighted_edges(4, [(0, 1, 5), (1, 2, 5), (2, 3, 5), (3, 0, 5), (0, 0, 2)]),
    ]
    for g in cases:
        got = engine_run(g, mode=mode)
        ref = oracle.louvain(g.off, g.col, g.w, mode=mode)
        if mode == 0:
            assert np.array_equal(got["top"], ref.top)
            assert got["exact"] == (ref.q_num, ref.M)
        else:
            assert got["q"] >= ref.Q - 0.01


def test_empty_graph():
    from paper_2301_12390_gb300 import Louvain
    with Louvain(device=0) as lv:
        lv.load_csr(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
        lv.run()
        assert lv.modularity() == 0.0 and len(lv.membership()) == 0


# ------------------------------------------------------ modularity API

def test_modularity_of_arbitrary_memberships():
    from paper_2301_12390_gb300 import Louvain
    rng = np.random.default_rng(3)
    for g in (G["sbm600"], G["rmat14"]):
        with Louvain(device=0) as lv:
            lv.load_csr(g.off, g.col, g.w)
            for k in (1, 7, g.n):
                memb = rng.integers(0, k, g.n).astype(np.int32)
                q, num, M = lv.modularity_of(memb)
                rq, rnum, rM = oracle.modularity(g.off, g.col, g.w, memb)
                assert (num, M) == (rnum, rM) and q == rq


# ---------------------------------------------------------- input errors

def test_input_errors():
    from paper_2301_12390_gb300 import Louvain, LouvainError
    g = G["sbm600"]
    with Louvain(device=0) as lv:
        with pytest.raises(LouvainError) as e:
            lv.run()
        assert e.value.code == -7                                   # STATE: run before load
        bad = g.w.copy()
        bad[0] += 1                                                 # (u,v) and (v,u) weights differ
        with pytest.raises(LouvainError) as e:
            lv.load_csr(g.off, g.col, bad)
        assert e.value.code == -2
        bad = g.w.copy()
        bad[3] = 0
        with pytest.raises(LouvainError) as e:
            lv.load_csr(g.off, g.col, bad)
        assert e.value.code == -3
        badc = g.col.copy()
        badc[5] = g.n
        with pytest.raises(LouvainError) as e:
            lv.load_csr(g.off, badc, g.w)
        assert e.value.code == -3
        bado = g.off.copy()
        bado[10], bado[11] = bado[11], bado[10] + 5
        with pytest.raises(LouvainError) as e:
            lv.load_csr(bado, g.col, g.w)
        assert e.value.code == -3
        lv.load_csr(g.off, g.col, g.w)                              # still usable afterwards
        lv.run()
        assert lv.modularity() > 0.3


# ------------------------------------------------------- device inputs

def test_device_pointers_match_host():
    import torch
    from paper_2301_12390_gb300 import Louvain
    g = G["rmat14"]
    host = engine_run(g, mode=0)
    with Louvain(device=0, mode=0) as lv:
        lv.load_csr(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.col).cuda(), torch.from_numpy(g.w).cuda())
        lv.run()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        lv.membership(out)
        assert np.array_equal(out.cpu().numpy(), host["top"])


def test_local_moving_byte_model():
    """lm_bytes follows the algorithmic model: 12 per scanned entry (32-bit
    weights), 32 per visited vertex, 8 per candidate community, 16 per move;
    every visited vertex with a neighbour outside its community has at least
    one candidate, and there are never more candidates than scanned entries."""
    g = G["rmat14"]
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.load_csr(g.off, g.col, g.w)
        lv.run()
        st = lv.stats()
    assert 0 < st.lm_candidates <= st.lm_edges
    assert st.lm_bytes == 12 * st.lm_edges + 32 * st.lm_vertices + 8 * st.lm_candidates + 16 * st.moves
