"""Several graphs in one run (louvain_load_batch) give, per graph, exactly
what each graph gives alone: synchronous mode bit-exact against the plain
engine run of the graph and against the oracle; asynchronous mode within 0.01
of the oracle per graph."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from engine_util import async_within_tolerance, assert_async_quality_over_graphs
from paper_2301_12390_gb300 import Louvain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def batch_graphs():
    gs = []
    for (seed, n, k, p_in, p_out) in gg.batch_sbm_specs(0x5EED, 24, nmin=64, nmax=3000, kmin=2, kmax=20,
                                                       pin_lo=0.05, pin_hi=0.25, p_out=0.01):
        gs.append(gg.sbm(seed, n, k, p_in, p_out, wmin=1, wmax=5))
    gs.insert(3, gg.from_weighted_edges(5, []))                      # no edges
    gs.insert(7, gg.from_weighted_edges(1, [(0, 0, 3)]))             # one vertex, a self-loop
    gs.insert(11, gg.rmat(77, 13, 16, wmin=1, wmax=8))                # heavy-tailed, hubs
    gs.insert(15, gg.grid_road(78, 40))                               # low degree, many passes
    return gs


GS = batch_graphs()


def run_batch(gs, **opt):
    big, vo = gg.concat(gs)
    with Louvain(device=0, **opt) as lv:
        lv.load_batch(vo, big.off, big.col, big.w)
        lv.run()
        memb = lv.membership()
        q, nums, Ms = lv.batch_modularity()
        iters = [lv.batch_iterations(g) for g in range(len(gs))]
    return [memb[vo[g]:vo[g + 1]] for g in range(len(gs))], q, nums, Ms, iters


def run_alone(g, **opt):
    with Louvain(device=0, **opt) as lv:
        lv.load_csr(g.off, g.col, g.w)
        lv.run()
        return lv.membership(), lv.modularity(), lv.modularity_exact(), lv.iterations()


@pytest.mark.parametrize("prune,subrounds", [(0, 1), (1, 1), (1, 4)])
def test_sync_batch_equals_each_graph_alone(prune, subrounds):
    membs, q, nums, Ms, iters = run_batch(GS, mode=0, prune=prune, subrounds=subrounds)
    for g, graph in enumerate(GS):
        m1, q1, (num1, M1), it1 = run_alone(graph, mode=0, prune=prune, subrounds=subrounds)
        assert np.array_equal(membs[g], m1), g
        assert (nums[g], Ms[g]) == (num1, M1) and q[g] == q1, g
        assert iters[g] == it1, g
        ref = oracle.louvain(graph.off, graph.col, graph.w, mode=oracle.SYNC, prune=prune, subrounds=subrounds)
        assert np.array_equal(membs[g], ref.top) and nums[g] == ref.q_num, g


def test_sync_batch_with_colour_classes_equals_each_graph_alone():
    """Colour classes are drawn from local ids, so a graph gets the same
    classes, and the same synchronous result, alone and in a batch."""
    membs, q, nums, Ms, iters = run_batch(GS, mode=0, prune=1, colour_classes=1)
    for g, graph in enumerate(GS):
        m1, q1, (num1, M1), it1 = run_alone(graph, mode=0, prune=1, colour_classes=1)
        assert np.array_equal(membs[g], m1), g
        assert (nums[g], Ms[g]) == (num1, M1) and iters[g] == it1, g
        ref = oracle.louvain(graph.off, graph.col, graph.w, mode=oracle.SYNC, prune=1, colour_classes=1)
        assert np.array_equal(membs[g], ref.top) and nums[g] == ref.q_num, g


def test_sync_batch_with_recomputed_stop_rule_equals_each_graph_alone():
    """stop_rule 1 keeps each graph's own iteration stop in a batch: every
    graph's recomputed Q change is its own, so its result equals its result
    alone and the oracle's."""
    membs, q, nums, Ms, iters = run_batch(GS, mode=0, prune=1, stop_rule=1)
    for g, graph in enumerate(GS):
        m1, q1, (num1, M1), it1 = run_alone(graph, mode=0, prune=1, stop_rule=1)
        assert np.array_equal(membs[g], m1), g
        assert (nums[g], Ms[g]) == (num1, M1) and iters[g] == it1, g
        ref = oracle.louvain(graph.off, graph.col, graph.w, mode=oracle.SYNC, prune=1, stop_rule=1)
        assert np.array_equal(membs[g], ref.top) and nums[g] == ref.q_num, g


def test_async_batch_quality_per_graph():
    membs, q, nums, Ms, iters = run_batch(GS, mode=1, prune=1)
    assert_async_quality_over_graphs(
        [(async_within_tolerance(graph.off, graph.col, graph.w, q[g]), q[g]) for g, graph in enumerate(GS)])
    for g, graph in enumerate(GS):
        _, num, M = oracle.modularity(graph.off, graph.col, graph.w, membs[g])
        assert (num, M) == (nums[g], Ms[g]), g


def test_async_batch_of_large_graphs_quality_per_graph():
    """A batch holding graphs of every class-schedule category: a large sparse
    road grid (fewer than 8 entries per vertex), a large dense R-MAT and small
    SBMs; each graph keeps its own schedule and ends within 0.01 of the oracle."""
    gs = [gg.sbm(5, 900, 6, 0.2, 0.01, wmin=1, wmax=5),
          gg.grid_road(79, 320, 0.1, 0.001, wmin=1, wmax=100),   # 102,400 vertices, ~3.6 entries each
          gg.rmat(80, 17, 8, wmin=1, wmax=8),                     # 131,072 vertices, hubs
          gg.sbm(6, 2500, 12, 0.1, 0.005, wmin=1, wmax=5)]
    membs, q, nums, Ms, iters = run_batch(gs, mode=1, prune=1)
    for g, graph in enumerate(gs):
        ok, q_id, ref = async_within_tolerance(graph.off, graph.col, graph.w, q[g])
        assert ok, (g, q[g], q_id, ref)
        _, num, M = oracle.modularity(graph.off, graph.col, graph.w, membs[g])
        assert (num, M) == (nums[g], Ms[g]), g


def test_batch_rejects_entries_between_graphs():
    from paper_2301_12390_gb300 import LouvainError
    a, b = gg.sbm(1, 50, 2, 0.3, 0.05), gg.sbm(2, 60, 2, 0.3, 0.05)
    big, vo = gg.concat([a, b])
    with Louvain(device=0) as lv:
        with pytest.raises(LouvainError) as e:
            lv.load_batch(np.array([0, 40, big.n]), big.off, big.col, big.w)   # cuts graph a in two
        assert e.value.code == -3
        lv.load_batch(vo, big.off, big.col, big.w)
        lv.run()
        assert lv.num_graphs() == 2


def test_load_parts_equals_load_batch():
    """Graphs loaded from separate host CSRs (copied side by side on the
    device) run exactly as their block-diagonal concatenation."""
    membs, q, nums, Ms, iters = run_batch(GS, mode=0, prune=1)
    with Louvain(device=0, mode=0, prune=1) as lv:
        lv.load_parts([(g.off, g.col, g.w) for g in GS])
        lv.run()
        memb = lv.membership()
        q2, nums2, Ms2 = lv.batch_modularity()
    big, vo = gg.concat(GS)
    for g in range(len(GS)):
        assert np.array_equal(memb[vo[g]:vo[g + 1]], membs[g]), g
    assert list(nums2) == list(nums) and list(Ms2) == list(Ms)
