"""Pins of the oracle against facts fixed outside it (no GPU).

Each test ties one part of the oracle to something other than its own code:
an independent formula (pairwise modularity in exact fractions), a library
(networkx), brute force over all partitions, closed forms, invariants, and
runs worked by hand (tests/golden/hand_runs.json).  Together they are chosen
so that a dropped term, a wrong sign, a swapped index or a wrong tie rule in
the oracle fails at least one of them.
"""
import itertools
import json
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_runs.json")


# ---------------------------------------------------------------- helpers

def dense(g):
    """Dense adjacency (CSR entry values; a self-loop appears once on the diagonal)."""
    A = [[0] * g.n for _ in range(g.n)]
    for u in range(g.n):
        for e in range(int(g.off[u]), int(g.off[u + 1])):
            A[u][int(g.col[e])] += int(g.w[e])
    return A


def q_pairwise(A, memb):
    """Newman-Girvan in its pairwise form, exact: (1/M) sum_ij [A_ij - K_i K_j / M] delta(c_i, c_j)."""
    n = len(A)
    K = [sum(r) for r in A]
    M = sum(K)
    if M == 0:
        return Fraction(0)
    tot = Fraction(0)
    for i in range(n):
        for j in range(n):
            if memb[i] == memb[j]:
                tot += Fraction(A[i][j]) - Fraction(K[i] * K[j], M)
    return tot / M


def random_graph(rng, n, p, wmax=5, loops=True):
    edges = []
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                edges.append((u, v, rng.randint(1, wmax)))
        if loops and rng.random() < 0.2:
            edges.append((u, u, rng.randint(1, wmax)))
    return gg.from_weighted_edges(n, edges)


def bell(n):
    row = [1]
    for _ in range(n - 1):
        nxt = [row[-1]]
        for x in row:
            nxt.append(nxt[-1] + x)
        row = nxt
    return row[-1]


def cliques(k, s, ring=False):
    edges = []
    for c in range(k):
        base = c * s
        for a in range(s):
            for b in range(a + 1, s):
                edges.append((base + a, base + b, 1))
        if ring and k > 1:
            edges.append((base + s - 1, ((c + 1) % k) * s, 1))
    return gg.from_weighted_edges(k * s, edges)


def run(g, **kw):
    return oracle.louvain(g.off, g.col, g.w, **kw)


# ----------------------------------------------------------- modularity (a9)

def test_modularity_matches_pairwise_form_exactly():
    rng = random.Random(1)
    for _ in range(40):
        n = rng.randint(1, 9)
        g = random_graph(rng, n, 0.5)
        A = dense(g)
        memb = [rng.randrange(n) for _ in range(n)]
        q, num, M = oracle.modularity(g.off, g.col, g.w, memb)
        exact = q_pairwise(A, memb)
        if M:
            assert Fraction(num, M * M) == exact
        assert M == sum(map(sum, A))


def test_modularity_matches_networkx_without_self_loops():
    nx = pytest.importorskip("networkx")
    rng = random.Random(2)
    for _ in range(20):
        n = rng.randint(2, 30)
        g = random_graph(rng, n, 0.3, loops=False)
        if g.nnz == 0:
            continue
        G = nx.Graph()
        G.add_nodes_from(range(n))
        for u in range(n):
            for e in range(int(g.off[u]), int(g.off[u + 1])):
                v = int(g.col[e])
                if u < v:
                    G.add_edge(u, v, weight=int(g.w[e]))
        memb = [rng.randrange(min(4, n)) for _ in range(n)]
        comms = [set(i for i in range(n) if memb[i] == c) for c in set(memb)]
        q, _, _ = oracle.modularity(g.off, g.col, g.w, memb)
        assert abs(q - nx.community.modularity(G, comms, weight="weight")) < 1e-12


def test_modularity_closed_form_disjoint_cliques():
    for k, s in [(2, 3), (4, 5), (7, 4), (16, 6)]:
        g = cliques(k, s)
        memb = np.repeat(np.arange(k), s)
        _, num, M = oracle.modularity(g.off, g.col, g.w, memb)
        assert Fraction(num, M * M) == 1 - Fraction(1, k)


def test_modularity_closed_form_ring_of_cliques():
    for k, s in [(3, 4), (8, 5), (30, 3)]:
        g = cliques(k, s, ring=True)
        memb = np.repeat(np.arange(k), s)
        _, num, M = oracle.modularity(g.off, g.col, g.w, memb)
        assert Fraction(num, M * M) == Fraction(s * (s - 1), s * (s - 1) + 2) - Fraction(1, k)


def test_modularity_singletons_and_one_community():
    rng = random.Random(3)
    g = random_graph(rng, 8, 0.6, loops=False)
    A = dense(g)
    K = [sum(r) for r in A]
    M = sum(K)
    _, num, _ = oracle.modularity(g.off, g.col, g.w, np.arange(8))
    assert Fraction(num, M * M) == -Fraction(sum(k * k for k in K), M * M)
    _, num, _ = oracle.modularity(g.off, g.col, g.w, np.zeros(8, np.int32))
    assert num == 0


# ----------------------------------------------------------- gain (a3)

def test_gain_equals_exact_modularity_difference():
    """For every vertex and candidate: gain * 2 / M^2 == Q(after) - Q(before), exactly."""
    rng = random.Random(4)
    checked = 0
    for _ in range(30):
        n = rng.randint(2, 9)
        g = random_graph(rng, n, 0.5)
        A = dense(g)
        M = sum(map(sum, A))
        if M == 0:
            continue
        memb = [rng.randrange(n) for _ in range(n)]
        q0 = q_pairwise(A, memb)
        for i in range(n):
            gains = oracle.vertex_gains(g.off, g.col, g.w, memb, i)
            nb = {memb[int(g.col[e])] for e in range(int(g.off[i]), int(g.off[i + 1])) if int(g.col[e]) != i}
            assert set(gains) == nb - {memb[i]}
            for c, gain in gains.items():
                after = list(memb)
                after[i] = c
                assert Fraction(2 * gain, M * M) == q_pairwise(A, after) - q0
                checked += 1
    assert checked > 100


# ------------------------------------------------------ brute force (O2)

def test_brute_force_enumerates_bell_numbers_and_known_optima():
    for n in range(1, 9):
        g = gg.from_weighted_edges(n, [(i, i + 1, 1) for i in range(n - 1)])
        _, _, cnt = oracle.brute_best(g.off, g.col, g.w)
        assert cnt == bell(n)
    with open(GOLDEN) as f:
        case = [c for c in json.load(f)["cases"] if c["name"] == "two_triangles_bridge_optimum"][0]
    g = gg.from_weighted_edges(case["n"], [tuple(e) for e in case["edges"]])
    best, memb, cnt = oracle.brute_best(g.off, g.col, g.w)
    assert best == case["expect"]["best_q_num"] and cnt == case["expect"]["partitions"]
    assert len(set(memb[:3])) == 1 and len(set(memb[3:])) == 1 and memb[0] != memb[3]
    # complete graph: nothing beats one community (Q = 0)
    g = cliques(1, 6)
    best, _, _ = oracle.brute_best(g.off, g.col, g.w)
    assert best == 0


def test_brute_force_agrees_with_exhaustive_pairwise_search():
    rng = random.Random(5)
    for _ in range(5):
        n = rng.randint(2, 6)
        g = random_graph(rng, n, 0.5)
        A = dense(g)
        M = sum(map(sum, A))
        if M == 0:
            continue
        best_exact = max(q_pairwise(A, m) for m in itertools.product(range(n), repeat=n))
        best, _, _ = oracle.brute_best(g.off, g.col, g.w)
        assert Fraction(best, M * M) == best_exact


# ---------------------------------------------------------- Louvain runs

def test_hand_worked_runs():
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        if case["options"] is None:
            continue
        g = gg.from_weighted_edges(case["n"], [tuple(e) for e in case["edges"]])
        o = dict(case["options"])
        mode = oracle.SYNC if o.pop("mode") == "sync" else oracle.ASYNC
        for prune in ([o.pop("prune")] if "prune" in o else (0, 1)):
            r = run(g, mode=mode, prune=prune, **o)
            ex = case["expect"]
            assert list(r.top) == ex["top"], case["name"]
            assert r.q_num == ex["q_num"] and r.M == ex["M"], case["name"]
            assert r.Q == ex["Q"], case["name"]
            assert [list(t) for t in r.iterations] == ex["iterations"], case["name"]


@pytest.mark.parametrize("mode,colour", [(oracle.SYNC, 0), (oracle.ASYNC, 0), (oracle.SYNC, 1)])
def test_louvain_never_beats_brute_force_and_finds_clique_optimum(mode, colour):
    rng = random.Random(6)
    for _ in range(25):
        n = rng.randint(2, 10)
        g = random_graph(rng, n, 0.4)
        if g.nnz == 0:
            continue
        r = run(g, mode=mode, colour_classes=colour)
        best, _, _ = oracle.brute_best(g.off, g.col, g.w)
        assert r.q_num <= best
        _, num, _ = oracle.modularity(g.off, g.col, g.w, r.top)
        assert num == r.q_num
    for k, s in [(2, 4), (3, 3), (5, 5)]:
        g = cliques(k, s)
        r = run(g, mode=mode, colour_classes=colour)
        assert Fraction(r.q_num, r.M * r.M) == 1 - Fraction(1, k)
        best, _, _ = oracle.brute_best(g.off, g.col, g.w) if k * s <= 10 else (r.q_num, None, None)
        assert r.q_num == best


@pytest.mark.parametrize("mode,colour", [(oracle.SYNC, 0), (oracle.ASYNC, 0), (oracle.SYNC, 1)])
def test_louvain_ring_of_cliques_reaches_clique_partition(mode, colour):
    for k, s in [(6, 5), (12, 4)]:
        g = cliques(k, s, ring=True)
        r = run(g, mode=mode, colour_classes=colour)
        clique_q = Fraction(s * (s - 1), s * (s - 1) + 2) - Fraction(1, k)
        assert Fraction(r.q_num, r.M * r.M) >= clique_q


@pytest.mark.parametrize("mode,colour", [(oracle.SYNC, 0), (oracle.ASYNC, 0), (oracle.SYNC, 1)])
@pytest.mark.parametrize("prune", [0, 1])
@pytest.mark.parametrize("subrounds", [1, 4])
def test_pass_invariants(mode, colour, prune, subrounds):
    """Aggregation keeps M and Q; levels compose to the top membership; k shrinks."""
    g = gg.sbm(11, 600, 12, 0.15, 0.01, wmin=1, wmax=9)
    r = run(g, mode=mode, prune=prune, subrounds=subrounds, record_levels=True, colour_classes=colour)
    assert r.Q > 0.3
    off, col, w = g.off, g.col, g.w.astype(np.int64)
    top = np.arange(g.n)
    for p, ps in enumerate(r.passes):
        assert ps.n == len(off) - 1
        if ps.level is None:
            break
        k = ps.k
        assert sorted(set(ps.level.tolist())) == list(range(k))
        # Q numerator after the pass equals the modularity of the level on the pass graph
        _, num, M = oracle.modularity(off, col, w, ps.level)
        assert num == ps.n_after and M == r.M
        top = ps.level[top]
        if ps.coarse is not None:
            co, cc, cw = ps.coarse
            assert int(cw.sum()) == r.M                     # total weight preserved
            _, num_c, _ = oracle.modularity(co, cc, cw, np.arange(k))
            assert num_c == ps.n_after                     # Q preserved exactly
            oo, oc, ow = oracle.aggregate(off, col, w, ps.level, k)
            assert np.array_equal(oo, co) and np.array_equal(oc, cc) and np.array_equal(ow, cw)
            for C in range(k):                             # canonical rows
                row = cc[co[C]:co[C + 1]]
                assert np.all(np.diff(row) > 0)
            # coarse degrees are the community totals Sigma_C of the fine graph
            K = np.array([w[off[i]:off[i + 1]].sum() for i in range(len(off) - 1)], np.int64)
            sig = np.bincount(ps.level, weights=K, minlength=k).astype(np.int64)
            coarse_K = np.array([cw[co[C]:co[C + 1]].sum() for C in range(k)], np.int64)
            assert np.array_equal(sig, coarse_K)
            off, col, w = co, cc, cw
            assert p + 1 < len(r.passes)
            assert r.passes[p + 1].n == k and k < ps.n
    assert np.array_equal(top, r.top)
    _, num, _ = oracle.modularity(g.off, g.col, g.w, r.top)
    assert num == r.q_num


def test_async_gains_sum_to_the_exact_modularity_change():
    """Sequential Gauss-Seidel: S of an iteration equals the true Q change * M^2 / 2."""
    g = gg.sbm(12, 400, 8, 0.2, 0.02)
    for iters in (1, 2, 3):
        r = run(g, mode=oracle.ASYNC, max_iterations=iters, max_passes=1, tolerance=0.0)
        total_S = sum(S for (p, m, S) in r.iterations if p == 0)
        assert 2 * total_S == r.passes[0].n_after - r.passes[0].n_before


def test_recomputed_stop_rule_equals_sum_of_gains_in_sequential_order():
    """stop_rule 1 (the exact Q change of each iteration, recomputed) and
    stop_rule 0 (2S) agree in sequential asynchronous order, where every gain
    is the true change: same traces, memberships and Q on random and SBM
    graphs.  A ΔN taken over the wrong span (say since the pass began) or
    without the factor of two would stop at other iterations."""
    rng = random.Random(14)
    graphs = [gg.sbm(13, 600, 10, 0.12, 0.01, wmin=1, wmax=7), gg.rmat(15, 11, 8, wmin=1, wmax=5)]
    graphs += [random_graph(rng, rng.randint(5, 12), 0.4) for _ in range(20)]
    for g in graphs:
        for tol in (0.01, 0.001, 0.05):
            a = run(g, mode=oracle.ASYNC, prune=1, tolerance=tol)
            b = run(g, mode=oracle.ASYNC, prune=1, tolerance=tol, stop_rule=1)
            assert a.iterations == b.iterations
            assert np.array_equal(a.top, b.top) and a.q_num == b.q_num


def test_recomputed_stop_rule_in_synchronous_order():
    """In synchronous order the recomputed change is what the moves did:
    each pass's iterations end at the first iteration whose own exact change
    N(after) - N(before) is at most tolerance * M^2 (replayed here iteration by
    iteration, with max_iterations cut, from runs of the oracle itself)."""
    g = gg.sbm(16, 900, 12, 0.1, 0.01, wmin=1, wmax=4)
    full = run(g, mode=oracle.SYNC, stop_rule=1, max_passes=1, tolerance=0.01)
    M2 = full.M * full.M
    n_prev = full.passes[0].n_before
    for t in range(1, full.passes[0].iterations + 1):
        r = run(g, mode=oracle.SYNC, stop_rule=1, max_passes=1, tolerance=0.01, max_iterations=t)
        n_t = r.passes[0].n_after
        settled = float(n_t - n_prev) / float(M2) <= 0.01
        assert settled == (t == full.passes[0].iterations and t < 20), t
        n_prev = n_t
    # and the sum-of-gains rule over-counts here: 2 * sum S exceeds the pass's exact change
    s0 = run(g, mode=oracle.SYNC, max_passes=1, tolerance=0.01)
    assert 2 * sum(S for (_, _, S) in s0.iterations) > s0.passes[0].n_after - s0.passes[0].n_before


def test_modularity_range_and_sync_async_quality():
    """Q stays in [-1/2, 1] (Section 1); sync and async reach equivalent quality (Section 3.2)."""
    g = gg.sbm(0x5EED, 2048, 16, 0.1, 0.002)
    rs = run(g, mode=oracle.SYNC, prune=1)
    rp = run(g, mode=oracle.SYNC, prune=1, subrounds=8)
    ra = run(g, mode=oracle.ASYNC, prune=1)
    for r in (rs, rp, ra):
        assert -0.5 <= r.Q <= 1.0
    assert abs(rs.Q - ra.Q) < 0.05 and abs(rp.Q - ra.Q) < 0.02
    # the planted partition is (near) optimal here; Louvain should come close to it
    q_truth, _, _ = oracle.modularity(g.off, g.col, g.w, g.truth)
    assert ra.Q >= q_truth - 0.02


def test_plain_jacobi_oscillates_and_guard_fixes_it():
    """Plain Jacobi swaps singleton pairs (the slow sync convergence of Section 3.2);
    the singleton guard restores quality close to the sequential (async) run."""
    g = gg.sbm(11, 600, 12, 0.15, 0.01, wmin=1, wmax=9)
    plain = run(g, mode=oracle.SYNC, singleton_guard=0)
    guard = run(g, mode=oracle.SYNC, singleton_guard=1)
    seq = run(g, mode=oracle.ASYNC)
    assert plain.iterations[0][1] == g.n and plain.passes[0].iterations == 20
    assert guard.Q > plain.Q + 0.2 and guard.Q > seq.Q - 0.02


def test_empty_and_edgeless_graphs():
    g = gg.from_weighted_edges(0, [])
    r = run(g)
    assert r.Q == 0.0 and len(r.top) == 0 and r.passes == []
    g = gg.from_weighted_edges(5, [])
    r = run(g)
    assert r.Q == 0.0 and list(r.top) == list(range(5))
    g = gg.from_weighted_edges(3, [(1, 1, 4)])   # a lone self-loop: nothing to move to
    r = run(g)
    assert list(r.top) == [0, 1, 2] and r.passes[0].moves == 0


# ------------------------------------------ incremental re-runs (warm start)

@pytest.mark.parametrize("mode", [oracle.SYNC, oracle.ASYNC])
@pytest.mark.parametrize("prune", [0, 1])
def test_warm_start_from_singletons_is_the_cold_run(mode, prune):
    """Starting from the singleton partition is the method as stated: the
    same iterations, passes, levels and result."""
    rng = random.Random(7)
    for trial in range(4):
        g = gg.sbm(100 + trial, 120, 4, 0.3, 0.03, wmin=1, wmax=4)
        cold = run(g, mode=mode, prune=prune, record_levels=True)
        warm = run(g, mode=mode, prune=prune, record_levels=True, initial=np.arange(g.n))
        assert np.array_equal(cold.top, warm.top) and cold.q_num == warm.q_num
        assert cold.iterations == warm.iterations
        for a, b in zip(cold.passes, warm.passes):
            assert (a.n, a.nnz, a.k, a.moves, a.n_before, a.n_after) == (b.n, b.nnz, b.k, b.moves, b.n_before, b.n_after)


def test_warm_start_async_never_lowers_the_initial_modularity():
    """Sequential moves only take positive gains and aggregation keeps Q, so
    an asynchronous re-run ends at least at the initial partition's Q."""
    rng = random.Random(11)
    for trial in range(12):
        g = gg.sbm(200 + trial, 90, 3, 0.3, 0.05, wmin=1, wmax=5)
        init = np.array([rng.randrange(g.n) for _ in range(g.n)], np.int32)
        q0, _, _ = oracle.modularity(g.off, g.col, g.w, init)
        r = run(g, mode=oracle.ASYNC, initial=init)
        assert r.passes[0].n_before == oracle.modularity(g.off, g.col, g.w, init)[1]
        assert r.Q >= q0 - 1e-12, (r.Q, q0)


def test_warm_start_where_nothing_can_move_keeps_the_initial_partition():
    """No vertex has a neighbour outside its community (one community per
    connected piece): nothing moves, and the result is the initial partition,
    renumbered, with its own modularity; from the clique partition of
    disjoint cliques likewise (Q = 1 - 1/k)."""
    g = cliques(3, 4)
    one = np.zeros(g.n, np.int32)
    for mode in (oracle.SYNC, oracle.ASYNC):
        r = run(g, mode=mode, initial=one)
        assert len(r.passes) == 1 and r.passes[0].moves == 0
        assert np.array_equal(r.top, one) and r.q_num == oracle.modularity(g.off, g.col, g.w, one)[1]
        blocks = (np.arange(g.n) // 4).astype(np.int32) * 4   # ids 0, 4, 8: renumbered to 0, 1, 2
        r = run(g, mode=mode, initial=blocks)
        assert np.array_equal(r.top, np.arange(g.n) // 4)
        assert Fraction(int(r.q_num), r.M * r.M) == 1 - Fraction(1, 3)


def test_warm_start_rejects_out_of_range_memberships():
    g = cliques(2, 3)
    for bad in ([0, 1, 2, 3, 4, 6], [-1, 0, 0, 0, 0, 0]):
        with pytest.raises(ValueError):
            run(g, initial=np.array(bad, np.int32))


# ------------------------------------------------ colour classes (option f1)

def _check_greedy_classes(g, cls, k):
    """Pins of a capped greedy colouring that do not depend on the priority
    order: classes below 63 hold no two neighbours; a vertex in class c < 63
    has a neighbour in every class below c (it took the smallest free one);
    one in class 63 has neighbours in all of 0..62; the count is max + 1."""
    assert k == (int(cls.max()) + 1 if g.n else 1)
    assert cls.min(initial=0) >= 0 and cls.max(initial=0) <= 63
    for v in range(g.n):
        nb = {int(cls[u]) for u in g.col[g.off[v]:g.off[v + 1]] if u != v}
        c = int(cls[v])
        if c < 63:
            assert c not in nb, (v, c)
            assert set(range(c)) <= nb, (v, c)
        else:
            assert set(range(63)) <= nb, v


@pytest.mark.parametrize("seed", range(6))
def test_colour_classes_are_a_greedy_colouring(seed):
    rng = random.Random(seed)
    g = random_graph(rng, 60, 0.15 + 0.1 * seed)
    for p in range(3):
        cls, k = oracle.colour_classes(g.off, g.col, p)
        _check_greedy_classes(g, cls, k)
    big = gg.rmat(seed, 11, 8, wmin=1, wmax=4)
    cls, k = oracle.colour_classes(big.off, big.col, 0)
    _check_greedy_classes(big, cls, k)


def test_colour_classes_special_cases():
    # a clique of 70: classes 0..62 once each, the last 7 vertices share 63
    c70 = cliques(1, 70)
    cls, k = oracle.colour_classes(c70.off, c70.col, 0)
    assert k == 64 and sorted(cls.tolist()) == list(range(63)) + [63] * 7
    # a star takes two classes, whichever vertex comes first; isolated vertices take 0
    star = gg.from_weighted_edges(9, [(0, v, 1) for v in range(1, 8)])
    cls, k = oracle.colour_classes(star.off, star.col, 0)
    assert k == 2 and cls[8] == 0 and all(cls[v] != cls[0] for v in range(1, 8))
    empty = gg.from_weighted_edges(0, [])
    assert oracle.colour_classes(empty.off, empty.col, 0)[1] == 1
    # deterministic, and drawn anew for every pass
    g = gg.sbm(3, 500, 5, 0.1, 0.01)
    a0, _ = oracle.colour_classes(g.off, g.col, 0)
    assert np.array_equal(a0, oracle.colour_classes(g.off, g.col, 0)[0])
    assert not np.array_equal(a0, oracle.colour_classes(g.off, g.col, 1)[0])


def test_colour_class_runs_reach_closed_forms_and_exact_q():
    for k, s in [(3, 4), (5, 6), (8, 3)]:
        r = run(cliques(k, s), mode=oracle.SYNC, colour_classes=1)
        assert Fraction(r.q_num, r.M * r.M) == 1 - Fraction(1, k)
    g = gg.sbm(11, 600, 12, 0.15, 0.01, wmin=1, wmax=9)
    for prune in (0, 1):
        r = run(g, mode=oracle.SYNC, colour_classes=1, prune=prune)
        _, num, _ = oracle.modularity(g.off, g.col, g.w, r.top)
        assert num == r.q_num and r.Q > 0.3


def test_colour_classes_on_a_clique_are_the_sequential_order():
    """On a clique every vertex has a class of its own, so the colour-class
    run (Jacobi per class, no guard) is the sequential run in class order:
    the oracle's asynchronous run on the vertices renumbered by class."""
    rng = random.Random(5)
    n = 40
    # weights from a wide range: no two candidate gains tie, so the lowest-id
    # tie rule (which the renumbering would change) never decides
    edges = [(u, v, rng.randint(1, 1_000_000)) for u in range(n) for v in range(u + 1, n)]
    g = gg.from_weighted_edges(n, edges)
    cls, k = oracle.colour_classes(g.off, g.col, 0)
    assert k == n and sorted(cls.tolist()) == list(range(n))
    # renumber: new id = class
    edges2 = [(int(cls[u]), int(cls[v]), w) for (u, v, w) in edges]
    g2 = gg.from_weighted_edges(n, edges2)
    a = run(g, mode=oracle.SYNC, colour_classes=1, singleton_guard=0, max_passes=1)
    b = run(g2, mode=oracle.ASYNC, max_passes=1)
    assert a.q_num == b.q_num
    assert a.iterations == b.iterations                  # every iteration's moves and gain sum
    pairs = {(int(a.top[v]), int(b.top[cls[v]])) for v in range(n)}
    assert len(pairs) == len({x for x, _ in pairs}) == len({y for _, y in pairs})   # the same partition


def test_relabelled_graph_keeps_modularity_and_async_reference():
    """The relabelling used for the asynchronous reference (engine_util) is a
    graph isomorphism: same M, same modularity of the correspondingly renamed
    membership, still symmetric; and a run at the id-order Q meets it."""
    from engine_util import relabelled, async_within_tolerance
    g = gg.sbm(21, 500, 9, 0.1, 0.01, wmin=1, wmax=6)
    memb = np.random.default_rng(3).integers(0, 9, g.n).astype(np.int32)
    off, col, w = relabelled(g.off, g.col, g.w, 7)
    perm = np.random.default_rng(7).permutation(g.n)
    memb2 = np.empty_like(memb)
    memb2[perm] = memb
    assert oracle.modularity(off, col, w, memb2) == oracle.modularity(g.off, g.col, g.w, memb)
    A = {}
    for u in range(g.n):
        for e in range(off[u], off[u + 1]):
            A[(u, int(col[e]))] = int(w[e])
    assert all(A.get((v, u)) == x for (u, v), x in A.items())
    q_id = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1).Q
    assert async_within_tolerance(g.off, g.col, g.w, q_id)[0]
    assert not async_within_tolerance(g.off, g.col, g.w, -1.0)[0]
