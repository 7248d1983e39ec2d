"""Pins for the oracle's Alg. 3 (Explore) and RemoveDominated (CPU only)."""
import os

import numpy as np
import pytest

import scenegen
from _search_ref import (brute_fronts, check_invariants, dijkstra, random_graph,
                         weighted_sum_search)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BIG = (1 << 62)


def _csr(orc, g):
    return orc.roadmap_from_csr(*g)


@pytest.mark.parametrize("seed", range(40))
def test_fronts_equal_brute_force(orc, seed):
    """With goal termination off, Explore runs until P_open is empty; its final
    fronts must equal the Pareto fronts of all walk labels (exhaustive
    enumeration), for any group width."""
    rng = np.random.default_rng(seed)
    V = int(rng.integers(3, 8))
    g = random_graph(rng, V, dmax=3)
    row_ptr, dst, cq, S, C, goal = g
    beta = int(rng.choice([3, 6, 10, 1 << 40]))
    bound = 5 * V * 6
    ref = brute_fronts(V, row_ptr, dst, cq, S, C, beta, bound)
    ref_big = brute_fronts(V, row_ptr, dst, cq, S, C, beta, bound + bound // 2)
    assert ref == ref_big          # the enumeration bound is not binding
    rm = _csr(orc, g)
    for lam in (1, 3, 1000):
        res = orc.explore(rm, beta, lam, goal_termination=False)
        assert res.status in (0, 1)
        got = [res.front(v) for v in range(V)]
        assert got == ref, (lam, got, ref)


@pytest.mark.parametrize("seed", range(40))
def test_unit_group_width_is_optimal(orc, seed):
    """With Lambda = one cost quantum the goal test cannot fire early: the returned
    cost is the constrained optimum over all walks (brute force)."""
    rng = np.random.default_rng(1000 + seed)
    V = int(rng.integers(3, 9))
    g = random_graph(rng, V)
    row_ptr, dst, cq, S, C, goal = g
    beta = int(rng.choice([4, 8, 1 << 40]))
    ref = brute_fronts(V, row_ptr, dst, cq, S, C, beta, 8 * V * 6)
    goal_labels = [ch for v in range(V) if goal[v] for ch in ref[v]]
    rm = _csr(orc, g)
    res = orc.explore(rm, beta, 1)
    if not goal_labels:
        assert res.status == 1
    else:
        assert res.status == 0
        assert (res.cost, res.h) == min(goal_labels)
        gg = rm.graph()
        check_invariants(gg, res, beta)


def test_large_group_width_terminates_early(orc):
    """Sec. 3: a large group factor can stop the search before the optimal plan
    reaches X_goal.  Direct edge 0 -> 1 (cost 10) versus 0 -> 2 -> 1 (cost 2)."""
    row_ptr = np.array([0, 2, 2, 3], np.uint32)
    dst = np.array([1, 2, 1], np.uint32)
    cq = np.array([10, 1, 1], np.int32)
    z = np.zeros(3, np.int32)
    goal = np.array([0, 1, 0], np.uint8)
    rm = orc.roadmap_from_csr(row_ptr, dst, cq, z, z, goal)
    wide = orc.explore(rm, BIG, 100)
    assert (wide.status, wide.cost, list(wide.path)) == (0, 10, [0, 1])
    narrow = orc.explore(rm, BIG, 1)
    assert (narrow.status, narrow.cost, list(narrow.path)) == (0, 2, [0, 2, 1])


def test_narrow_passage_fig2(orc):
    lines = [l.split() for l in open(os.path.join(GOLDEN, "narrow_passage_fig2.txt"))
             if l.strip() and not l.startswith("#")]
    V, beta, goal_node = map(int, lines[0])
    edges = [tuple(map(int, l)) for l in lines[1:-1]]
    exp = list(map(int, lines[-1]))
    edges.sort()
    row_ptr = np.zeros(V + 1, np.uint32)
    for s, *_ in edges:
        row_ptr[s + 1:] += 1
    dst = np.array([e[1] for e in edges], np.uint32)
    cq = np.array([e[2] for e in edges], np.int32)
    S = np.array([e[3] for e in edges], np.int32)
    C = np.array([e[4] for e in edges], np.int32)
    goal = np.zeros(V, np.uint8); goal[goal_node] = 1
    assert weighted_sum_search(row_ptr, dst, cq, S, C, goal, beta, 0.2) is None
    rm = orc.roadmap_from_csr(row_ptr, dst, cq, S, C, goal)
    res = orc.explore(rm, beta, 1)
    assert [res.status, res.cost, res.h] + list(res.path) == exp
    # both partial plans survive at the passage entrance
    assert res.front(3) == [(2, 5), (4, 0)]


@pytest.mark.parametrize("k", [3, 12, 20])
def test_constant_level_reduces_to_dijkstra(orc, k):
    """Constant quality level: h = M (n_f - k) cost for k < n_f, h = 0 otherwise,
    so fronts collapse to one plan and the exhaustive search cost is the shortest
    path (textbook Dijkstra on the same graph)."""
    sc = scenegen.make_scene("2d", 6)
    sc.grid = np.full(sc.grid.size, k, np.uint8)
    rm = orc.build_roadmap(sc, n=400, r=0.1)
    g = rm.graph()
    dist = dijkstra(g.row_ptr, g.dst, g.cost_q)
    goal_d = min(dist[v] for v in range(g.V) if g.is_goal[v] and dist[v] is not None)
    Lam = orc.group_width(0.5, 0.1)
    res = orc.explore(rm, BIG, Lam, goal_termination=False)
    assert res.status == 0 and res.cost == goal_d
    assert max(np.diff(res.front_ptr)) == 1
    scale = 16 * max(12 - k, 0)
    assert res.h == scale * goal_d
    check_invariants(g, res, BIG)
    if scale:
        ok = orc.explore(rm, scale * goal_d, Lam, goal_termination=False)
        assert ok.status == 0 and ok.cost == goal_d
        bad = orc.explore(rm, scale * goal_d - 1, Lam, goal_termination=False)
        assert bad.status == 1


def test_integer_graph_dijkstra_with_goal_stop(orc):
    rng = np.random.default_rng(77)
    for _ in range(30):
        V = int(rng.integers(5, 30))
        row_ptr, dst, cq, S, C, goal = random_graph(rng, V, p_edge=0.25, cmax=9)
        z = np.zeros_like(S)
        rm = orc.roadmap_from_csr(row_ptr, dst, cq, z, z, goal)
        dist = dijkstra(row_ptr, dst, cq)
        gd = [dist[v] for v in range(V) if goal[v] and dist[v] is not None]
        res = orc.explore(rm, BIG, 1)
        if not gd:
            assert res.status == 1
        else:
            assert res.status == 0 and res.cost == min(gd) and res.h == 0


@pytest.mark.parametrize("name,seed,n", [("2d", 1, 1000), ("2d", 3, 1000), ("3d", 2, 1500),
                                         ("6d", 1, 2500)])
def test_invariants_on_scenes(orc, name, seed, n):
    sc = scenegen.make_scene(name, seed)
    r = sc.cfg.r if name != "6d" else 20.0
    rm = orc.build_roadmap(sc, n=n, r=r)
    g = rm.graph()
    beta = orc.beta_percentile(rm)
    res = orc.explore(rm, beta, orc.group_width(0.5, r))
    assert res.status in (0, 1)
    check_invariants(g, res, beta)
    agn = orc.explore(rm, BIG, orc.group_width(0.5, r))
    check_invariants(g, agn, BIG)
    # 2D/3D edge costs are symmetric
    if name != "6d":
        cost = {}
        for v in range(g.V):
            for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
                cost[(v, int(g.dst[e]))] = int(g.cost_q[e])
        for (a, b), c in cost.items():
            if (b, a) in cost:
                assert cost[(b, a)] == c
