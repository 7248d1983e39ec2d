"""Pins of the "for all t" form of the perception constraint (Eq. 2): per edge
the peak of the heuristic over its sub-steps is max(Cmax, h + Smax), and with
the interior check Explore's fronts equal exhaustive enumeration of walks whose
heuristic stays within beta at every sub-step (CPU only)."""
import numpy as np
import pytest

import scenegen
from _search_ref import pareto, steps_to_SC

BIG = 1 << 62


def _peaks(d):
    S, h, Smax, Cmax = 0, 0, None, 0
    for x in d:
        S += int(x)
        h = max(0, h + int(x))
        Smax = S if Smax is None else max(Smax, S)
        Cmax = max(Cmax, h)
    return (0 if Smax is None else Smax), Cmax


def _step_walk(h, d, beta):
    """Literal stepping; None if some sub-step exceeds beta."""
    for x in d:
        h = max(0, h + int(x))
        if h > beta:
            return None
    return h


@pytest.mark.parametrize("name,seed", [("2d", 1), ("6d", 2)])
def test_oracle_peaks_equal_literal_stepping(orc, name, seed):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rm = orc.build_roadmap(sc, n=300, r=(sc.cfg.r * 2 if name == "2d" else 20.0))
    g = rm.graph()
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(g.V), np.diff(g.row_ptr))
    for e in rng.choice(len(g.dst), size=min(60, len(g.dst)), replace=False):
        u, v = int(src[e]), int(g.dst[e])
        d = rm.edge_eval(u, v)["d"]
        assert (int(g.S[e]), int(g.C[e])) == steps_to_SC(d)
        for h0 in (0, 1, 7 * 2 ** 20, 2 ** 28):
            hs, h = [], h0
            for x in d:
                h = max(0, h + int(x))
                hs.append(h)
            assert max(hs) == max(int(g.Cmax[e]), h0 + int(g.Smax[e]))


def _random_steps_graph(rng, V, p_edge=0.4, cmax=6, dmax=4, steps=4):
    rows, dst, cq, st = [0], [], [], []
    for v in range(V):
        for u in range(V):
            if u != v and rng.random() < p_edge:
                dst.append(u)
                cq.append(int(rng.integers(1, cmax + 1)))
                st.append(rng.integers(-dmax, dmax + 1, steps))
        rows.append(len(dst))
    goal = (rng.random(V) < 0.3).astype(np.uint8)
    goal[0] = 0
    if goal.sum() == 0:
        goal[V - 1] = 1
    return np.array(rows, np.uint32), np.array(dst, np.uint32), np.array(cq, np.int32), st, goal


def _brute_fronts_interior(V, row_ptr, dst, cq, steps, beta, bound):
    start = (0, 0, 0)
    seen = {start}
    frontier = [start]
    while frontier:
        nxt = []
        for (v, c, h) in frontier:
            for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
                c2 = c + int(cq[e])
                if c2 > bound:
                    continue
                h2 = _step_walk(h, steps[e], beta)
                if h2 is None:
                    continue
                lab = (int(dst[e]), c2, h2)
                if lab not in seen:
                    seen.add(lab)
                    nxt.append(lab)
        frontier = nxt
    per = [[] for _ in range(V)]
    for v, c, h in seen:
        per[v].append((c, h))
    return [pareto(p) for p in per]


@pytest.mark.parametrize("seed", range(30))
def test_interior_fronts_equal_brute_force(orc, seed):
    rng = np.random.default_rng(7000 + seed)
    V = int(rng.integers(3, 8))
    row_ptr, dst, cq, steps, goal = _random_steps_graph(rng, V, dmax=3)
    SC = [steps_to_SC(d) for d in steps]
    PK = [_peaks(d) for d in steps]
    S = np.array([a for a, _ in SC], np.int32)
    C = np.array([b for _, b in SC], np.int32)
    Smax = np.array([a for a, _ in PK], np.int32)
    Cmax = np.array([b for _, b in PK], np.int32)
    beta = int(rng.choice([2, 4, 7, BIG]))
    ref = _brute_fronts_interior(V, row_ptr, dst, cq, steps, beta, 5 * V * 6)
    assert ref == _brute_fronts_interior(V, row_ptr, dst, cq, steps, beta, 8 * V * 6)
    rm = orc.roadmap_from_csr(row_ptr, dst, cq, S, C, goal, Smax=Smax, Cmax=Cmax)
    for lam in (1, 3, 1000):
        res = orc.explore(rm, beta, lam, goal_termination=False, check_interior=True)
        assert [res.front(v) for v in range(V)] == ref, lam


def test_interior_check_is_at_least_as_strict(orc):
    sc = scenegen.make_scene("2d", 3, query_id=3)
    rm = orc.build_roadmap(sc, n=500)
    beta = orc.beta_percentile(rm)
    lam = orc.group_width(0.5, sc.cfg.r)
    a = orc.explore(rm, beta, lam, goal_termination=False)
    b = orc.explore(rm, beta, lam, goal_termination=False, check_interior=True)
    assert b.expansions <= a.expansions
    # every front entry of the interior search is reachable without it: it is
    # dominated by or equal to an entry of the head-only front
    for v in range(rm.V):
        fa, fb = a.front(v), b.front(v)
        for c, h in fb:
            assert any(ca <= c and ha <= h for ca, ha in fa)
