"""Independent reference computations used by the oracle pins (pure Python, no
oracle code): exhaustive label enumeration, Dijkstra, a weighted-sum single-label
search, random tiny graphs, and checks of the invariants every explore result must
satisfy."""
import heapq

import numpy as np


def transfer(S, C, h):
    return max(int(C), int(h) + int(S))


def steps_to_SC(d):
    h, S = 0, 0
    for x in d:
        S += int(x)
        h = max(0, h + int(x))
    return S, h


def random_graph(rng, V, p_edge=0.4, cmax=6, dmax=4, steps=4):
    rows, dst, cq, S, C = [0], [], [], [], []
    for v in range(V):
        for u in range(V):
            if u != v and rng.random() < p_edge:
                d = rng.integers(-dmax, dmax + 1, steps)
                s, c = steps_to_SC(d)
                dst.append(u); cq.append(int(rng.integers(1, cmax + 1))); S.append(s); C.append(c)
        rows.append(len(dst))
    goal = (rng.random(V) < 0.3).astype(np.uint8)
    goal[0] = 0
    if goal.sum() == 0:
        goal[V - 1] = 1
    return (np.array(rows, np.uint32), np.array(dst, np.uint32), np.array(cq, np.int32),
            np.array(S, np.int32), np.array(C, np.int32), goal)


def brute_labels(row_ptr, dst, cq, S, C, beta, bound):
    """Every (node, cost, h) label of walks from node 0 with cost <= bound whose
    heuristic never exceeds beta at a plan head (Alg. 3 cutoff)."""
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
                h2 = transfer(S[e], C[e], h)
                if h2 > beta:
                    continue
                lab = (int(dst[e]), c2, h2)
                if lab not in seen:
                    seen.add(lab)
                    nxt.append(lab)
        frontier = nxt
    return seen


def pareto(values):
    """Weak-Pareto minimal (cost, h) pairs, sorted by cost."""
    vals = sorted(set(values))
    out = []
    best_h = None
    for c, h in vals:
        if best_h is None or h < best_h:
            out.append((c, h))
            best_h = h
    return out


def brute_fronts(V, row_ptr, dst, cq, S, C, beta, bound):
    labs = brute_labels(row_ptr, dst, cq, S, C, beta, bound)
    per = [[] for _ in range(V)]
    for v, c, h in labs:
        per[v].append((c, h))
    return [pareto(p) for p in per]


def dijkstra(row_ptr, dst, cq, src=0):
    V = len(row_ptr) - 1
    dist = [None] * V
    dist[src] = 0
    pq = [(0, src)]
    while pq:
        d, v = heapq.heappop(pq)
        if d > dist[v]:
            continue
        for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
            u = int(dst[e]); nd = d + int(cq[e])
            if dist[u] is None or nd < dist[u]:
                dist[u] = nd
                heapq.heappush(pq, (nd, u))
    return dist


def weighted_sum_search(row_ptr, dst, cq, S, C, goal, beta, w):
    """Single label per node, ordered by cost + w h (the combined-cost alternative
    that Sec. 3 argues against); labels violating beta are discarded."""
    V = len(row_ptr) - 1
    best = [None] * V
    best[0] = (0.0, 0, 0)
    pq = [(0.0, 0, 0, 0)]
    while pq:
        key, v, c, h = heapq.heappop(pq)
        if best[v] is not None and (key, c, h) != best[v]:
            continue
        if goal[v]:
            return c, h
        for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
            u = int(dst[e]); c2 = c + int(cq[e]); h2 = transfer(S[e], C[e], h)
            if h2 > beta:
                continue
            k2 = c2 + w * h2
            if best[u] is None or k2 < best[u][0]:
                best[u] = (k2, c2, h2)
                heapq.heappush(pq, (k2, u, c2, h2))
    return None


def check_invariants(g, res, beta):
    """Properties every Explore result satisfies (fronts strictly monotone and
    non-dominated, h within beta, the path a walk whose recomputed (cost, h) is the
    result, the result the best goal plan)."""
    V = g.V if hasattr(g, "V") else len(g.row_ptr) - 1
    for v in range(V):
        f = res.front(v)
        for (c0, h0), (c1, h1) in zip(f, f[1:]):
            assert c1 > c0 and h1 < h0, (v, f)
        for c, h in f:
            assert h <= beta
    assert res.front(0)[0] == (0, 0)
    if res.status != 0:
        return
    path = [int(x) for x in res.path]
    assert path[0] == 0 and g.is_goal[path[-1]]
    c, h = 0, 0
    for a, b in zip(path, path[1:]):
        es = [e for e in range(int(g.row_ptr[a]), int(g.row_ptr[a + 1])) if int(g.dst[e]) == b]
        assert len(es) == 1
        e = es[0]
        c += int(g.cost_q[e]); h = transfer(g.S[e], g.C[e], h)
        assert h <= beta
    assert (c, h) == (res.cost, res.h)
    goal_plans = [ch for v in range(V) if g.is_goal[v] for ch in res.front(v)]
    assert min(goal_plans) == (res.cost, res.h)
