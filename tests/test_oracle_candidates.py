"""Pins of the oracle's candidate export (P_candidates, Alg. 3 final lines) and of
its trajectory features (the certification surrogate's input) -- CPU only.

Candidates are checked against exhaustive label enumeration on tiny graphs and by
re-walking every candidate's node sequence through the exported edges; features
against closed forms on straight-line plans in the unit square."""
import math

import numpy as np
import pytest

from _search_ref import brute_fronts, random_graph, transfer

BIG = 1 << 62


def _walk(row_ptr, dst, cq, S, C, path):
    """(cost, h) of a node sequence, re-walked through the CSR edges."""
    cost, h = 0, 0
    for a, b in zip(path[:-1], path[1:]):
        es = [e for e in range(int(row_ptr[a]), int(row_ptr[a + 1])) if int(dst[e]) == int(b)]
        assert es, (a, b)
        e = es[0]
        cost += int(cq[e])
        h = transfer(S[e], C[e], h)
    return cost, h


@pytest.mark.parametrize("seed", range(30))
def test_candidates_are_the_goal_fronts_in_order(orc, seed):
    rng = np.random.default_rng(4000 + seed)
    V = int(rng.integers(3, 8))
    g = random_graph(rng, V, dmax=3)
    row_ptr, dst, cq, S, C, goal = g
    beta = int(rng.choice([3, 6, 10, BIG]))
    ref = brute_fronts(V, row_ptr, dst, cq, S, C, beta, 5 * V * 6)
    want = sorted((c, h, v) for v in range(V) if goal[v] for (c, h) in ref[v])
    res = orc.explore(orc.roadmap_from_csr(*g), beta, 1, goal_termination=False, candidates=256)
    if not want:
        assert res.status == 1 and res.candidates is None
        return
    cand = res.candidates
    assert cand["total"] == len(want) == len(cand["paths"])
    got = [(int(c), int(h), int(p[-1])) for c, h, p in zip(cand["cost"], cand["h"], cand["paths"])]
    assert got == want
    # the first candidate is the returned solution
    assert (cand["cost"][0], cand["h"][0]) == (res.cost, res.h)
    np.testing.assert_array_equal(cand["paths"][0], res.path)
    for c, h, p in zip(cand["cost"], cand["h"], cand["paths"]):
        assert int(p[0]) == 0 and goal[int(p[-1])]
        assert _walk(row_ptr, dst, cq, S, C, p) == (int(c), int(h))


def test_candidate_cap_keeps_the_prefix(orc):
    rng = np.random.default_rng(77)
    g = random_graph(rng, 7, p_edge=0.6, dmax=4)
    rm = orc.roadmap_from_csr(*g)
    full = orc.explore(rm, BIG, 1, goal_termination=False, candidates=1000).candidates
    assert full["total"] >= 2
    part = orc.explore(rm, BIG, 1, goal_termination=False, candidates=2).candidates
    assert part["total"] == full["total"] and len(part["paths"]) == 2
    np.testing.assert_array_equal(part["cost"], full["cost"][:2])


# ---------------------------------------------------------------------------
# features
# ---------------------------------------------------------------------------
K = 24


def _line(orc, pts, grid, G, boxes=None, M=16):
    """Roadmap whose nodes are `pts` (2D), chained by the r-disk graph."""
    pts = np.asarray(pts, np.float64)
    x = np.zeros((6, len(pts)), np.float32)
    x[0], x[1] = pts[:, 0], pts[:, 1]
    gaps = np.linalg.norm(np.diff(pts, axis=0), axis=1)
    lo = np.zeros((0, 3)) if boxes is None else np.asarray(boxes[0], np.float32)
    hi = np.zeros((0, 3)) if boxes is None else np.asarray(boxes[1], np.float32)
    rm = orc.build_roadmap_from_points(2, lo, hi, np.asarray(grid, np.uint8), G, x,
                                       r=float(gaps.max()) * 1.01, M=M, goal_radius=0.001)
    return rm, np.arange(len(pts), dtype=np.uint32)


def _checkpoints(pts, M=16):
    pts = np.asarray(pts, np.float64)
    out = []
    for a, b in zip(pts[:-1], pts[1:]):
        for m in range(1, M + 1):
            out.append(a + (m / M) * (b - a))
    return np.array(out)


def test_features_of_a_free_diagonal(orc):
    """Constant level L, no boxes: max = L/K, sum = (checkpoints in bin) L/(64 K),
    clearance = distance to the nearest wall along the diagonal."""
    L = 7
    pts = [(0.2, 0.2), (0.5, 0.5), (0.8, 0.8)]
    rm, path = _line(orc, pts, np.full(4, L), 2)
    f = orc.plan_features(rm, [path])[0]
    ck = _checkpoints(pts)                       # 32 checkpoints, 2 per bin
    for j in range(16):
        c = ck[2 * j:2 * j + 2]
        assert f[j] == pytest.approx(L / K, rel=1e-7)
        assert f[16 + j] == pytest.approx(2 * L / (64 * K), rel=1e-7)
        clr = np.min(np.minimum(c, 1 - c))
        assert f[32 + j] == pytest.approx(4 * min(0.25, clr), abs=1e-6)


def test_features_of_a_plan_through_a_box_and_two_levels(orc):
    """A box on the diagonal makes the clearance negative (minus the distance to
    the nearest face); a 2x2 grid with levels 3 (lower left) and 11 (upper right)
    gives the levels along the diagonal."""
    pts = [(0.2, 0.2), (0.515, 0.515), (0.83, 0.83)]
    grid = [3, 0, 0, 11]                        # x fastest: cell (0,0) = 3, (1,1) = 11
    boxes = ([[0.45, 0.40, 0.0]], [[0.60, 0.58, 0.0]])
    rm, path = _line(orc, pts, grid, 2, boxes)
    f = orc.plan_features(rm, [path])[0]
    ck = _checkpoints(pts)
    lev = np.where(ck[:, 0] < 0.5, 3, 11)
    lo, hi = np.array(boxes[0][0][:2]), np.array(boxes[1][0][:2])
    for j in range(16):
        c = ck[2 * j:2 * j + 2]
        lv = lev[2 * j:2 * j + 2]
        assert f[j] == pytest.approx(lv.max() / K, rel=1e-7)
        assert f[16 + j] == pytest.approx(lv.sum() / (64 * K), rel=1e-7)
        box = np.max(np.maximum(lo - c, c - hi), axis=1)
        wall = np.min(np.minimum(c, 1 - c), axis=1)
        clr = np.min(np.minimum(box, wall))
        assert f[32 + j] == pytest.approx(4 * min(0.25, clr), abs=1e-6)
    # the bins inside the box are negative
    inside = [j for j in range(16) if np.all((_checkpoints(pts)[2 * j:2 * j + 2] > lo)
                                             & (_checkpoints(pts)[2 * j:2 * j + 2] < hi))]
    assert inside and all(f[32 + j] < 0 for j in inside)


def test_feature_bins_for_uneven_counts(orc):
    """One edge with M = 20 checkpoints: bin j holds s with floor(16 s / 20) = j,
    so bins 0, 4, 8, 12 hold two checkpoints and the rest one."""
    pts = [(0.3, 0.3), (0.31, 0.32)]
    rm, path = _line(orc, pts, np.full(4, 5), 2, M=20)
    f = orc.plan_features(rm, [path])[0]
    counts = np.bincount([(16 * s) // 20 for s in range(20)], minlength=16)
    assert list(counts) == [2, 1, 1, 1, 2, 1, 1, 1, 2, 1, 1, 1, 2, 1, 1, 1]
    np.testing.assert_allclose(f[16:32], counts * 5 / (64 * K), rtol=1e-7)
    np.testing.assert_allclose(f[:16], 5 / K, rtol=1e-7)
