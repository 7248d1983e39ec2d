"""Pins for the parts of the oracle's roadmap that other pins leave open (CPU
only): the double-integrator edge set of Alg. 2 (Near with the fixed-time
minimum-energy cost, Collision at the interior checkpoints of the cubic, the
unit workspace), the cell index of 3D quality grids, and the heuristic increment
round(T 2^24) (n_f - k) of double-integrator edges (Sec. 4.1)."""
import numpy as np
import pytest

import scenegen


# ----------------------------------------------- 6D Near + Collision (Alg. 2)
def _di6_truth(x, T, M, lo, hi, r):
    """Every ordered pair of a double-integrator roadmap in float64: the cost
    T + J of the fixed-time minimum-energy connection (Sec. 4.1 steering), and
    whether the cubic p(t) = p0 + t v0 + t^2 a0 / 2 + t^3 j / 6 leaves the unit
    cube or meets a closed box at an interior checkpoint t_m = m T / M,
    m = 1 .. M-1.  Also a margin: the smallest distance of any interior
    checkpoint to a box face or a wall, for skipping pairs that float32 rounding
    could decide either way."""
    p = x[:3].T.astype(np.float64)          # [V, 3]
    v = x[3:].T.astype(np.float64)
    V = p.shape[0]
    dp = p[None, :, :] - p[:, None, :] - v[:, None, :] * T        # [u, w, 3]: p1 - p0 - v0 T
    dv = v[None, :, :] - v[:, None, :]
    J = (12 * dp ** 2 / T ** 3 - 12 * dp * dv / T ** 2 + 4 * dv ** 2 / T).sum(-1)
    cost = T + J
    a0 = 6 * dp / T ** 2 - 2 * dv / T
    j = 6 * dv / T ** 2 - 12 * dp / T ** 3
    hit = np.zeros((V, V), bool)
    margin = np.full((V, V), np.inf)
    for m in range(1, M):
        t = m * T / M
        q = p[:, None, :] + t * v[:, None, :] + t * t * a0 / 2 + t ** 3 * j / 6     # [u, w, 3]
        out = ((q < 0) | (q > 1)).any(-1)
        margin = np.minimum(margin, np.abs(q).min(-1))
        margin = np.minimum(margin, np.abs(q - 1).min(-1))
        for b in range(lo.shape[0]):
            inside = ((q >= lo[b]) & (q <= hi[b])).all(-1)
            hit |= inside
            # distance to the box surface (inside: to the nearest face; outside: 0 only when touching)
            d_in = np.minimum(q - lo[b], hi[b] - q).min(-1)
            d_out = np.sqrt((np.maximum(0, np.maximum(lo[b] - q, q - hi[b])) ** 2).sum(-1))
            margin = np.minimum(margin, np.where(inside, d_in, d_out))
        hit |= out
    return cost, hit, margin


def test_di6_edge_set_brute_force(orc):
    """Every robust ordered pair of a small 6D roadmap is an edge iff T + J < r and
    no interior checkpoint of its cubic leaves the unit cube or enters a closed
    box; pairs near the cost threshold or with a checkpoint within 1e-5 of a
    face are skipped.  Among the compared pairs there are connections that
    collide only by leaving the unit cube and connections that meet a box only
    at interior checkpoints, so dropping the workspace rule or testing the
    endpoints only would change the edge set."""
    sc = scenegen.make_scene("6d", 3)
    T, M, r = 0.25, 16, 40.0
    rm = orc.build_roadmap(sc, n=300, r=r)
    g = rm.graph()
    cost, hit, margin = _di6_truth(g.x, T, M, sc.box_lo.astype(np.float64), sc.box_hi.astype(np.float64), r)
    edges = np.zeros((g.V, g.V), bool)
    for u in range(g.V):
        edges[u, g.dst[g.row_ptr[u]:g.row_ptr[u + 1]]] = True
    robust = (np.abs(cost - r) > 1e-4 * r) & (margin > 1e-5)
    np.fill_diagonal(robust, False)
    want = (cost < r) & ~hit
    assert robust.sum() > 20000
    np.testing.assert_array_equal(edges[robust], want[robust])
    # both collision causes occur among compared near pairs
    near = robust & (cost < r)
    p = g.x[:3].T.astype(np.float64)
    in_box_only = np.zeros_like(hit)
    out_only = np.zeros_like(hit)
    for m in range(1, M):
        t = m * T / M
        v = g.x[3:].T.astype(np.float64)
        dp = p[None, :, :] - p[:, None, :] - v[:, None, :] * T
        dv = v[None, :, :] - v[:, None, :]
        a0 = 6 * dp / T ** 2 - 2 * dv / T
        j = 6 * dv / T ** 2 - 12 * dp / T ** 3
        q = p[:, None, :] + t * v[:, None, :] + t * t * a0 / 2 + t ** 3 * j / 6
        out_only |= ((q < 0) | (q > 1)).any(-1)
        for b in range(sc.cfg.nb):
            in_box_only |= ((q >= sc.box_lo[b]) & (q <= sc.box_hi[b])).all(-1)
    assert (near & out_only & ~in_box_only).sum() > 20
    assert (near & in_box_only & ~out_only).sum() > 20


# ----------------------------------------------------- 3D grid cells (Sec. 4.1)
# Levels per octant o = c0 + 2 c1 + 4 c2 of a G = 2 grid (x fastest, then y, z).
OCT = [2, 16, 5, 9, 8, 23, 20, 0]


def test_3d_grid_cells_hand_computed():
    """Three edges of length 0.4 along x, y and z, each from a point 0.31 into its
    cell (M = 16: checkpoints 0.31 + 0.025 m, in the first cell for m = 1..7 and
    in the next for m = 8..16), on a 2x2x2 grid with a distinct level per
    octant.  Per step the heuristic gains cost_q (n_f - k) (n_f = 12); a grid read
    with its axes in another order would see other octants.
      x-edge, octants 0 -> 1 (levels 2, 16):  7 x +10, 9 x -4   S = 34, C = 34, peaks 70, 70
      y-edge, octants 4 -> 6 (levels 8, 20):  7 x +4,  9 x -8   S = -44, C = 0, peaks 28, 28
      z-edge, octants 3 -> 7 (levels 9, 0):   7 x +3,  9 x +12  S = 129, C = 129, peaks 129, 129
      x-edge reversed, octants 1 -> 0:        8 x -4,  8 x +10  S = 48, C = 80, peaks 48, 80
    (all in units of cost_q)."""
    import oracle
    grid = np.array(OCT, np.uint8)
    P = np.array([[0.31, 0.1, 0.1], [0.71, 0.1, 0.1],
                  [0.1, 0.31, 0.9], [0.1, 0.71, 0.9],
                  [0.9, 0.9, 0.31], [0.9, 0.9, 0.71]], np.float32)
    x = np.zeros((6, 6), np.float32)
    x[:3] = P.T
    rm = oracle.build_roadmap_from_points(3, np.zeros((0, 3)), np.zeros((0, 3)), grid, 2, x, r=0.41, M=16)
    g = rm.graph()
    E = {}
    for u in range(g.V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            E[(u, int(g.dst[e]))] = (int(g.cost_q[e]), int(g.S[e]), int(g.C[e]), int(g.Smax[e]), int(g.Cmax[e]))
    assert sorted(E) == [(0, 1), (1, 0), (2, 3), (3, 2), (4, 5), (5, 4)]
    want = {(0, 1): (34, 34, 70, 70), (2, 3): (-44, 0, 28, 28), (4, 5): (129, 129, 129, 129),
            (1, 0): (48, 80, 48, 80)}
    for key, (S, C, Smax, Cmax) in want.items():
        cq = E[key][0]
        assert E[key][1:] == (S * cq, C * cq, Smax * cq, Cmax * cq), key


# ------------------------------------ 6D heuristic increment round(T 2^24) (n_f - k)
@pytest.mark.parametrize("T,inc", [
    (0.25, 4194304),     # 0.25 2^24 exact
    (0.4, 6710886),      # float(0.4) 2^24 = 6710886.5: round half to even
    (0.1, 1677722),      # float(0.1) 2^24 = 1677721.625
])
def test_di6_increment_hand_computed(T, inc):
    """A double-integrator edge at constant velocity (1, 0, 0) over duration T
    from x = 0.31 (its cubic is the straight line x = 0.31 + t, so checkpoint m is
    at 0.31 + m T / 16) on a two-cell grid along x (levels 3 and 19 for x below
    and above 0.5).  Every sub-step lasts T / M, so the increment per step is
    round(T 2^24) (n_f - k) whatever the edge's energy: inc (12 - 3) = 9 inc for
    the steps left of 0.5 and -7 inc for the others.  The expected inc values
    are float32(T) 2^24 rounded to the nearest integer, ties to even."""
    import oracle
    M = 16
    grid = np.zeros(8, np.uint8)
    grid[[0, 2, 4, 6]] = 3      # x cell 0
    grid[[1, 3, 5, 7]] = 19     # x cell 1
    x0 = np.float32(0.31)
    x1 = np.float32(x0 + np.float32(T))
    x = np.zeros((6, 2), np.float32)
    x[:, 0] = [x0, 0.2, 0.2, 1.0, 0.0, 0.0]
    x[:, 1] = [x1, 0.2, 0.2, 1.0, 0.0, 0.0]
    rm = oracle.build_roadmap_from_points(6, np.zeros((0, 3)), np.zeros((0, 3)), grid, 2, x, r=T + 0.5, T=T, M=M)
    g = rm.graph()
    assert g.row_ptr[1] - g.row_ptr[0] == 1 and int(g.dst[0]) == 1
    # checkpoints left of x = 0.5: 0.31 + m T / 16 < 0.5
    left = sum(1 for m in range(1, M + 1) if 0.31 + m * T / M < 0.5)
    right = M - left
    S = inc * (9 * left - 7 * right)
    h, peak = 0, 0
    for m in range(M):
        h = max(0, h + inc * (9 if m < left else -7))
        peak = max(peak, h)
    assert (int(g.S[0]), int(g.C[0]), int(g.Cmax[0])) == (S, h, peak)
    # the increment does not depend on the connection's energy or length
    ev = rm.edge_eval(0, 1)
    np.testing.assert_array_equal(ev["d"], [inc * (9 if m < left else -7) for m in range(M)])
