"""Pins for the oracle's camera-heading form of the perception heuristic (Sec.
4.1: features count only in the field of view of the yaw, a single-integrator
state): node yaws drawn from Philox, yaw interpolated along each edge the short
way round, the level table of the nearest of Y headings at every checkpoint.
CPU only."""
import math

import numpy as np
import pytest

import scenegen

K, NF = 24, 12


def _graph_equal(a, b):
    ga, gb = a.graph(), b.graph()
    for k in ("row_ptr", "dst", "cost_q", "S", "C", "Smax", "Cmax"):
        np.testing.assert_array_equal(getattr(ga, k), getattr(gb, k))


@pytest.mark.parametrize("name,n,r", [("2d", 400, None), ("3d", 600, None), ("6d", 700, 18.0)])
def test_one_table_or_identical_tables_reduce_to_the_grid_form(orc, name, n, r):
    sc = scenegen.make_scene(name, 3, query_id=3)
    rr = sc.cfg.r if r is None else r
    base = orc.build_roadmap(sc, n=n, r=rr)
    for Y in (1, 8):
        hd = orc.build_roadmap(sc, n=n, r=rr, heading=np.stack([sc.grid] * Y))
        _graph_equal(base, hd)
    # the certification reads the same levels
    g = base.graph()
    path = np.array([0, g.dst[g.row_ptr[0]]], np.uint32)
    hd = orc.build_roadmap(sc, n=n, r=rr, heading=np.stack([sc.grid] * 8))
    m = (512, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx * 8, sc.shift)
    assert orc.certify(base, path, *m) == orc.certify(hd, path, *m)


def test_node_yaws_are_uniform_on_the_circle(orc):
    sc = scenegen.make_scene("6d", 5, query_id=5)
    rm = orc.build_roadmap(sc, n=4000, r=12.0, heading=np.stack([sc.grid] * 4))
    yaw = rm.yaw().astype(np.float64)
    assert (yaw >= -math.pi).all() and (yaw < math.pi).all()
    counts = np.histogram(yaw, bins=16, range=(-math.pi, math.pi))[0]
    expected = len(yaw) / 16
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 40.0            # 15 degrees of freedom: p ~ 5e-4
    other = orc.build_roadmap(scenegen.make_scene("6d", 6, query_id=6), n=4000, r=12.0,
                              heading=np.stack([sc.grid] * 4)).yaw()
    assert not np.array_equal(yaw, other)


def _two_nodes(orc, yaw_a, yaw_b, tables, dim=2):
    """One 2D edge from (0.3, 0.3) to (0.36, 0.3) (the rest of the graph is the
    reverse edge), constant levels per table."""
    x = np.zeros((6, 2), np.float32)
    x[0] = [0.3, 0.36]; x[1] = [0.3, 0.3]
    G = 2
    head = np.stack([np.full(G * G, lv, np.uint8) for lv in tables])
    rm = orc.build_roadmap_from_points(dim, np.zeros((0, 3)), np.zeros((0, 3)), head[0], G, x, r=0.1,
                                       M=16, goal_radius=0.001, heading=head,
                                       yaw=np.array([yaw_a, yaw_b], np.float32))
    g = rm.graph()
    e = int(np.nonzero(g.dst[g.row_ptr[0]:g.row_ptr[1]] == 1)[0][0]) + int(g.row_ptr[0])
    return int(g.cost_q[e]), int(g.S[e]), int(g.C[e])


def test_heading_switch_along_an_edge_by_hand(orc):
    """Y = 4 headings (0, pi/2, pi, -pi/2).  Yaw 0 -> 1 rad: checkpoint m has yaw
    m/16 rad, nearest heading index round(m/16 * 4 / (2 pi)): 0 for m <= 12
    (0.4775 at m = 12) and 1 for m >= 13 (0.5173).  Table 0 has level 4, table 1
    level 20: 12 steps of n_f - 4 = 8 and 4 steps of n_f - 20 = -8, times the
    edge's quantised length."""
    cq, S, C = _two_nodes(orc, 0.0, 1.0, [4, 20, 0, 0])
    d = [cq * 8] * 12 + [cq * -8] * 4
    assert S == sum(d)
    h = 0
    for dm in d:
        h = max(0, h + dm)
    assert C == h == cq * 8 * 8
    # constant yaw: every checkpoint in one table
    for yaw, lv in ((0.0, 4), (math.pi / 2, 20), (-math.pi / 2, 7)):
        cq2, S2, C2 = _two_nodes(orc, yaw, yaw, [4, 20, 11, 7])
        assert S2 == 16 * cq2 * (NF - lv) and cq2 == cq


def test_yaw_wraps_the_short_way(orc):
    """Yaw 3.0 -> -3.0 rad turns +0.283 rad through pi (heading index 2 all the
    way); turning -6.0 rad instead would sweep through headings 1, 0 and 3."""
    cq, S, C = _two_nodes(orc, 3.0, -3.0, [0, 0, 18, 0])
    assert S == 16 * cq * (NF - 18)
    assert C == 0
