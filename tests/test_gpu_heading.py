"""The camera-heading form of the perception heuristic (Sec. 4.1: features in the
field of view of a single-integrator yaw) on the GPU against the oracle: node
yaws, every CSR array with the transfers and their peaks, search results,
certification counts and plan features -- bit-exact."""
import numpy as np
import pytest

import scenegen
from _gpu import BIG, assert_same_graph, assert_same_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def _tables(sc, Y, seed):
    """Y level tables of the scene's grid size, one seeded quality field each."""
    return np.stack([scenegen.make_scene(sc.cfg, seed * 100 + k).grid for k in range(Y)])


@pytest.mark.parametrize("name,seed,n,r,Y", [("2d", 1, 800, None, 8), ("3d", 2, 1500, None, 8),
                                             ("6d", 3, 2000, 18.0, 8), ("6d", 4, 1500, 18.0, 5)])
def test_heading_roadmap_search_and_certification_match_oracle(mp, orc, name, seed, n, r, Y):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rr = sc.cfg.r if r is None else r
    head = _tables(sc, Y, seed)
    ro = orc.build_roadmap(sc, n=n, r=rr, heading=head)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=rr, heading=head)
    np.testing.assert_array_equal(rg.yaw(), ro.yaw())
    g = ro.graph()
    assert_same_graph(rg.export(), g)
    np.testing.assert_array_equal(np.stack(rg.peaks()), np.stack([g.Smax, g.Cmax]))
    # the heading form changes the transfers against the grid form
    plain = orc.build_roadmap(sc, n=n, r=rr).graph()
    assert not np.array_equal(plain.S, g.S)
    beta = orc.beta_percentile(ro)
    ws = mp.Workspace(rg.V, front_cap=2048, max_plans=1 << 22)
    a = mp.search(ws, rg, beta, lam=0.5)
    b = orc.explore(ro, beta, orc.group_width(0.5, rr))
    assert_same_search(a, b, ws)
    if b.status == 0:
        m = (1024, sc.mc_seed, 2, sc.delta_fx, sc.sigma_fx * 3, sc.shift)
        assert mp.certify(rg, a.path, *m) == orc.certify(ro, b.path, *m)
        np.testing.assert_array_equal(mp.plan_features(rg, [a.path]), orc.plan_features(ro, [b.path]))


def test_one_table_equal_to_the_grid_is_the_grid_form(mp):
    sc = scenegen.make_scene("6d", 7, query_id=7)
    base = mp.build_roadmap_for_scene(sc, n=1500, r=18.0).export()
    one = mp.build_roadmap_for_scene(sc, n=1500, r=18.0, heading=sc.grid[None, :]).export()
    for k in ("row_ptr", "dst", "cost_q", "S", "C"):
        np.testing.assert_array_equal(base[k], one[k])


def test_batched_build_mixes_heading_and_grid_forms(mp, orc):
    scs = [scenegen.make_scene("6d", 8, query_id=8), scenegen.make_scene("3d", 9, query_id=9),
           scenegen.make_scene("6d", 10, query_id=10)]
    heads = [_tables(scs[0], 8, 8), None, _tables(scs[2], 6, 10)]
    ns, rs = [1500, 1200, 1800], [18.0, None, 18.0]
    specs = [mp.scene_spec(sc, n=n, r=(sc.cfg.r if r is None else r), heading=h)
             for sc, n, r, h in zip(scs, ns, rs, heads)]
    rms = mp.build_roadmaps(specs)
    for sc, n, r, h, rg in zip(scs, ns, rs, heads, rms):
        ro = orc.build_roadmap(sc, n=n, r=(sc.cfg.r if r is None else r), heading=h)
        assert_same_graph(rg.export(), ro.graph())
        np.testing.assert_array_equal(rg.yaw(), ro.yaw())


def test_update_of_a_heading_roadmap(mp, orc):
    """Boxes can be added (the result equals construction from the same nodes and
    yaws); replacing the levels is refused."""
    sc = scenegen.make_scene("6d", 11, query_id=11)
    head = _tables(sc, 8, 11)
    rg = mp.build_roadmap_for_scene(sc, n=1500, r=18.0, heading=head)
    x = orc.build_roadmap(sc, n=1500, r=18.0, heading=head).graph().x
    yaw = rg.yaw()
    lo = np.array([[0.4, 0.4, 0.4], [0.6, 0.2, 0.5]], np.float32)
    hi = lo + np.float32(0.1)
    rg.update(lo, hi)
    ro = orc.build_roadmap_from_points(6, np.concatenate([sc.box_lo, lo]), np.concatenate([sc.box_hi, hi]),
                                       sc.grid, sc.cfg.grid_G, x, 18.0, T=sc.cfg.T_edge, M=sc.cfg.M,
                                       heading=head, yaw=yaw)
    assert_same_graph(rg.export(), ro.graph())
    with pytest.raises(mp.MpapError) as e:
        rg.update(None, None, sc.grid)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
