"""GPU visible-feature perception levels against the oracle, bit for bit: range,
horizontal field of view per yaw heading and occlusion by boxes, for 2D and 3D
grids, host and device arrays; and a roadmap on the all-direction table."""
import numpy as np
import pytest

import scenegen
from _gpu import BIG, assert_same_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.mark.parametrize("name,seed,G,Y,half_deg,rng,F", [
    ("2d", 1, 64, 8, 45.0, 0.5, 256),
    ("2d", 2, 32, 3, 60.0, 0.3, 700),      # more features than one shared-memory tile
    ("3d", 2, 16, 8, 45.0, 0.5, 256),
    ("6d", 3, 32, 1, None, 2.0, 256),      # the all-direction grid of a 6D scene
    ("3d", 5, 8, 5, 80.0, 1.0, 1),
])
def test_levels_match_oracle(mp, orc, name, seed, G, Y, half_deg, rng, F):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    f = scenegen.feature_points(sc, F)
    heads = scenegen.yaw_headings(Y)
    ch = -2.0 if half_deg is None else float(np.float32(np.cos(np.radians(half_deg))))
    a = mp.feature_levels(sc.cfg.dim_kind, sc.box_lo, sc.box_hi, f, G, heads, ch, rng, K=24)
    b = orc.feature_levels(2 if sc.cfg.dim_kind == 2 else 3, sc.box_lo, sc.box_hi, f, G, heads, ch, rng, 24)
    assert a.shape == b.shape == (Y, G ** (2 if sc.cfg.dim_kind == 2 else 3))
    np.testing.assert_array_equal(a, b)
    assert len(np.unique(a)) > 1 or F == 1


def test_device_arrays_and_edge_cases(mp, orc):
    import torch
    sc = scenegen.make_scene("3d", 7, query_id=7)
    f = scenegen.feature_points(sc, 300)
    heads = scenegen.yaw_headings(4)
    host = mp.feature_levels(3, sc.box_lo, sc.box_hi, f, 16, heads, 0.7, 0.6)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dev = mp.feature_levels(3, t(sc.box_lo), t(sc.box_hi), t(f), 16, t(heads), 0.7, 0.6)
    np.testing.assert_array_equal(dev.cpu().numpy(), host)
    # no boxes, no features
    nob = np.zeros((0, 3), np.float32)
    np.testing.assert_array_equal(mp.feature_levels(2, nob, nob, f[:0], 4), np.zeros((1, 16), np.uint8))
    np.testing.assert_array_equal(mp.feature_levels(2, nob, nob, f[:30], 4, K=7), np.full((1, 16), 7, np.uint8))
    # G = 1 and range 0
    np.testing.assert_array_equal(mp.feature_levels(3, sc.box_lo, sc.box_hi, f, 1, range_=0.0),
                                  orc.feature_levels(3, sc.box_lo, sc.box_hi, f, 1, range_=0.0))


def test_roadmap_on_the_all_direction_table(mp, orc):
    """The all-direction table serves as a scene's quality grid: roadmap and
    search on it equal the oracle's."""
    sc = scenegen.make_scene("3d", 3, query_id=3)
    f = scenegen.feature_points(sc, 256)
    sc.grid = mp.feature_levels(3, sc.box_lo, sc.box_hi, f, sc.cfg.grid_G, range_=0.6)[0].copy()
    np.testing.assert_array_equal(sc.grid, orc.feature_levels(3, sc.box_lo, sc.box_hi, f, sc.cfg.grid_G,
                                                              range_=0.6)[0])
    rg = mp.build_roadmap_for_scene(sc, n=1500)
    ro = orc.build_roadmap(sc, n=1500)
    assert_same_graph(rg.export(), ro.graph())
    ws = mp.Workspace(rg.V, front_cap=1024, max_plans=1 << 22)
    beta = orc.beta_percentile(ro)
    a = mp.search(ws, rg, beta, lam=0.5)
    b = orc.explore(ro, beta, orc.group_width(0.5, sc.cfg.r))
    assert (a.status, a.cost, a.h) == (b.status, b.cost, b.h)
    np.testing.assert_array_equal(a.path, b.path)
