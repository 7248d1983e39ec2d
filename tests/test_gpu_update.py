"""Online roadmap update (boxes added, grid replaced) against the oracle's
construction from the same nodes on the updated scene: edges, transfers, peaks,
reverse CSR, and the search and certification that run on the result."""
import numpy as np
import pytest

import scenegen
from _gpu import assert_reverse_is_transpose, assert_same_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def _added_boxes(name, seed, k):
    rng = np.random.default_rng(seed + 77)
    dp = 2 if name == "2d" else 3
    lo = np.zeros((k, 3), np.float32); hi = np.zeros((k, 3), np.float32)
    c = rng.uniform(0.2, 0.8, (k, dp)); s = rng.uniform(0.04, 0.12, (k, dp))
    lo[:, :dp] = c - s / 2; hi[:, :dp] = c + s / 2
    if dp == 2:
        hi[:, 2] = 1.0
    return lo, hi


@pytest.mark.parametrize("name,seed,n,r,k,new_grid", [
    ("2d", 1, 900, None, 3, True),
    ("2d", 6, 700, 0.2, 2, False),     # rows beyond 128 edges
    ("3d", 2, 1500, None, 4, True),
    ("6d", 1, 2000, 18.0, 3, True),
    ("6d", 4, 2000, 18.0, 0, True),    # grid only
    ("6d", 5, 2000, 18.0, 5, False),   # boxes only
])
def test_update_equals_construction_from_the_same_nodes(mp, orc, name, seed, n, r, k, new_grid):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rr = sc.cfg.r if r is None else r
    rg = mp.build_roadmap_for_scene(sc, n=n, r=rr)
    x = orc.build_roadmap(sc, n=n, r=rr).graph().x          # the oracle's own nodes
    lo, hi = _added_boxes(name, seed, k)
    grid = scenegen.make_scene(name, seed + 100).grid if new_grid else None
    E0 = rg.E
    rg.update(lo if k else None, hi if k else None, grid)
    all_lo = np.concatenate([sc.box_lo, lo]); all_hi = np.concatenate([sc.box_hi, hi])
    ro = orc.build_roadmap_from_points(sc.cfg.dim_kind, all_lo, all_hi, sc.grid if grid is None else grid,
                                       sc.cfg.grid_G, x, rr, T=sc.cfg.T_edge, M=sc.cfg.M)
    g = ro.graph()
    assert_same_graph(rg.export(), g)
    np.testing.assert_array_equal(np.stack(rg.peaks()), np.stack([g.Smax, g.Cmax]))
    assert_reverse_is_transpose(rg)
    if k:
        assert rg.E < E0
    # search and certification on the updated roadmap
    beta = orc.beta_percentile(ro)
    ws = mp.Workspace(rg.V, front_cap=2048, max_plans=1 << 22)
    a = mp.search(ws, rg, beta, lam=0.5)
    b = orc.explore(ro, beta, orc.group_width(0.5, rr))
    assert (a.status, a.cost, a.h) == (b.status, b.cost, b.h)
    if b.status == 0:
        np.testing.assert_array_equal(a.path, b.path)
        m = (512, sc.mc_seed, 3, sc.delta_fx, sc.sigma_fx, sc.shift)
        assert mp.certify(rg, a.path, *m) == orc.certify(ro, b.path, *m)


def _local_grid(sc, seed, side=0.3):
    """The scene's grid with the levels of the cells inside one cube of the given
    side replaced by those of another seeded grid (new features mapped there)."""
    rng = np.random.default_rng(seed + 991)
    G = sc.cfg.grid_G
    g = sc.grid.copy()
    other = scenegen.make_scene(sc.cfg, seed + 200).grid
    dp = 2 if sc.cfg.dim_kind == 2 else 3
    lo = rng.uniform(0.0, 1.0 - side, dp)
    idx = [np.arange(G)] * dp
    cen = (np.arange(G) + 0.5) / G
    inside = [(cen >= lo[i]) & (cen < lo[i] + side) for i in range(dp)]
    if dp == 2:
        m = inside[1][:, None] & inside[0][None, :]
    else:
        m = inside[2][:, None, None] & inside[1][None, :, None] & inside[0][None, None, :]
    g.reshape(m.shape)[m] = other.reshape(m.shape)[m]
    return g


@pytest.mark.parametrize("name,seed,n,r,k,mode", [
    ("2d", 3, 900, None, 3, "local"),
    ("3d", 4, 1500, None, 2, "local"),
    ("6d", 2, 2000, 18.0, 3, "local"),
    ("6d", 6, 2000, 18.0, 0, "local"),    # grid only, a local change
    ("6d", 7, 2000, 18.0, 2, "same"),     # the same grid again: no transfer changes
    ("3d", 8, 1500, None, 0, "same"),
])
def test_update_skips_edges_away_from_the_changes(mp, orc, name, seed, n, r, k, mode):
    """The update re-tests only the edges whose checkpoint bound meets an added box
    and re-transfers only those whose bound meets a changed cell; with a local
    grid change (or the same grid again) the result must still equal the
    construction from the same nodes on the updated scene."""
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rr = sc.cfg.r if r is None else r
    rg = mp.build_roadmap_for_scene(sc, n=n, r=rr)
    x = orc.build_roadmap(sc, n=n, r=rr).graph().x
    lo, hi = _added_boxes(name, seed, k)
    grid = _local_grid(sc, seed) if mode == "local" else sc.grid.copy()
    if mode == "local":
        assert (grid != sc.grid).any()
    before = rg.export()
    rg.update(lo if k else None, hi if k else None, grid)
    ro = orc.build_roadmap_from_points(sc.cfg.dim_kind, np.concatenate([sc.box_lo, lo]),
                                       np.concatenate([sc.box_hi, hi]), grid, sc.cfg.grid_G, x, rr,
                                       T=sc.cfg.T_edge, M=sc.cfg.M)
    g = ro.graph()
    assert_same_graph(rg.export(), g)
    np.testing.assert_array_equal(np.stack(rg.peaks()), np.stack([g.Smax, g.Cmax]))
    assert_reverse_is_transpose(rg)
    if mode == "same" and k == 0:
        after = rg.export()
        for key in ("row_ptr", "dst", "cost_q", "S", "C"):
            np.testing.assert_array_equal(after[key], before[key])


def test_update_with_device_arrays_and_repeated(mp, orc):
    import torch
    sc = scenegen.make_scene("3d", 6, query_id=6)
    rg = mp.build_roadmap_for_scene(sc, n=1200)
    x = orc.build_roadmap(sc, n=1200).graph().x
    lo1, hi1 = _added_boxes("3d", 1, 2)
    lo2, hi2 = _added_boxes("3d", 2, 3)
    grid = scenegen.make_scene("3d", 60).grid
    rg.update(torch.from_numpy(lo1).cuda(), torch.from_numpy(hi1).cuda(), torch.from_numpy(grid).cuda())
    rg.update(lo2, hi2)
    ro = orc.build_roadmap_from_points(3, np.concatenate([sc.box_lo, lo1, lo2]),
                                       np.concatenate([sc.box_hi, hi1, hi2]), grid, sc.cfg.grid_G, x, sc.cfg.r)
    assert_same_graph(rg.export(), ro.graph())
    assert_reverse_is_transpose(rg)


def test_batched_update_equals_construction_from_the_same_nodes(mp, orc):
    """mpap_roadmap_update_batch: mixed dimensions, boxes only, grid only and both,
    in one call."""
    cases = [("2d", 1, 900, None, 3, True), ("3d", 2, 1500, None, 4, False), ("6d", 1, 2000, 18.0, 3, True),
             ("6d", 4, 2000, 18.0, 0, True), ("2d", 6, 700, 0.2, 2, False)]
    rms, adds_lo, adds_hi, grids, want = [], [], [], [], []
    for name, seed, n, r, k, new_grid in cases:
        sc = scenegen.make_scene(name, seed, query_id=seed)
        rr = sc.cfg.r if r is None else r
        rms.append(mp.build_roadmap_for_scene(sc, n=n, r=rr))
        x = orc.build_roadmap(sc, n=n, r=rr).graph().x
        lo, hi = _added_boxes(name, seed, k)
        grid = scenegen.make_scene(name, seed + 100).grid if new_grid else None
        adds_lo.append(lo); adds_hi.append(hi); grids.append(grid)
        ro = orc.build_roadmap_from_points(sc.cfg.dim_kind, np.concatenate([sc.box_lo, lo]),
                                           np.concatenate([sc.box_hi, hi]), sc.grid if grid is None else grid,
                                           sc.cfg.grid_G, x, rr, T=sc.cfg.T_edge, M=sc.cfg.M)
        want.append(ro.graph())
    mp.roadmap_update_batch(rms, adds_lo, adds_hi, grids)
    for rg, g in zip(rms, want):
        assert_same_graph(rg.export(), g)
        np.testing.assert_array_equal(np.stack(rg.peaks()), np.stack([g.Smax, g.Cmax]))
        assert_reverse_is_transpose(rg)
