"""The grid-wide merge of huge nodes (one node's front and candidates merged by
every warp of the persistent wavefront kernel: members bucketed by cost, an
exclusive prefix minimum of h over the buckets, exact resolution inside each
bucket, an exclusive prefix sum placing the survivors) against the oracle and
against the one-warp merge.  With the threshold lowered to 33 entries nearly
every merge of the parity cases runs grid-wide; on 2D queries whose single
fronts pass 10^4 plans a threshold of 8192 takes it, and the results
equal those with the grid-wide merge switched off.  Fronts, solutions and
counters bit-exact."""
import numpy as np
import pytest

import scenegen
from _gpu import BIG, assert_same_search
from _search_ref import random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    m.tuning_clear()
    yield m
    m.tuning_clear()


def _threshold(mp, V, thr):
    for d in (0, 2, 3, 6):
        mp.tuning_set(d, V, grid_merge_from=thr)


@pytest.fixture(scope="module")
def ws(mp):
    return mp.Workspace(40000, front_cap=2048, max_plans=1 << 23)


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_grid_merge(mp, orc, ws, seed):
    rng = np.random.default_rng(900 + seed)
    V = int(rng.integers(3, 40))
    g = random_graph(rng, V, p_edge=float(rng.uniform(0.2, 0.6)), cmax=int(rng.integers(1, 9)),
                     dmax=int(rng.integers(1, 6)))
    ro = orc.roadmap_from_csr(*g)
    rg = mp.roadmap_from_csr(*g)
    _threshold(mp, rg.V, 33)
    for beta in (int(rng.integers(0, 12)), BIG):
        for lam in (1, 7, 1000):
            for stop in (True, False):
                a = orc.explore(ro, beta, lam, goal_termination=stop)
                b = mp.search(ws, rg, beta, group_width_q=lam, goal_stop=stop)
                assert_same_search(b, a, ws)
    mp.tuning_clear()


@pytest.mark.parametrize("name,seed,n,beta_mode", [
    ("2d", 1, 1000, "pct"), ("2d", 3, 1000, "inf"), ("2d", 6, 1500, "pct"), ("3d", 1, 2500, "pct"),
    ("6d", 1, 3000, "pct"), ("6d", 2, 3000, "inf"),
])
def test_scenes_grid_merge(mp, orc, ws, name, seed, n, beta_mode):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro = orc.build_roadmap(sc, n=n, r=r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    beta = {"pct": orc.beta_percentile(ro), "inf": BIG}[beta_mode]
    lam_q = orc.group_width(0.5, r)
    _threshold(mp, rg.V, 33)
    for stop in (True, False):
        a = orc.explore(ro, beta, lam_q, goal_termination=stop)
        b = mp.search(ws, rg, beta, lam=0.5, goal_stop=stop)
        assert_same_search(b, a, ws)
    mp.tuning_clear()


def test_mixed_batch_grid_merge(mp, orc):
    batch = []
    for d, n, s in scenegen.batch_specs(12, seed=21, n_lo=800, n_hi=3000):
        cfg = scenegen.scaled_config(d, n)
        batch.append((cfg, scenegen.make_scene(cfg, s, query_id=s)))
    rms = mp.build_roadmaps([mp.scene_spec(sc) for _, sc in batch])
    ros = [orc.build_roadmap(sc) for _, sc in batch]
    betas = [orc.beta_percentile(ro) for ro in ros]
    ws = mp.Workspace(sum(rg.V for rg in rms), front_cap=2048, max_plans=1 << 24)
    _threshold(mp, max(rg.V for rg in rms), 33)
    res = mp.search_batch(ws, rms, [mp.make_query(b, 0.5) for b in betas])
    for i, ((cfg, sc), ro, b) in enumerate(zip(batch, ros, betas)):
        assert_same_search(res[i], orc.explore(ro, b, orc.group_width(0.5, cfg.r)), ws, index=i)
    mp.tuning_clear()


# 2D queries of the mixed workload whose largest single front passes 10^4 plans
LARGE_2D = [(2485, 879894124), (2057, 909177283)]


@pytest.mark.parametrize("n,seed", LARGE_2D)
def test_large_fronts_grid_vs_warp_merge(mp, orc, n, seed):
    cfg = scenegen.scaled_config(scenegen.DIM_2D, n)
    sc = scenegen.make_scene(cfg, seed, query_id=seed)
    beta = orc.beta_percentile(orc.build_roadmap(sc))
    rg = mp.build_roadmaps([mp.scene_spec(sc)])[0]
    ws = mp.Workspace(rg.V, front_cap=16384, max_plans=1 << 26)
    out = []
    for thr in (8192, 1 << 30):
        _threshold(mp, rg.V, thr)
        r = mp.search(ws, rg, beta, lam=scenegen.LAMBDA)
        out.append((r, ws.fronts(0)))
    (a, fa), (b, fb) = out
    assert a.status == 0
    assert (a.status, a.cost, a.h, a.wavefronts, a.expansions, a.plans) == \
        (b.status, b.cost, b.h, b.wavefronts, b.expansions, b.plans)
    np.testing.assert_array_equal(a.path, b.path)
    for x, y in zip(fa, fb):
        np.testing.assert_array_equal(x, y)
    assert np.diff(fa[0][:rg.V + 1].astype(np.int64)).max() > 8192    # the grid-wide merge ran
    mp.tuning_clear()
