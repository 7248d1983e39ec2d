"""Batched queries (many roadmaps of mixed dimension and size in one build, one
lock-step search and one certification launch) against the oracle, and the
launch-shape autotuner: results must not depend on the tuned shapes."""
import numpy as np
import pytest

import scenegen
from _gpu import assert_same_graph, assert_same_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    m.tuning_clear()
    yield m
    m.tuning_clear()


def _mixed(count, seed, n_lo, n_hi):
    out = []
    for d, n, s in scenegen.batch_specs(count, seed=seed, n_lo=n_lo, n_hi=n_hi):
        cfg = scenegen.scaled_config(d, n)
        out.append((cfg, scenegen.make_scene(cfg, s, query_id=s)))
    return out


def test_mixed_batch_matches_oracle(mp, orc):
    batch = _mixed(15, 11, 800, 4000)
    assert {c.dim_kind for c, _ in batch} == {2, 3, 6}
    rms = mp.build_roadmaps([mp.scene_spec(sc) for _, sc in batch])
    ros = [orc.build_roadmap(sc) for _, sc in batch]
    for rg, ro in zip(rms, ros):
        assert_same_graph(rg.export(), ro.graph())
    betas = [orc.beta_percentile(ro) for ro in ros]
    qs = [mp.make_query(b, 0.5) for b in betas]
    ws = mp.Workspace(sum(rg.V for rg in rms), front_cap=2048, max_plans=1 << 24)
    res = mp.search_batch(ws, rms, qs)
    solved = []
    for i, ((cfg, sc), ro, b) in enumerate(zip(batch, ros, betas)):
        a = orc.explore(ro, b, orc.group_width(0.5, cfg.r))
        assert_same_search(res[i], a, ws, index=i)
        if a.status == 0:
            solved.append(i)
    assert len(solved) >= 10
    mcs = [(256, batch[i][1].mc_seed, 3, batch[i][1].delta_fx, batch[i][1].sigma_fx, batch[i][1].shift)
           for i in solved]
    got = mp.certify_batch([rms[i] for i in solved], [res[i].path for i in solved], mcs)
    for i, m, g in zip(solved, mcs, got):
        assert g == orc.certify(ros[i], res[i].path, *m)


def test_autotune_search_keeps_results(mp):
    batch = _mixed(9, 5, 1000, 3000)
    rms = mp.build_roadmaps([mp.scene_spec(sc) for _, sc in batch])
    qs = [mp.make_query(1 << 62, 0.5) for _ in batch]
    ws = mp.Workspace(sum(rg.V for rg in rms), front_cap=2048, max_plans=1 << 24)
    mp.tuning_clear()
    ref = mp.search_batch(ws, rms, qs)
    ref_fronts = [ws.fronts(i) for i in range(len(rms))]
    tun, ms = mp.autotune_search(ws, rms, qs, reps=1)
    assert ms > 0 and tun["front_cap"] >= 16 and (tun["front_cap"] & (tun["front_cap"] - 1)) == 0
    Vmax = max(rg.V for rg in rms)
    assert mp.tuning_get(0, Vmax) == tun            # stored under the mixed-batch key
    for bps, lf in [(1, 1), (32, 2), (64, 64), (2, 33), (tun["wave_blocks_per_sm"], tun["plan_lanes_from"])]:
        mp.tuning_set(0, Vmax, wave_blocks_per_sm=bps, plan_lanes_from=lf)
        got = mp.search_batch(ws, rms, qs)
        for i in range(len(rms)):
            assert (got[i].status, got[i].cost, got[i].h, got[i].expansions, got[i].wavefronts) == \
                (ref[i].status, ref[i].cost, ref[i].h, ref[i].expansions, ref[i].wavefronts)
            np.testing.assert_array_equal(got[i].path, ref[i].path)
            for a, b in zip(ws.fronts(i), ref_fronts[i]):
                np.testing.assert_array_equal(a, b)
    mp.tuning_clear()


def test_autotune_build_keeps_roadmaps(mp):
    batch = _mixed(6, 3, 1000, 2500)
    specs = [mp.scene_spec(sc) for _, sc in batch]
    mp.tuning_clear()
    ref = [rg.export() for rg in mp.build_roadmaps(specs)]
    tun, ms, rms = mp.autotune_build(specs, reps=1)
    assert tun["edge_warps"] in (4, 8) and ms > 0
    dims = {c.dim_kind for c, _ in batch}
    assert {d for d, _, _ in mp.tuning_export()} == dims
    for w in (4, 8):
        for d in dims:
            vmax = max(c.n + 2 for c, _ in batch if c.dim_kind == d)
            mp.tuning_set(d, vmax, edge_warps=w)
        rms = mp.build_roadmaps(specs, rms=rms)
        for rg, want in zip(rms, ref):
            got = rg.export()
            for k in want:
                np.testing.assert_array_equal(got[k], want[k])
    mp.tuning_clear()
