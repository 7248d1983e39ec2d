"""GPU Monte Carlo certification vs the oracle: hit counts bit-exact."""
import numpy as np
import pytest

import scenegen
from _gpu import BIG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def _plan(orc, sc, n, r):
    ro = orc.build_roadmap(sc, n=n, r=r)
    res = orc.explore(ro, BIG, orc.group_width(0.5, r))
    assert res.status == 0
    return ro, res.path


@pytest.mark.parametrize("name,seed,n,R", [("2d", 1, 1000, 1024), ("3d", 2, 2000, 1024),
                                           ("6d", 3, 3000, 4096), ("2d", 9, 500, 333)])
def test_certify_matches_oracle(mp, orc, name, seed, n, R):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro, path = _plan(orc, sc, n, r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    for call_id, scale in ((0, 1), (3, 4)):
        sig = sc.sigma_fx * scale
        a = orc.certify(ro, path, R, sc.mc_seed, call_id, sc.delta_fx, sig, sc.shift)
        b = mp.certify(rg, path, R, sc.mc_seed, call_id, sc.delta_fx, sig, sc.shift)
        assert a == b
        assert 0 <= b["hits_any"] <= R


def test_certify_batch_and_edge_cases(mp, orc):
    jobs = []
    for name, seed, n in (("2d", 1, 800), ("3d", 2, 1500), ("6d", 3, 2500)):
        sc = scenegen.make_scene(name, seed, query_id=seed)
        r = sc.cfg.r if name != "6d" else 18.0
        ro, path = _plan(orc, sc, n, r)
        rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
        jobs.append((sc, ro, rg, path))
    mcs = [(777, sc.mc_seed, 5, sc.delta_fx, sc.sigma_fx * 2, sc.shift) for sc, _, _, _ in jobs]
    out = mp.certify_batch([j[2] for j in jobs], [j[3] for j in jobs], mcs)
    for (sc, ro, rg, path), m, o in zip(jobs, mcs, out):
        assert o == orc.certify(ro, path, *m)
    # single-node path: no steps, no failures; zero rollouts
    sc, ro, rg, path = jobs[0]
    assert mp.certify(rg, path[:1], 100, 1, 0, sc.delta_fx, sc.sigma_fx, sc.shift)["hits_any"] == 0
    assert mp.certify(rg, path, 0, 1, 0, sc.delta_fx, sc.sigma_fx, sc.shift)["rollouts"] == 0


@pytest.mark.parametrize("name,nb,seed,n", [("3d", 32, 4, 1500), ("3d", 40, 4, 1500), ("6d", 33, 5, 2500),
                                            ("2d", 36, 6, 800)])
def test_certify_around_the_box_prefilter_limit(mp, orc, name, nb, seed, n):
    """Rollouts of scenes with at most 32 boxes take the point-in-box prefilter
    table, larger scenes the pass over every box: the hit counts are the
    oracle's either way, with collisions among them."""
    sc = scenegen.make_scene(scenegen.config(name, nb=nb), seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro, path = _plan(orc, sc, n, r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    for call_id, scale in ((1, 1), (1, 4)):
        sig = sc.sigma_fx * scale
        a = orc.certify(ro, path, 1024, sc.mc_seed, call_id, sc.delta_fx, sig, sc.shift)
        b = mp.certify(rg, path, 1024, sc.mc_seed, call_id, sc.delta_fx, sig, sc.shift)
        assert a == b
    assert b["hits_coll"] > 0
