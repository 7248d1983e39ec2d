"""mpap_certify_noalloc: certification for callers that cannot allocate device
memory while running (e.g. a planner in a real-time control loop with a fixed
memory budget).  Its scratch lives in a fixed device array inside the library;
the results must equal those of the allocating mpap_certify, call after call,
since every call reuses (and must reset) the same array."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu

BIG = 1 << 62


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def _plan(mp, name, seed, n, r):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    ws = mp.Workspace(rg.V, front_cap=1024, max_plans=1 << 22)
    res = mp.search(ws, rg, BIG, lam=0.5)
    assert res.status == 0 and len(res.path) >= 2
    return sc, rg, res.path


def test_noalloc_matches_allocating_certify_on_consecutive_calls(mp):
    jobs = [_plan(mp, "2d", 1, 800, None), _plan(mp, "6d", 3, 2000, 18.0)]
    # two calls in a row on different plans, scenes and noise scales: the shared
    # array keeps the previous call's contents, the results must not depend on it
    for (sc, rg, path), rollouts, scale, call_id in zip(jobs, (1024, 4096), (3, 10), (0, 7)):
        sig = sc.sigma_fx * scale
        want = mp.certify(rg, path, rollouts, sc.mc_seed, call_id, sc.delta_fx, sig, sc.shift)
        got = mp.certify_noalloc(rg, path, rollouts, sc.mc_seed, call_id, sc.delta_fx, sig, sc.shift)
        assert got == want
        assert got["rollouts"] == rollouts and 0 < got["hits_any"] <= rollouts
    # and once more on the first plan after the second
    sc, rg, path = jobs[0]
    want = mp.certify(rg, path, 333, sc.mc_seed, 1, sc.delta_fx, sc.sigma_fx * 3, sc.shift)
    got = mp.certify_noalloc(rg, path, 333, sc.mc_seed, 1, sc.delta_fx, sc.sigma_fx * 3, sc.shift)
    assert got == want


def test_noalloc_rejects_inputs_beyond_its_fixed_size(mp):
    sc, rg, path = _plan(mp, "2d", 2, 500, None)
    too_long = np.resize(path, 5000).astype(np.uint32)   # more than 4096 nodes
    with pytest.raises(mp.MpapError) as e:
        mp.certify_noalloc(rg, too_long, 16, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx, sc.shift)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
    assert "4096" in str(e.value)


def test_noalloc_rejects_too_many_checkpoints(mp):
    """A plan within the node limit whose edges hold more checkpoints than the
    fixed array has room for: (3000 - 1) edges x 32 sub-steps > 65536.  (The
    level-table limit, K + 1 <= 256, always holds: a roadmap's K is at most
    255.)"""
    sc = scenegen.make_scene("2d", 2, query_id=2)
    rg = mp.build_roadmap_for_scene(sc, n=500, M=32)
    ws = mp.Workspace(rg.V, front_cap=1024, max_plans=1 << 22)
    res = mp.search(ws, rg, BIG, lam=0.5)
    assert res.status == 0
    plan = np.resize(res.path, 3000).astype(np.uint32)
    with pytest.raises(mp.MpapError) as e:
        mp.certify_noalloc(rg, plan, 16, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx, sc.shift)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
    assert "65536" in str(e.value)
