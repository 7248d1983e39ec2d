"""GPU wavefront search (Alg. 3) vs the oracle: final Pareto fronts of every node,
solution cost, heuristic and path, wavefront and expansion counts -- bit-exact."""
import os

import numpy as np
import pytest

import scenegen
from _gpu import BIG, assert_same_search
from _search_ref import random_graph

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.fixture(scope="module")
def ws(mp):
    return mp.Workspace(40000, front_cap=2048, max_plans=1 << 23)


@pytest.mark.parametrize("seed", range(30))
def test_random_graphs(mp, orc, ws, seed):
    rng = np.random.default_rng(500 + seed)
    V = int(rng.integers(3, 40))
    g = random_graph(rng, V, p_edge=float(rng.uniform(0.1, 0.5)), cmax=int(rng.integers(1, 9)),
                     dmax=int(rng.integers(1, 6)))
    ro = orc.roadmap_from_csr(*g)
    rg = mp.roadmap_from_csr(*g)
    for beta in (int(rng.integers(0, 12)), BIG):
        for lam in (1, 2, 7, 1000):
            for stop in (True, False):
                a = orc.explore(ro, beta, lam, goal_termination=stop)
                b = mp.search(ws, rg, beta, group_width_q=lam, goal_stop=stop)
                assert_same_search(b, a, ws)


def test_narrow_passage(mp, ws):
    lines = [l.split() for l in open(os.path.join(GOLDEN, "narrow_passage_fig2.txt"))
             if l.strip() and not l.startswith("#")]
    V, beta, goal_node = map(int, lines[0])
    edges = sorted(tuple(map(int, l)) for l in lines[1:-1])
    exp = list(map(int, lines[-1]))
    row_ptr = np.zeros(V + 1, np.uint32)
    for s, *_ in edges:
        row_ptr[s + 1:] += 1
    cols = list(zip(*edges))
    goal = np.zeros(V, np.uint8); goal[goal_node] = 1
    rg = mp.roadmap_from_csr(row_ptr, cols[1], cols[2], cols[3], cols[4], goal)
    r = mp.search(ws, rg, beta, group_width_q=1)
    assert [r.status, r.cost, r.h] + list(r.path) == exp


@pytest.mark.parametrize("name,seed,n,beta_mode", [
    ("2d", 1, 1000, "pct"), ("2d", 2, 1000, "pct"), ("2d", 3, 1000, "pct"), ("2d", 4, 1000, "inf"),
    ("2d", 5, 600, "zero"), ("3d", 1, 2500, "pct"), ("6d", 1, 3000, "pct"), ("6d", 2, 3000, "inf"),
])
def test_scenes(mp, orc, ws, name, seed, n, beta_mode):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro = orc.build_roadmap(sc, n=n, r=r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    beta = {"pct": orc.beta_percentile(ro), "inf": BIG, "zero": 0}[beta_mode]
    lam_q = orc.group_width(0.5, r)
    a = orc.explore(ro, beta, lam_q)
    b = mp.search(ws, rg, beta, lam=0.5)
    assert_same_search(b, a, ws)
    # exhaustive variant (no goal stop)
    a2 = orc.explore(ro, beta, lam_q, goal_termination=False)
    b2 = mp.search(ws, rg, beta, lam=0.5, goal_stop=False)
    assert_same_search(b2, a2, ws)
    # a front pool that runs out is reported, not truncated: with one pool entry
    # per node it lasts for at most V / 16 touched nodes (blocks hold 16 or more)
    touched = int((np.diff(a2.front_ptr) > 0).sum())
    if touched > rg.V // 16 + 1:
        small = mp.Workspace(rg.V, front_cap=1, max_plans=1 << 23)
        with pytest.raises(mp.MpapError) as e:
            mp.search(small, rg, beta, lam=0.5, goal_stop=False)
        assert e.value.status == mp.MPAP_ERR_CAPACITY


def test_batch_matches_individual(mp, orc):
    specs = [("2d", 1, 1000), ("3d", 2, 1500), ("6d", 3, 2000), ("2d", 7, 333), ("6d", 4, 1200)]
    rgs, ros, qs, betas = [], [], [], []
    for name, seed, n in specs:
        sc = scenegen.make_scene(name, seed, query_id=seed)
        r = sc.cfg.r if name != "6d" else 18.0
        ro = orc.build_roadmap(sc, n=n, r=r)
        rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
        beta = orc.beta_percentile(ro)
        ros.append((ro, r)); rgs.append(rg); betas.append(beta)
        qs.append(mp.make_query(beta, 0.5))
    total = sum(rg.V for rg in rgs)
    wsb = mp.Workspace(total, front_cap=1024, max_plans=1 << 23)
    res = mp.search_batch(wsb, rgs, qs)
    for i, ((ro, r), beta) in enumerate(zip(ros, betas)):
        a = orc.explore(ro, beta, orc.group_width(0.5, r))
        assert_same_search(res[i], a, wsb, index=i)


def test_capacity_and_iteration_limits(mp, orc):
    sc = scenegen.make_scene("2d", 2, query_id=2)
    ro = orc.build_roadmap(sc)
    rg = mp.build_roadmap_for_scene(sc)
    beta = orc.beta_percentile(ro)
    small = mp.Workspace(rg.V, front_cap=2, max_plans=1 << 20)
    with pytest.raises(mp.MpapError) as e:
        mp.search(small, rg, beta)
    assert e.value.status == mp.MPAP_ERR_CAPACITY
    tiny_arena = mp.Workspace(rg.V, front_cap=1024, max_plans=64)
    with pytest.raises(mp.MpapError) as e:
        mp.search(tiny_arena, rg, beta)
    assert e.value.status == mp.MPAP_ERR_CAPACITY
    big = mp.Workspace(rg.V, front_cap=1024, max_plans=1 << 22)
    a = orc.explore(ro, beta, orc.group_width(0.5, sc.cfg.r), max_iters=5)
    assert a.status == -4
    with pytest.raises(mp.MpapError) as e:
        mp.search(big, rg, beta, max_iters=5)
    assert e.value.status == mp.MPAP_ERR_ITER_LIMIT
    # the workspace stays usable after errors
    ok = mp.search(big, rg, beta)
    assert_same_search(ok, orc.explore(ro, beta, orc.group_width(0.5, sc.cfg.r)), big)


def test_start_in_goal_and_isolated_start(mp, orc, ws):
    # x_init inside X_goal: the first group already holds a goal plan
    g = (np.array([0, 1, 1], np.uint32), np.array([1], np.uint32), np.array([3], np.int32),
         np.array([0], np.int32), np.array([0], np.int32), np.array([1, 0], np.uint8))
    r = mp.search(ws, mp.roadmap_from_csr(*g), BIG, group_width_q=1)
    assert (r.status, r.cost, list(r.path), r.wavefronts, r.expansions) == (0, 0, [0], 0, 0)
    # no out-edges at x_init: P_open empties after one wavefront
    g = (np.array([0, 0, 0], np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.int32),
         np.zeros(0, np.int32), np.zeros(0, np.int32), np.array([0, 1], np.uint8))
    r = mp.search(ws, mp.roadmap_from_csr(*g), BIG, group_width_q=1)
    a = orc.explore(orc.roadmap_from_csr(*g), BIG, 1)
    assert r.status == a.status == 1 and r.wavefronts == a.wavefronts


def test_full_size_6d(mp, orc):
    """The 6D, 16000-sample configuration the benchmark times: full comparison."""
    sc = scenegen.make_scene("6d", 1, query_id=1)
    ro = orc.build_roadmap(sc)
    rg = mp.build_roadmap_for_scene(sc)
    beta = orc.beta_percentile(ro)
    wsf = mp.Workspace(rg.V, front_cap=64, max_plans=1 << 24)
    a = orc.explore(ro, beta, orc.group_width(0.5, sc.cfg.r))
    b = mp.search(wsf, rg, beta, lam=0.5)
    assert_same_search(b, a, wsf)


def test_query_error_stays_with_its_query(mp, orc):
    """In one batch, a query that stops at its own iteration cap fails alone: the
    other queries' results stay exact."""
    specs = [("2d", 3, 800), ("6d", 2, 1500), ("3d", 4, 1200)]
    rgs, ros, qs, betas = [], [], [], []
    for name, seed, n in specs:
        sc = scenegen.make_scene(name, seed, query_id=seed)
        r = sc.cfg.r if name != "6d" else 18.0
        ro = orc.build_roadmap(sc, n=n, r=r)
        rgs.append(mp.build_roadmap_for_scene(sc, n=n, r=r)); ros.append((ro, r))
        betas.append(orc.beta_percentile(ro))
    total = sum(rg.V for rg in rgs)
    wsb = mp.Workspace(total, front_cap=1024, max_plans=1 << 22)
    qs = [mp.make_query(betas[0], 0.5, max_iters=3), mp.make_query(betas[1], 0.5), mp.make_query(betas[2], 0.5)]
    res = mp.search_batch(wsb, rgs, qs, check=False)
    assert res[0].status == mp.MPAP_ERR_ITER_LIMIT
    for i in (1, 2):
        ro, r = ros[i]
        assert_same_search(res[i], orc.explore(ro, betas[i], orc.group_width(0.5, r)), wsb, index=i)


def test_pool_share_exhaustion_stays_with_its_query(mp, orc):
    """Every query of a batch owns a share of half the front pool in proportion
    to its nodes, and may borrow from the other half: a 2D query whose fronts
    outgrow both fails, and the 6D query beside it (within its share) is still
    exact."""
    s2 = scenegen.make_scene("2d", 2, query_id=2)
    s6 = scenegen.make_scene("6d", 3, query_id=3)
    r2 = mp.build_roadmap_for_scene(s2)
    o6 = orc.build_roadmap(s6, n=1500, r=18.0)
    r6 = mp.build_roadmap_for_scene(s6, n=1500, r=18.0)
    b2 = orc.beta_percentile(orc.build_roadmap(s2))
    b6 = orc.beta_percentile(o6)
    wsb = mp.Workspace(r2.V + r6.V, front_cap=64, max_plans=1 << 22)
    qs = [mp.make_query(b2, 0.5, goal_stop=False), mp.make_query(b6, 0.5)]
    for _ in range(2):
        res = mp.search_batch(wsb, [r2, r6], qs, check=False)
        assert res[0].status == mp.MPAP_ERR_CAPACITY
        assert_same_search(res[1], orc.explore(o6, b6, orc.group_width(0.5, 18.0)), wsb, index=1)


def test_pool_common_half_and_own_share(mp, orc):
    """Half of the front pool is shared out among the queries of a batch in
    proportion to their nodes and half is common to the batch: a query whose
    fronts outgrow its share borrows from the common half, and its result (and
    every front) equals that of a run on its own.  With MPAP_QUERY_OWN_SHARE the
    same query ends with a capacity status instead, and the query beside it is
    exact either way."""
    cfg = scenegen.scaled_config(scenegen.DIM_2D, 1000)
    sb = scenegen.make_scene(cfg, 2, query_id=2)     # fronts of hundreds of plans
    ss = scenegen.make_scene(cfg, 1, query_id=1)
    rb, rs = mp.build_roadmaps([mp.scene_spec(sb), mp.scene_spec(ss)])
    bb = orc.beta_percentile(orc.build_roadmap(sb))
    bs = orc.beta_percentile(orc.build_roadmap(ss))
    big = mp.Workspace(rb.V, front_cap=4096, max_plans=1 << 24)
    ref_b = mp.search(big, rb, bb, lam=0.5)
    fr_b = big.fronts(0)
    used_b = big.stats()[1]
    ref_s = mp.search(big, rs, bs, lam=0.5)
    fr_s = big.fronts(0)
    total = rb.V + rs.V
    fc = -(-2 * used_b // total)           # pool ~ 2x what the big query uses alone
    assert (fc * total // 2) * rb.V // total < used_b     # its share alone is too small
    wsb = mp.Workspace(total, front_cap=fc, max_plans=1 << 24)

    def same(a, b, fr, index):
        assert (a.status, a.cost, a.h, a.wavefronts, a.expansions, a.plans) == \
            (b.status, b.cost, b.h, b.wavefronts, b.expansions, b.plans)
        np.testing.assert_array_equal(a.path, b.path)
        ptr, cost, h = wsb.fronts(index)
        V = rb.V
        np.testing.assert_array_equal(ptr[:V + 1], fr[0][:V + 1])
        np.testing.assert_array_equal(cost, fr[1])
        np.testing.assert_array_equal(h, fr[2])

    res = mp.search_batch(wsb, [rb, rs], [mp.make_query(bb, 0.5), mp.make_query(bs, 0.5)], check=False)
    assert res[0].status == 0
    same(res[0], ref_b, fr_b, 0)
    same(res[1], ref_s, fr_s, 1)
    res = mp.search_batch(wsb, [rb, rs], [mp.make_query(bb, 0.5, own_share=True), mp.make_query(bs, 0.5)],
                          check=False)
    assert res[0].status == mp.MPAP_ERR_CAPACITY
    same(res[1], ref_s, fr_s, 1)


def test_barrier_timeout_is_reported(mp, orc, ws):
    """A grid-barrier wait of the device wavefront loop that runs past its limit
    ends the search with MPAP_ERR_TIMEOUT instead of hanging, and the workspace
    stays usable.  With a 1 us limit on a grid of hundreds of blocks some wait
    runs out (the first block at a barrier waits for all the others); the
    barrier itself never waits unbounded, so nothing on the GPU hangs."""
    sc = scenegen.make_scene("2d", 1, query_id=1)
    ro = orc.build_roadmap(sc, n=600)
    rg = mp.build_roadmap_for_scene(sc, n=600)
    beta = orc.beta_percentile(ro)
    with pytest.raises(mp.MpapError) as e:
        mp.search(ws, rg, beta, lam=0.5, wait_us=1)
    assert e.value.status == mp.MPAP_ERR_TIMEOUT
    ok = mp.search(ws, rg, beta, lam=0.5)
    assert_same_search(ok, orc.explore(ro, beta, orc.group_width(0.5, sc.cfg.r)), ws)
