"""The "for all t" form of the perception constraint (Eq. 2) on the GPU against
the oracle: per-edge transfer peaks of built roadmaps, and searches with the
interior check (fronts, results, counts) bit-exact."""
import numpy as np
import pytest

import scenegen
from _gpu import BIG, assert_same_search
from _search_ref import steps_to_SC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.fixture(scope="module")
def ws(mp):
    return mp.Workspace(40000, front_cap=2048, max_plans=1 << 23)


def _peaks(d):
    S, h, Smax, Cmax = 0, 0, None, 0
    for x in d:
        S += int(x)
        h = max(0, h + int(x))
        Smax = S if Smax is None else max(Smax, S)
        Cmax = max(Cmax, h)
    return Smax, Cmax


@pytest.mark.parametrize("seed", range(12))
def test_interior_random_graphs(mp, orc, ws, seed):
    rng = np.random.default_rng(8000 + seed)
    V = int(rng.integers(3, 30))
    rows, dst, cq, steps = [0], [], [], []
    for v in range(V):
        for u in range(V):
            if u != v and rng.random() < 0.3:
                dst.append(u)
                cq.append(int(rng.integers(1, 7)))
                steps.append(rng.integers(-3, 4, 5))
        rows.append(len(dst))
    goal = (rng.random(V) < 0.3).astype(np.uint8)
    goal[0] = 0
    goal[V - 1] = 1
    SC = np.array([steps_to_SC(d) for d in steps] or np.zeros((0, 2)), np.int64).reshape(-1, 2)
    PK = np.array([_peaks(d) for d in steps] or np.zeros((0, 2)), np.int64).reshape(-1, 2)
    args = (np.array(rows, np.uint32), np.array(dst, np.uint32), np.array(cq, np.int32), SC[:, 0], SC[:, 1], goal)
    ro = orc.roadmap_from_csr(*args, Smax=PK[:, 0], Cmax=PK[:, 1])
    rg = mp.roadmap_from_csr(*args, Smax=PK[:, 0], Cmax=PK[:, 1])
    for beta in (int(rng.integers(1, 8)), BIG):
        for stop in (True, False):
            a = orc.explore(ro, beta, 2, goal_termination=stop, check_interior=True)
            b = mp.search(ws, rg, beta, group_width_q=2, goal_stop=stop, interior=True)
            assert_same_search(b, a, ws)


@pytest.mark.parametrize("name,seed,n", [("2d", 3, 800), ("3d", 2, 2000), ("6d", 1, 2500), ("6d", 5, 2500)])
def test_interior_on_scenes(mp, orc, ws, name, seed, n):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro = orc.build_roadmap(sc, n=n, r=r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    g = ro.graph()
    Sm, Cm = rg.peaks()
    np.testing.assert_array_equal(Sm, g.Smax)
    np.testing.assert_array_equal(Cm, g.Cmax)
    assert np.all(Sm >= g.S) and np.all(Cm >= g.C)
    beta = orc.beta_percentile(ro)
    lam = orc.group_width(0.5, r)
    for stop in (True, False):
        a = orc.explore(ro, beta, lam, goal_termination=stop, check_interior=True)
        b = mp.search(ws, rg, beta, lam=0.5, goal_stop=stop, interior=True)
        assert_same_search(b, a, ws)
