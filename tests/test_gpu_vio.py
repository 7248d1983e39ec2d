"""GPU closed-loop VIO Monte Carlo certification (LQR tracking, inertial
prediction, Kalman position fixes; Sec. 4.1) vs the oracle: hit counts
bit-exact (integer rollouts on the same Philox normals, Kalman gains from the
same double recursion rounded to Q16)."""
import numpy as np
import pytest

import oracle.vio as vio
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


def _gains(weights=vio.LQR_WEIGHTS):
    kp, kw, _ = vio.lqr_gain(*weights)
    return vio.q16(kp), vio.q16(kw)


@pytest.mark.parametrize("name,seed,n", [("2d", 1, 1000), ("3d", 2, 2000), ("6d", 3, 3000), ("2d", 9, 500)])
def test_vio_matches_oracle(mp, orc, name, seed, n):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro, path = _plan(orc, sc, n, r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    kp, kv = _gains()
    cases = [(1024, 0, 2000, vio.Q_A_FX, vio.r_table()),              # fixes above level 3
             (1024, 3, 1500, 4 * vio.Q_A_FX, vio.r_table(r_max=600)),   # noisier inertia, tighter fixes
             (777, 5, 3000, vio.Q_A_FX, np.zeros(25, np.int32))]       # dead reckoning
    for R, call_id, delta, q_a, table in cases:
        a = orc.certify_vio(ro, path, R, sc.mc_seed, call_id, delta, q_a, kp, kv, table)
        b = mp.certify_vio(rg, path, R, sc.mc_seed, call_id, delta, q_a, kp, kv, table)
        assert a == b
        assert 0 <= b["hits_any"] <= R


def test_vio_line_with_a_box_and_uncontrolled(mp, orc):
    """A plan along a free diagonal with a box 0.002 beside it: the controller,
    acting on the estimate, moves the executed path off the nominal and into the
    box in some rollouts; without control (gains 0) the executed path is the
    nominal and never collides."""
    x = np.zeros((6, 10), np.float32)
    x[0] = np.linspace(0.2, 0.8, 10); x[1] = np.linspace(0.2, 0.8, 10)
    grid = np.full(4, 6, np.uint8)
    lo = np.array([[0.502, 0.40, 0.0]], np.float32); hi = np.array([[0.60, 0.4995, 1.0]], np.float32)
    rr = 1.2 * 0.6 * np.sqrt(2.0) / 9
    ro = orc.build_roadmap_from_points(2, lo, hi, grid, 2, x, r=rr, M=16, goal_radius=0.001)
    rg = mp.build_roadmap_from_points(2, lo, hi, grid, 2, x, r=rr, M=16, goal_radius=0.001)
    path = np.arange(10, dtype=np.uint32)
    got = []
    for kp, kv in (_gains(), (0, 0)):
        a = orc.certify_vio(ro, path, 2048, 17, 2, 1 << 30, 400, kp, kv, vio.r_table())
        b = mp.certify_vio(rg, path, 2048, 17, 2, 1 << 30, 400, kp, kv, vio.r_table())
        assert a == b
        got.append(b)
    assert got[0]["hits_coll"] > 0 and got[1]["hits_coll"] == 0


def test_vio_batch_equals_single_calls(mp, orc):
    jobs = []
    for name, seed, n in (("2d", 1, 800), ("3d", 2, 1500), ("6d", 3, 2500), ("6d", 4, 2000)):
        sc = scenegen.make_scene(name, seed, query_id=seed)
        r = sc.cfg.r if name != "6d" else 18.0
        ro, path = _plan(orc, sc, n, r)
        jobs.append((sc, ro, mp.build_roadmap_for_scene(sc, n=n, r=r), path))
    kp, kv = _gains()
    mcs = [(600 + 100 * i, sc.mc_seed, i, 1800) for i, (sc, _, _, _) in enumerate(jobs)]
    vios = [(vio.Q_A_FX * (i + 1), kp, kv, vio.r_table()) for i in range(len(jobs))]
    out = mp.certify_vio_batch([j[2] for j in jobs], [j[3] for j in jobs], mcs, vios)
    for (sc, ro, rg, path), m, v, o in zip(jobs, mcs, vios, out):
        assert o == orc.certify_vio(ro, path, *m, *v)
        assert o == mp.certify_vio(rg, path, *m, *v)
    # a single-node plan has no steps; zero rollouts count nothing
    sc, ro, rg, path = jobs[0]
    assert mp.certify_vio(rg, path[:1], 100, 1, 0, 1800, 60, kp, kv, vio.r_table())["hits_any"] == 0
    assert mp.certify_vio(rg, path, 0, 1, 0, 1800, 60, kp, kv, vio.r_table())["rollouts"] == 0
