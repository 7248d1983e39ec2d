"""Pins for the oracle's primitives (CPU only): Philox, SampleFree, Near/Collision
(Alg. 2), the 6D steering connection and the per-edge heuristic transfer."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import scenegen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        vals = [int(t, 16) for t in row]
        out = orc.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_philox_uniformity(orc):
    # chi^2 over 64 bins of the top 6 bits of 4 * 20000 outputs
    words = np.concatenate([orc.philox4x32_10([i, 7, 3, 0], [123, 456]) for i in range(20000)])
    hist = np.bincount(words >> 26, minlength=64)
    exp = words.size / 64
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 120.0   # 63 dof: p ~ 1e-5 threshold


# ----------------------------------------------------------------------- SampleFree
def _inside_any(p, lo, hi, dp):
    return np.any(np.all((p[None, :dp] >= lo[:, :dp]) & (p[None, :dp] <= hi[:, :dp]), axis=1))


@pytest.mark.parametrize("name", ["2d", "3d", "6d"])
def test_sample_free(orc, name):
    sc = scenegen.make_scene(name, 3)
    n = 600
    rm = orc.build_roadmap(sc, n=n, r=0.05 if name != "6d" else 0.3)
    g = rm.graph()
    assert g.V == n + 2
    dp = scenegen.pos_dims(sc.dim_kind)
    np.testing.assert_array_equal(g.x[:, 0], sc.x_init)
    np.testing.assert_array_equal(g.x[:, 1], sc.x_goal)
    for v in range(2, g.V):
        p = g.x[:3, v]
        assert not _inside_any(p, sc.box_lo, sc.box_hi, dp)
        assert np.all((p[:dp] >= 0) & (p[:dp] < 1))
        if name == "6d":
            vel = g.x[3:, v].astype(np.float64)
            assert float(vel @ vel) <= 1.0 + 1e-6
        else:
            assert np.all(g.x[dp:, v] == 0)
    # determinism and independence of the query id
    g2 = orc.build_roadmap(sc, n=n, r=0.05 if name != "6d" else 0.3).graph()
    np.testing.assert_array_equal(g.x, g2.x)
    # the samples are the first n accepted candidates: check against a direct
    # Python draw of the first few candidates from Philox
    seed = sc.sample_seed
    key = [seed & 0xFFFFFFFF, seed >> 32]
    kept = []
    att = 0
    while len(kept) < 20:
        w = orc.philox4x32_10([att, 0, sc.query_id, 0], key)
        p = np.zeros(3, np.float32)
        p[:dp] = (w[:dp] >> 8).astype(np.float32) * np.float32(2.0 ** -24)
        ok = not _inside_any(p, sc.box_lo, sc.box_hi, dp)
        if ok and name == "6d":
            wv = orc.philox4x32_10([att, 1, sc.query_id, 0], key)
            u = (wv[:3] >> 8).astype(np.float64) * 2.0 ** -24
            vel = 2.0 * u - 1.0
            ok = float(vel @ vel) <= 1.0
        if ok:
            kept.append(p)
        att += 1
    np.testing.assert_array_equal(np.array(kept)[:, :dp], g.x[:dp, 2:22].T)


def test_goal_region(orc):
    sc = scenegen.make_scene("2d", 4)
    g = orc.build_roadmap(sc, n=3000, r=0.03).graph()
    d = np.sqrt(((g.x[:2].astype(np.float64) - g.x[:2, 1:2]) ** 2).sum(0))
    robust = np.abs(d - 0.05) > 1e-6
    assert g.is_goal[1] == 1
    np.testing.assert_array_equal(g.is_goal[robust], (d[robust] <= 0.05).astype(np.uint8))
    assert g.is_goal.sum() >= 3


# ------------------------------------------------------------------ slab collision
def _exact_hit(a, b, lo, hi, dp):
    """Closed segment vs closed box in exact rational arithmetic."""
    t0, t1 = Fraction(0), Fraction(1)
    for i in range(dp):
        A, B = Fraction(float(a[i])), Fraction(float(b[i]))
        L, H = Fraction(float(lo[i])), Fraction(float(hi[i]))
        d = B - A
        if d == 0:
            if A < L or A > H:
                return False
            continue
        ta, tb = (L - A) / d, (H - A) / d
        t0 = max(t0, min(ta, tb))
        t1 = min(t1, max(ta, tb))
    return t0 <= t1


def _seg(orc, dp, a, b, lo, hi):
    f = lambda v: np.array(list(v) + [0.0] * (3 - len(v)), np.float32)
    return orc.lib().orc_segment_hits_box(dp, f(a), f(b), f(lo), f(hi))


def test_slab_truth_table(orc):
    lo, hi = (0.25, 0.25), (0.5, 0.5)
    cases = [
        ((0.0, 0.375), (1.0, 0.375), 1),     # straight through
        ((0.0, 0.25), (1.0, 0.25), 1),       # along the bottom face (touching counts)
        ((0.0, 0.0), (0.25, 0.25), 1),       # ends exactly on a corner
        ((0.0, 0.5), (0.5, 0.0), 1),         # grazes the corner (0.25, 0.25)
        ((0.0, 0.5), (0.49, 0.0), 0),        # passes just outside the corner
        ((0.375, 0.375), (0.4, 0.4), 1),     # starts inside
        ((0.0, 0.125), (1.0, 0.125), 0),     # parallel below
        ((0.125, 0.0), (0.125, 1.0), 0),     # parallel left (d_x = 0, outside slab)
        ((0.375, 0.0), (0.375, 1.0), 1),     # d_x = 0 inside the slab
        ((0.0, 0.375), (0.2, 0.375), 0),     # stops short
        ((0.6, 0.6), (0.9, 0.9), 0),         # entirely beyond
    ]
    for a, b, want in cases:
        assert _seg(orc, 2, a, b, lo, hi) == want, (a, b)
        assert _seg(orc, 2, b, a, lo, hi) == want, (b, a)


def test_slab_vs_exact_random(orc):
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(3000):
        dp = int(rng.choice([2, 3]))
        a = rng.random(dp).astype(np.float32); b = rng.random(dp).astype(np.float32)
        c = rng.random(dp); s = rng.uniform(0.05, 0.3, dp)
        lo = (c - s / 2).astype(np.float32); hi = (c + s / 2).astype(np.float32)
        # skip near-degenerate cases: the answer must be the same for boxes grown
        # and shrunk by 1e-5
        e = 1e-5
        g1 = _exact_hit(a, b, lo - e, hi + e, dp)
        g2 = _exact_hit(a, b, lo + e, hi - e, dp)
        if g1 != g2:
            continue
        got = _seg(orc, dp, a, b, lo, hi)
        assert got == int(g1)
        checked += 1
    assert checked > 2900


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_near_and_collision_brute_force(orc, name):
    """Alg. 2 on a small kinematic roadmap: every robust pair is an edge iff its
    float64 length is below r and the exact segment misses every box."""
    sc = scenegen.make_scene(name, 5)
    r = 0.12 if name == "2d" else 0.25
    rm = orc.build_roadmap(sc, n=250, r=r)
    g = rm.graph()
    dp = scenegen.pos_dims(sc.dim_kind)
    edges = set()
    for v in range(g.V):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            edges.add((v, int(g.dst[e])))
    P = g.x[:dp].T.astype(np.float64)
    compared = 0
    for v in range(g.V):
        d = np.sqrt(((P - P[v]) ** 2).sum(1))
        for u in np.nonzero(np.abs(d - r) > 1e-6)[0]:
            u = int(u)
            if u == v:
                continue
            want = d[u] < r
            if want:
                hits = [(_exact_hit(g.x[:dp, v], g.x[:dp, u], sc.box_lo[b] - 1e-5, sc.box_hi[b] + 1e-5, dp),
                         _exact_hit(g.x[:dp, v], g.x[:dp, u], sc.box_lo[b] + 1e-5, sc.box_hi[b] - 1e-5, dp))
                        for b in range(sc.cfg.nb)]
                if any(h1 != h2 for h1, h2 in hits):
                    continue
                want = not any(h1 for h1, _ in hits)
            assert ((v, u) in edges) == want, (v, u)
            compared += 1
    assert compared > 1000
    # every edge cost is the rounded length (within one quantum of the float64 length)
    for v in range(0, g.V, 7):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            u = int(g.dst[e])
            L = math.sqrt(float(((P[u] - P[v]) ** 2).sum()))
            assert abs(int(g.cost_q[e]) - L * 2 ** 24) <= 1.5


# --------------------------------------------------------------- 6D steering (P8)
def _di6_pair(orc, a, b, T=0.25, M=16):
    x = np.zeros((6, 2), np.float32)
    x[:, 0] = a; x[:, 1] = b
    rm = orc.build_roadmap_from_points(6, np.zeros((0, 3)), np.zeros((0, 3)),
                                       np.full(1, 12, np.uint8), 1, x, r=1e-3, T=T, M=M)
    return rm, rm.edge_eval(0, 1)


def test_di6_boundary_conditions_and_energy(orc):
    rng = np.random.default_rng(5)
    T = 0.25
    for _ in range(40):
        a = np.concatenate([rng.random(3), rng.uniform(-0.5, 0.5, 3)]).astype(np.float32)
        b = np.concatenate([rng.random(3), rng.uniform(-0.5, 0.5, 3)]).astype(np.float32)
        _, ev = _di6_pair(orc, a, b, T)
        a0 = ev["a0"].astype(np.float64); j = ev["jerk"].astype(np.float64)
        p0, v0 = a[:3].astype(np.float64), a[3:].astype(np.float64)
        p1, v1 = b[:3].astype(np.float64), b[3:].astype(np.float64)
        # x'' = a0 + j t reaches (p1, v1) at t = T
        pT = p0 + v0 * T + a0 * T ** 2 / 2 + j * T ** 3 / 6
        vT = v0 + a0 * T + j * T ** 2 / 2
        scale = 1.0 + np.abs(a0).max() * T ** 2
        np.testing.assert_allclose(pT, p1, atol=2e-6 * scale)
        np.testing.assert_allclose(vT, v1, atol=2e-6 * scale)
        # J equals the integral of |a|^2 (Simpson in float64)
        t = np.linspace(0.0, T, 2001)
        acc = a0[None, :] + j[None, :] * t[:, None]
        f = (acc ** 2).sum(1)
        Jq = (T / 6000.0) * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
        assert abs(ev["J"] - Jq) <= 1e-4 * max(1.0, Jq)
        assert abs(ev["cost"] - (T + Jq)) <= 1e-4 * max(1.0, Jq)
        # checkpoints follow the cubic
        for m in range(1, 17):
            tm = m * T / 16
            pm = p0 + v0 * tm + a0 * tm ** 2 / 2 + j * tm ** 3 / 6
            np.testing.assert_allclose(ev["ckpt"][m - 1], pm, atol=5e-6 * scale)


def test_di6_minimum_energy(orc):
    """Perturbations that keep both boundary conditions (int w = 0 and
    int (T - t) w = 0) never lower the control energy: the connection is optimal."""
    rng = np.random.default_rng(8)
    T = 0.25
    t = np.linspace(0.0, T, 4001)
    wts = np.ones_like(t); wts[1:-1:2] = 4; wts[2:-1:2] = 2; wts *= (T / 4000.0) / 3
    basis = np.stack([np.sin((k + 1) * np.pi * t / T) for k in range(6)] +
                     [np.cos((k + 1) * np.pi * t / T) for k in range(6)])
    # project out the two constraint directions (1 and T - t) under the quadrature
    cons = np.stack([np.ones_like(t), T - t])
    Gm = cons @ (wts[:, None] * cons.T)
    for _ in range(10):
        a = np.concatenate([rng.random(3), rng.uniform(-0.5, 0.5, 3)]).astype(np.float32)
        b = np.concatenate([rng.random(3), rng.uniform(-0.5, 0.5, 3)]).astype(np.float32)
        _, ev = _di6_pair(orc, a, b, T)
        acc = ev["a0"][None, :].astype(np.float64) + ev["jerk"][None, :].astype(np.float64) * t[:, None]
        J0 = float((wts[:, None] * acc ** 2).sum())
        for _ in range(10):
            w = (rng.normal(size=(3, basis.shape[0])) @ basis)
            coef = np.linalg.solve(Gm, cons @ (wts[:, None] * w.T))
            w = w - (coef.T @ cons)
            J1 = float((wts[:, None] * (acc + 0.3 * w.T) ** 2).sum())
            assert J1 >= J0 - 1e-9


def test_di6_zero_displacement(orc):
    a = np.array([0.3, 0.4, 0.5, 0.5, -0.25, 0.0], np.float32)
    b = a.copy(); b[:3] = a[:3] + a[3:] * np.float32(0.25)
    _, ev = _di6_pair(orc, a, b)
    assert abs(ev["J"]) < 1e-9 and abs(ev["cost"] - 0.25) < 1e-9


# ------------------------------------------------- heuristic transfer (P2, P4)
def _steps_transfer(d, h0):
    h = h0
    for x in d:
        h = max(0, h + int(x))
    return h


def test_transfer_closed_form_on_edges(orc):
    """F_e(h) = max(C_e, h + S_e) reproduces literal per-step stepping of the
    heuristic for every h >= 0, and edges compose associatively."""
    sc = scenegen.make_scene("2d", 2)
    rm = orc.build_roadmap(sc, n=300, r=0.12)
    g = rm.graph()
    rng = np.random.default_rng(1)
    for v in range(0, g.V, 13):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            ev = rm.edge_eval(v, int(g.dst[e]))
            d = ev["d"]
            assert int(d.sum()) == int(g.S[e])
            assert _steps_transfer(d, 0) == int(g.C[e])
            for h in rng.integers(0, 3 * 10 ** 8, 5):
                assert _steps_transfer(d, int(h)) == max(int(g.C[e]), int(h) + int(g.S[e]))
    # composition of two (S, C) maps is again of the same form
    for _ in range(500):
        d1 = rng.integers(-9, 10, 7); d2 = rng.integers(-9, 10, 5)
        S1, C1 = int(d1.sum()), _steps_transfer(d1, 0)
        S2, C2 = int(d2.sum()), _steps_transfer(d2, 0)
        S12, C12 = S1 + S2, max(C2, C1 + S2)
        for h in rng.integers(0, 60, 4):
            assert _steps_transfer(np.concatenate([d1, d2]), int(h)) == max(C12, int(h) + S12)


@pytest.mark.parametrize("k", [0, 5, 12, 20, 24])
def test_constant_level_transfer(orc, k):
    sc = scenegen.make_scene("2d", 1)
    grid = np.full(sc.grid.size, k, np.uint8)
    sc.grid = grid
    g = orc.build_roadmap(sc, n=300, r=0.1).graph()
    M, nf = 16, 12
    S = M * (nf - k) * g.cost_q.astype(np.int64)
    np.testing.assert_array_equal(g.S, S)
    np.testing.assert_array_equal(g.C, np.maximum(S, 0))


def test_history_dependent_transfer(orc):
    """A horizontal edge between a featureless half (level 0) and a feature-rich
    half (level 24).  From x = 0.31 the checkpoints 0.31 + 0.025 m fall left of
    x = 0.5 for m = 1..7 and right for m = 8..16; from x = 0.71 they fall right for
    m = 1..8 and left for m = 9..16."""
    grid = np.array([0, 24, 0, 24], np.uint8)       # G = 2, x fastest
    x = np.zeros((6, 2), np.float32)
    x[0] = [0.31, 0.71]; x[1] = [0.5, 0.5]
    rm = orc.build_roadmap_from_points(2, np.zeros((0, 3)), np.zeros((0, 3)), grid, 2, x,
                                       r=1.0, M=16)
    g = rm.graph()
    assert g.dst.size == 2
    cq = int(g.cost_q[0])
    assert cq == int(g.cost_q[1])
    # 0 -> 1: +12 cq for 7 steps, then -12 cq for 9 steps (clamped at 0)
    assert int(g.S[0]) == -24 * cq and int(g.C[0]) == 0
    # 1 -> 0: 8 steps of -12 cq at h = 0 (h stays 0), then +12 cq for 8 steps
    assert int(g.S[1]) == 0 and int(g.C[1]) == 96 * cq
