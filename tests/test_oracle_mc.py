"""Pins for the oracle's Monte Carlo certifier (CPU only)."""
import math

import numpy as np
import pytest

import scenegen

K = 24


def _line_roadmap(orc, n_nodes, level, M=16, boxes=None, x0=0.2, x1=0.8):
    """Nodes evenly spaced on the diagonal of the unit square, constant quality."""
    x = np.zeros((6, n_nodes), np.float32)
    x[0] = np.linspace(x0, x1, n_nodes); x[1] = np.linspace(x0, x1, n_nodes)
    grid = np.full(4, level, np.uint8)
    lo = np.zeros((0, 3)) if boxes is None else boxes[0]
    hi = np.zeros((0, 3)) if boxes is None else boxes[1]
    spacing = (x1 - x0) * math.sqrt(2.0) / (n_nodes - 1)
    rm = orc.build_roadmap_from_points(2, lo, hi, grid, 2, x, r=1.2 * spacing, M=M,
                                       goal_radius=0.001)
    return rm, np.arange(n_nodes, dtype=np.uint32)


def _tables(sigma, shift=0):
    return np.full(K + 1, sigma, np.int32), np.full(K + 1, shift, np.int32)


def test_zero_noise_never_fails(orc):
    sc = scenegen.make_scene("2d", 1)
    rm = orc.build_roadmap(sc, n=1000, r=0.08)
    res = orc.explore(rm, 1 << 62, orc.group_width(0.5, 0.08))
    sig, sh = _tables(0)
    out = orc.certify(rm, res.path, 256, 5, 0, 52429, sig, sh)
    assert out == dict(hits_loc=0, hits_coll=0, hits_any=0, rollouts=256)


def test_huge_noise_always_fails(orc):
    rm, path = _line_roadmap(orc, 4, 0)
    sig, sh = _tables(1 << 19)
    out = orc.certify(rm, path, 300, 9, 1, 52429, sig, sh)
    assert out["hits_loc"] == 300 and out["hits_any"] == 300


def _irwin_hall_pmf():
    """Exact pmf of the sum of 12 independent uniform integers on [0, 65535]."""
    n = 12 * 65535 + 1
    size = 1 << 20
    p = np.zeros(size); p[:65536] = 1.0 / 65536
    f = np.fft.rfft(p)
    pmf = np.fft.irfft(f ** 12, size)[:n]
    pmf = np.maximum(pmf, 0.0)
    return pmf / pmf.sum()


def test_one_step_exact_tail(orc):
    """One checkpoint, no contraction: P(e_x^2 + e_y^2 >= delta^2) with
    e = floor(sigma (S - 6 * 2^16) / 2^16) and S an Irwin-Hall(12) integer, computed
    exactly by convolution, against 100k oracle rollouts (5 binomial sigma)."""
    sigma, delta = 1500, 2000
    rm, path = _line_roadmap(orc, 2, 0, M=1)
    sig, sh = _tables(sigma)
    R = 100000
    out = orc.certify(rm, path, R, 1234, 7, delta, sig, sh)
    pmf = _irwin_hall_pmf()
    xi = np.arange(pmf.size, dtype=np.int64) - 6 * 65536
    e = (sigma * xi) >> 16
    emin = int(e.min())
    pe = np.bincount(e - emin, weights=pmf)
    vals = np.arange(pe.size) + emin
    absv = np.abs(vals)
    # P(|e_y| >= m) for every m
    tail_abs = np.zeros(int(absv.max()) + 2)
    np.add.at(tail_abs, absv, pe)
    tail_abs = np.cumsum(tail_abs[::-1])[::-1]
    p = 0.0
    for a, pa in zip(vals, pe):
        t = delta * delta - int(a) * int(a)
        if t <= 0:
            p += pa
        else:
            m = math.isqrt(t)
            if m * m < t:
                m += 1
            p += pa * (tail_abs[m] if m < tail_abs.size else 0.0)
    got = out["hits_loc"] / R
    assert 0.05 < p < 0.95
    assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / R), (got, p)
    assert out["hits_coll"] == 0


def test_contraction_matches_ar1_model(orc):
    """A long constant-quality path with contraction shift 2: the failure rate
    matches an independent float64 simulation of the AR(1) walk
    e <- (3/4) e + sigma N(0, 1) (tolerance covers the Irwin-Hall and rounding
    approximations)."""
    sigma, shift, delta = 800, 2, 4200
    rm, path = _line_roadmap(orc, 14, 0)
    steps = 16 * 13
    sig, sh = _tables(sigma, shift)
    R = 6000
    out = orc.certify(rm, path, R, 99, 3, delta, sig, sh)
    rng = np.random.default_rng(0)
    N = 40000
    e = np.zeros((N, 2)); fail = np.zeros(N, bool)
    for _ in range(steps):
        e = e * 0.75 + sigma * rng.standard_normal((N, 2))
        fail |= (e * e).sum(1) >= delta * delta
    p = fail.mean()
    got = out["hits_loc"] / R
    assert 0.05 < p < 0.6
    assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / R) + 0.02, (got, p)
    # without contraction the walk diffuses and nearly every rollout fails
    sig0, sh0 = _tables(sigma, 0)
    out0 = orc.certify(rm, path, 1000, 99, 3, delta, sig0, sh0)
    assert out0["hits_loc"] > 950


def test_collision_and_workspace_failures(orc):
    # a box just beside the nominal path: noise pushes executed states into it
    lo = np.array([[0.45, 0.58, 0.0]], np.float32); hi = np.array([[0.55, 0.65, 1.0]], np.float32)
    rm, path = _line_roadmap(orc, 5, 0, boxes=(lo, hi), x0=0.2, x1=0.8)
    g = rm.graph()
    # the nominal connections avoid the box, so the path is a walk of the roadmap
    for a, b in zip(path, path[1:]):
        assert b in set(g.dst[g.row_ptr[a]:g.row_ptr[a + 1]].tolist())
    sig, sh = _tables(3000)
    out = orc.certify(rm, path, 2000, 5, 0, 1 << 30, sig, sh)
    assert out["hits_loc"] == 0 and 0 < out["hits_coll"] < 2000
    assert out["hits_any"] == out["hits_coll"]
    # far from the box and the map edge: no collisions
    rm2, path2 = _line_roadmap(orc, 5, 0, x0=0.3, x1=0.35)
    out2 = orc.certify(rm2, path2, 2000, 5, 0, 1 << 30, sig, sh)
    assert out2["hits_coll"] == 0
    # near the map edge: leaving the unit square counts as a failure
    rm3, path3 = _line_roadmap(orc, 5, 0, x0=0.001, x1=0.01)
    out3 = orc.certify(rm3, path3, 2000, 5, 0, 1 << 30, sig, sh)
    assert out3["hits_coll"] > 0


def test_determinism_and_streams(orc):
    rm, path = _line_roadmap(orc, 6, 3)
    sig, sh = _tables(900)
    a = orc.certify(rm, path, 3000, 77, 0, 5000, sig, sh)
    b = orc.certify(rm, path, 3000, 77, 0, 5000, sig, sh)
    c = orc.certify(rm, path, 3000, 77, 1, 5000, sig, sh)
    assert a == b
    assert a != c
    assert max(a["hits_loc"], a["hits_coll"]) <= a["hits_any"] <= a["hits_loc"] + a["hits_coll"]
