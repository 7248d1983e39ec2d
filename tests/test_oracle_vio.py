"""Pins for the oracle's closed-loop VIO Monte Carlo model (LQR tracking,
inertial prediction, Kalman position fixes; Sec. 4.1) -- CPU only.  Each pin
comes from outside the model: scipy's Riccati solver, the closed-form
steady state of the alpha-beta tracker (the steady-state Kalman filter of the
white-acceleration double integrator, Kalata 1984), the closed-form variance of
dead reckoning, and the exact zero-noise and nominal-collision cases."""
import math

import numpy as np
import pytest

import oracle.vio as vio

K = 24
BIG = 1 << 30          # a localisation bound no rollout reaches (its square fits int64)


def _line_roadmap(orc, n_nodes, level, M=16, boxes=None, x0=0.2, x1=0.8):
    """Nodes evenly spaced on the diagonal of the unit square, constant quality."""
    x = np.zeros((6, n_nodes), np.float32)
    x[0] = np.linspace(x0, x1, n_nodes); x[1] = np.linspace(x0, x1, n_nodes)
    grid = np.full(4, level, np.uint8)
    lo = np.zeros((0, 3)) if boxes is None else boxes[0]
    hi = np.zeros((0, 3)) if boxes is None else boxes[1]
    spacing = (x1 - x0) * math.sqrt(2.0) / (n_nodes - 1)
    rm = orc.build_roadmap_from_points(2, lo, hi, grid, 2, x, r=1.2 * spacing, M=M, goal_radius=0.001)
    return rm, np.arange(n_nodes, dtype=np.uint32)


def _alpha_beta(lam):
    """Steady-state gains of the alpha-beta tracker for tracking index lam
    (process noise std per step / measurement noise std)."""
    s = math.sqrt(lam * lam + 8.0 * lam)
    alpha = -(lam * lam + 8.0 * lam - (lam + 4.0) * s) / 8.0
    beta = (lam * lam + 4.0 * lam - lam * s) / 4.0
    return alpha, beta


def test_lqr_gain_matches_scipy_riccati():
    la = pytest.importorskip("scipy.linalg")
    for qp, qw, r in [vio.LQR_WEIGHTS, (1.0, 1.0, 1.0), (5.0, 0.1, 0.3)]:
        kp, kw, P = vio.lqr_gain(qp, qw, r)
        Pr = la.solve_discrete_are(vio.A, vio.B, np.diag([qp, qw]), np.array([[r]]))
        Kr = np.linalg.solve(r + vio.B.T @ Pr @ vio.B, vio.B.T @ Pr @ vio.A)
        np.testing.assert_allclose(P, Pr, rtol=1e-8)
        np.testing.assert_allclose([kp, kw], Kr[0], rtol=1e-8)
        # the closed loop is stable
        assert np.max(np.abs(np.linalg.eigvals(vio.A - vio.B @ Kr))) < 1.0


@pytest.mark.parametrize("q_a,r", [(60, 2048), (300, 500), (20, 4000)])
def test_kalman_gains_reach_the_alpha_beta_steady_state(orc, q_a, r):
    rm, path = _line_roadmap(orc, 30, 10)          # 464 steps: converged to 1e-7 or better
    table = np.full(K + 1, r, np.int32)
    out = orc.certify_vio(rm, path, 1, 3, 0, BIG, q_a, 0, 0, table, trace=True)
    alpha, beta = _alpha_beta(q_a / r)
    Lp, Lw = out["gains"][-1]
    assert abs(Lp - alpha * 65536.0) <= 1.0
    assert abs(Lw - beta * 65536.0) <= 1.0
    # steady-state posterior position variance alpha r^2
    assert out["p00"][-1] == pytest.approx(alpha * r * r, rel=1e-6)


def test_rollout_error_variance_matches_the_filter(orc):
    """The integer rollouts' estimation error has the variance the covariance
    recursion predicts (20000 rollouts: 1 % standard error of a variance)."""
    q_a, r = 300, 500
    rm, path = _line_roadmap(orc, 12, 10)
    table = np.full(K + 1, r, np.int32)
    kp, kw, _ = vio.lqr_gain(*vio.LQR_WEIGHTS)
    out = orc.certify_vio(rm, path, 20000, 11, 0, BIG, q_a, vio.q16(kp), vio.q16(kw), table, trace=True)
    ep = out["ep_last"].astype(np.float64)
    assert abs(ep.mean()) < 4 * math.sqrt(out["p00"][-1] / len(ep)) + 2.0
    assert ep.var() == pytest.approx(out["p00"][-1], rel=0.05)


def test_dead_reckoning_variance_closed_form(orc):
    """No position fixes: the error of step s is sum_j (s - j + 1/2) na_j, so its
    variance is q_a^2 sum_{m=0..s} (m + 1/2)^2."""
    q_a = 60
    rm, path = _line_roadmap(orc, 6, 0)
    table = np.zeros(K + 1, np.int32)
    out = orc.certify_vio(rm, path, 20000, 5, 0, BIG, q_a, 0, 0, table, trace=True)
    S = len(out["p00"])
    closed = [q_a * q_a * sum((m + 0.5) ** 2 for m in range(s + 1)) for s in range(S)]
    np.testing.assert_allclose(out["p00"], closed, rtol=1e-12)
    assert (out["gains"] == 0).all()
    assert out["ep_last"].astype(np.float64).var() == pytest.approx(closed[-1], rel=0.05)


def test_lqr_regulates_the_estimated_deviation(orc):
    """The controller acts on the estimate p + ep, which then follows
    x' = (A - B K) x + B na: its stationary variance solves the discrete Lyapunov
    equation (scipy), while the estimation error alone (no fixes) keeps growing."""
    la = pytest.importorskip("scipy.linalg")
    q_a = 60
    rm, path = _line_roadmap(orc, 30, 0)
    kp, kw, _ = vio.lqr_gain(*vio.LQR_WEIGHTS)
    Kq = np.array([[vio.q16(kp), vio.q16(kw)]]) / 65536.0
    out = orc.certify_vio(rm, path, 20000, 21, 0, BIG, q_a, vio.q16(kp), vio.q16(kw), np.zeros(K + 1, np.int32),
                          trace=True)
    Acl = vio.A - vio.B @ Kq
    Sigma = la.solve_discrete_lyapunov(Acl, q_a * q_a * (vio.B @ vio.B.T))
    est = (out["p_last"] + out["ep_last"]).astype(np.float64)
    assert est.var() == pytest.approx(Sigma[0, 0], rel=0.05)
    assert out["ep_last"].astype(np.float64).var() > 100 * Sigma[0, 0]


def test_zero_noise_never_fails_and_a_blocked_nominal_always_does(orc):
    rm, path = _line_roadmap(orc, 8, 12)
    kp, kw, _ = vio.lqr_gain(*vio.LQR_WEIGHTS)
    none = np.zeros(K + 1, np.int32)
    out = orc.certify_vio(rm, path, 300, 1, 0, 1, 0, vio.q16(kp), vio.q16(kw), none)
    assert out == dict(hits_loc=0, hits_coll=0, hits_any=0, rollouts=300)
    # a box across the nominal path: every rollout collides, with or without noise
    box = (np.array([[0.45, 0.45, 0.0]]), np.array([[0.55, 0.55, 1.0]]))
    rmb, pathb = _line_roadmap(orc, 8, 12, boxes=box)
    for q_a, table in ((0, none), (60, vio.r_table())):
        out = orc.certify_vio(rmb, pathb, 200, 2, 0, BIG, q_a, vio.q16(kp), vio.q16(kw), table)
        assert out["hits_coll"] == 200 and out["hits_any"] == 200


def test_fixes_bound_the_error_and_failures_follow_delta(orc):
    """With position fixes the localisation failures at a bound of 3 steady-state
    standard deviations are rare; without them the error grows past it."""
    q_a, r = 60, 2048
    rm, path = _line_roadmap(orc, 12, 10)
    kp, kw, _ = vio.lqr_gain(*vio.LQR_WEIGHTS)
    fix = np.full(K + 1, r, np.int32)
    tr = orc.certify_vio(rm, path, 1, 3, 0, BIG, q_a, 0, 0, fix, trace=True)
    delta = int(3 * math.sqrt(tr["p00"][-1]) * 2)      # two axes: a generous radius
    with_fix = orc.certify_vio(rm, path, 4000, 7, 0, delta, q_a, vio.q16(kp), vio.q16(kw), fix)
    without = orc.certify_vio(rm, path, 4000, 7, 0, delta, q_a, vio.q16(kp), vio.q16(kw),
                              np.zeros(K + 1, np.int32))
    assert with_fix["hits_loc"] < 0.05 * 4000
    assert without["hits_loc"] > 0.5 * 4000


def test_determinism_and_streams(orc):
    rm, path = _line_roadmap(orc, 8, 10)
    kp, kw, _ = vio.lqr_gain(*vio.LQR_WEIGHTS)
    args = (rm, path, 512, 9, 0, 2500, 200, vio.q16(kp), vio.q16(kw), vio.r_table())
    a = orc.certify_vio(*args)
    assert a == orc.certify_vio(*args)
    b = orc.certify_vio(rm, path, 512, 9, 1, 2500, 200, vio.q16(kp), vio.q16(kw), vio.r_table())
    assert 0 < a["hits_loc"] < 512 and a != b
