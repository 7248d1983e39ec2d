"""Parameters of the closed-loop VIO Monte Carlo model -- TEST INFRASTRUCTURE ONLY.

Sec. 4.1 tracks the nominal trajectory with an LQR controller and localises with a
Kalman filter that fuses an inertial prediction with feature-based position fixes;
the rollouts themselves are `certify_vio` in mpap_oracle.cpp.  This module gives
the controller gains: per position axis the discrete double integrator over one
checkpoint step, state (p, w) with w = velocity x step, x' = A x + B a with
A = [1 1; 0 1] and B = (1/2, 1), state cost diag(q_p, q_w), control cost r.  The
infinite-horizon LQR gain K = (r + B^T P B)^-1 B^T P A, where P solves the
discrete algebraic Riccati equation, found here by iterating the Riccati
recursion from P = Q to a fixed point (float64).  Only tests/, smoke() and the
bench's CPU legs use it.
"""
from __future__ import annotations

import numpy as np

A = np.array([[1.0, 1.0], [0.0, 1.0]])
B = np.array([[0.5], [1.0]])


def lqr_gain(q_p: float, q_w: float, r: float, iters: int = 100000, tol: float = 1e-13):
    """(k_p, k_w) of a = -(k_p p + k_w w) and the Riccati solution P."""
    Q = np.diag([q_p, q_w])
    P = Q.copy()
    for _ in range(iters):
        BtP = B.T @ P
        K = np.linalg.solve(r + BtP @ B, BtP @ A)
        Pn = Q + A.T @ P @ A - A.T @ P @ B @ K
        if np.max(np.abs(Pn - P)) <= tol * max(1.0, np.max(np.abs(P))):
            P = Pn
            break
        P = Pn
    BtP = B.T @ P
    K = np.linalg.solve(r + BtP @ B, BtP @ A)
    return float(K[0, 0]), float(K[0, 1]), P


def q16(x: float) -> int:
    return int(np.rint(x * 65536.0))


# the model's stated parameters (per checkpoint step; positions in 2^-20 units)
Q_A_FX = 60            # inertial noise per step (integrated acceleration, 2^-20 units)
R_MAX_FX = 2048        # position-fix noise at the lowest level that still gives a fix
LEVEL_MIN = 3          # levels below this see too few features for a fix
LQR_WEIGHTS = (1.0, 0.5, 20.0)   # q_p, q_w, r


def r_table(K: int = 24, n_f: int = 12, r_max: int = R_MAX_FX, level_min: int = LEVEL_MIN) -> np.ndarray:
    """Position-fix noise per quality level: none below level_min, then falling as
    1 / sqrt(level / level_min) (more features in view, a tighter fix)."""
    k = np.arange(K + 1)
    r = np.where(k >= level_min, np.rint(r_max * np.sqrt(level_min / np.maximum(k, 1))), 0)
    return r.astype(np.int32)
