"""Oracle of the learned error-rate heuristic -- TEST INFRASTRUCTURE ONLY.

Sec. 5.1 (learned heuristic): the position-error rate of the on-board state
estimate is modelled as a Gaussian whose mean and standard deviation a small
feedforward network predicts from the vehicle's linear and angular velocities
and the number of visible features (two hidden layers of eight ReLU units and a
projection to the two parameters), fitted by maximum likelihood.  The network is
evaluated over the mapped states, and the resulting map is interpolated by
weighted nearest neighbours over position, velocity and yaw to give the
heuristic at unvisited states used while building the graph.

Plain float64 NumPy, written from that description; only tests/, smoke() and
the bench's CPU legs use it.  Readings (the paper gives no formulas):
  * inputs x = (v_x, v_y, v_z, w_x, w_y, w_z, n) with n the visible-feature count;
  * z = W3 relu(W2 relu(W1 x + b1) + b2) + b3; mean = z_0,
    std = softplus(z_1) + SIGMA_MIN (a positive standard deviation);
  * loss = mean over samples of log std + (r - mean)^2 / (2 std^2) (the negative
    log-likelihood of r without its constant);
  * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; Kingma and Ba 2015);
  * map distance d^2 = w_p |dp|^2 + w_v |dv|^2 + w_y wrap(dyaw)^2 with
    wrap(a) = a - 2 pi round(a / 2 pi); the k nearest mapped states (ties by
    lower index) weighted by 1 / (d + 1e-6);
  * a mapped mean error rate mu enters the grid form of the heuristic as the
    level k = clamp(floor(n_f (1 - mu / mu_ref) + 1/2), 0, K): the grid form gains
    dt (1 - k / n_f) per step, the learned one dt mu / mu_ref.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 7, 8, 2
SIGMA_MIN = 1e-3
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
KNN_EPS = 1e-6


def unpack(p) -> dict:
    p = np.asarray(p, np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def softplus(z):
    return np.logaddexp(0.0, z)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, X):
    """(mean, std, cache) for inputs X [n, 7]."""
    d = unpack(p)
    X = np.asarray(X, np.float64)
    a1 = X @ d["W1"].T + d["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ d["W2"].T + d["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ d["W3"].T + d["b3"]
    mu = z[:, 0]
    sd = softplus(z[:, 1]) + SIGMA_MIN
    return mu, sd, (X, a1, h1, a2, h2, z)


def loss(p, X, r):
    mu, sd, _ = forward(p, X)
    r = np.asarray(r, np.float64)
    return float(np.mean(np.log(sd) + (r - mu) ** 2 / (2.0 * sd ** 2)))


def loss_and_grad(p, X, r):
    """Mean negative log-likelihood and its gradient by back-propagation."""
    d = unpack(p)
    mu, sd, (X, a1, h1, a2, h2, z) = forward(p, X)
    r = np.asarray(r, np.float64)
    n = len(r)
    e = r - mu
    L = float(np.mean(np.log(sd) + e ** 2 / (2.0 * sd ** 2)))
    dmu = -e / sd ** 2 / n
    dsd = (1.0 / sd - e ** 2 / sd ** 3) / n
    dz = np.stack([dmu, dsd * sigmoid(z[:, 1])], 1)
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ d["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"], g["b2"] = da2.T @ h1, da2.sum(0)
    dh1 = da2 @ d["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"], g["b1"] = da1.T @ X, da1.sum(0)
    return L, pack(g)


class Adam:
    def __init__(self, n, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + self.eps)


def wrap(a):
    return a - 2.0 * np.pi * np.round(a / (2.0 * np.pi))


def knn_dist2(map_state, q, w):
    """Squared map distances [Q, N] between query states q [Q, 7] and mapped
    states [N, 7], both (position 3, velocity 3, yaw), weights w = (w_p, w_v, w_y)."""
    M = np.asarray(map_state, np.float64)
    Qs = np.asarray(q, np.float64)
    dp = Qs[:, None, 0:3] - M[None, :, 0:3]
    dv = Qs[:, None, 3:6] - M[None, :, 3:6]
    dy = wrap(Qs[:, None, 6] - M[None, :, 6])
    return w[0] * (dp ** 2).sum(-1) + w[1] * (dv ** 2).sum(-1) + w[2] * dy ** 2


def knn_map(map_state, map_vals, q, k, w):
    """Weighted k-nearest-neighbour interpolation of the mapped (mean, std)
    values [N, 2] at query states q: returns (values [Q, 2], neighbour indices
    [Q, k] in increasing (distance, index) order, their distances)."""
    d2 = knn_dist2(map_state, q, w)
    N = d2.shape[1]
    k = min(k, N)
    order = np.lexsort((np.broadcast_to(np.arange(N), d2.shape), d2), axis=1)[:, :k]
    dk = np.sqrt(np.take_along_axis(d2, order, 1))
    wt = 1.0 / (dk + KNN_EPS)
    V = np.asarray(map_vals, np.float64)[order]          # [Q, k, 2]
    vals = (wt[:, :, None] * V).sum(1) / wt.sum(1)[:, None]
    return vals, order, dk


def levels_from_rate(mu, mu_ref, n_f=12, K=24):
    """Grid-form levels of mapped mean error rates (see the module docstring)."""
    x = n_f * (1.0 - np.asarray(mu, np.float64) / mu_ref)
    return np.clip(np.floor(x + 0.5), 0, K).astype(np.int64)


def cell_centers(G, dp):
    """Centres ((2 i + 1) / (2 G), ...) of a G^dp grid, x fastest: [G^dp, 3]."""
    c = (2.0 * np.arange(G) + 1.0) / (2.0 * G)
    if dp == 2:
        y, x = np.meshgrid(c, c, indexing="ij")
        return np.stack([x.ravel(), y.ravel(), np.zeros(G * G)], 1)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
