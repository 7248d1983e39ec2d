"""Certification-surrogate MLP, CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use this
module.  It shares no code with the CUDA library.

The paper certifies the final plan by Monte Carlo (Sec. 3, final phase; Alg. 1
step 4) and has no learned certifier; this network is the project's screening
surrogate.  It maps the 48 trajectory features of a candidate plan to two logits,
z = (collision, localisation), through three ReLU layers of width 128:

    h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), h3 = relu(h2 W3^T + b3),
    z  = h3 W4^T + b4,      p = sigmoid(z)

trained with binary cross-entropy against Monte Carlo hit rates (soft labels),
averaged over samples and both outputs, and Adam (Kingma and Ba, ICLR 2015,
Algorithm 1, with its bias corrections).

Arithmetic.  Everything is float64.  With ``rounding=True`` the values the device
kernels store in bfloat16 are rounded the same way, at the same points: the
input features, the weights used in products (W1..W4; the fp32 master copies and
all biases stay unrounded), the activations h1..h3 after the ReLU, and the
back-propagated pre-activation gradients dz3, dz2, dz1 after the ReLU mask.  The
logits' gradient dz4 and every parameter gradient stay unrounded.  The gradient
treats the bfloat16 roundings as the identity (straight through).  With
``rounding=False`` this is the plain float64 network, whose gradient is pinned
against central finite differences of its loss.

Packed parameter vector (also the library's): W1[128][48], b1[128],
W2[128][128], b2[128], W3[128][128], b3[128], W4[2][128], b4[2].
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 48, 128, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via binary32 as the device
    does: the value is first rounded to float32, then its low 16 bits are rounded
    away with round-half-to-even."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def unpack(params) -> dict:
    p = np.asarray(params, np.float64).ravel()
    assert p.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def _r(x, rounding):
    return bf16(x) if rounding else np.asarray(x, np.float64)


def forward(params, x, rounding: bool = True):
    """Returns (logits [n,2], cache) for features x [n,48]."""
    P = unpack(params)
    xb = _r(x, rounding)
    W = [_r(P[f"W{i}"], rounding) for i in (1, 2, 3, 4)]
    h1 = _r(np.maximum(xb @ W[0].T + P["b1"], 0.0), rounding)
    h2 = _r(np.maximum(h1 @ W[1].T + P["b2"], 0.0), rounding)
    h3 = _r(np.maximum(h2 @ W[2].T + P["b3"], 0.0), rounding)
    z = h3 @ W[3].T + P["b4"]
    return z, (xb, W, h1, h2, h3)


def sigmoid(z):
    z = np.asarray(z, np.float64)
    return np.where(z >= 0, 1.0 / (1.0 + np.exp(-np.abs(z))), np.exp(-np.abs(z)) / (1.0 + np.exp(-np.abs(z))))


def bce_loss(z, y) -> float:
    """Mean over samples and outputs of softplus(z) - y z (= the binary
    cross-entropy of sigmoid(z) against the soft label y)."""
    z = np.asarray(z, np.float64)
    sp = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
    return float(np.mean(sp - np.asarray(y, np.float64) * z))


def loss_and_grad(params, x, y, rounding: bool = True):
    """Loss and the packed gradient of it with respect to the parameters."""
    z, (xb, W, h1, h2, h3) = forward(params, x, rounding)
    n = z.shape[0]
    dz4 = (sigmoid(z) - np.asarray(y, np.float64)) / (2 * n)
    g = {"W4": dz4.T @ h3, "b4": dz4.sum(0)}
    dz3 = _r((dz4 @ W[3]) * (h3 > 0), rounding)
    g["W3"], g["b3"] = dz3.T @ h2, dz3.sum(0)
    dz2 = _r((dz3 @ W[2]) * (h2 > 0), rounding)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dz1 = _r((dz2 @ W[1]) * (h1 > 0), rounding)
    g["W1"], g["b1"] = dz1.T @ xb, dz1.sum(0)
    return bce_loss(z, y), pack(g)


class Adam:
    """Adam (Kingma and Ba 2015, Algorithm 1): m and v are exponential moving
    averages of the gradient and its square, divided by (1 - beta^t) before the
    step lr * m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, n, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, params, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return params - self.lr * mh / (np.sqrt(vh) + self.eps)
