"""Pins of the surrogate-MLP oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: the bfloat16 format, the derivative of the loss
(central finite differences), networks whose output has a closed form, the loss
at z = 0, and the first Adam step (Kingma and Ba 2015, Algorithm 1)."""
import numpy as np
import pytest

from oracle import mlp


def _net(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.N_PARAMS)


def test_param_count_and_layout():
    assert mlp.N_PARAMS == 128 * 48 + 128 + 2 * (128 * 128 + 128) + 2 * 128 + 2 == 39554
    p = np.arange(mlp.N_PARAMS, dtype=np.float64)
    d = mlp.unpack(p)
    assert d["W1"][1, 0] == 48 and d["b1"][0] == 128 * 48 and d["b4"][1] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(d), p)


def test_bf16_rounding_matches_the_format():
    # bfloat16 keeps 8 significand bits: 1 + 2^-7 is representable, 1 + 2^-8 is
    # a tie between 1 and 1 + 2^-7 (even: 1), 1 + 3 * 2^-8 ties to 1 + 2^-6 (even)
    cases = {1.0: 1.0, 1 + 2 ** -7: 1 + 2 ** -7, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6,
             1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7, -2.5: -2.5, 0.0: 0.0, 3.0e38: 226 * 2.0 ** 120}   # 3e38 = 1.7633 * 2^127 -> 226/128 * 2^127
    for x, want in cases.items():
        assert mlp.bf16(np.array([x]))[0] == pytest.approx(want, rel=1e-7), x
    # every output has 7 explicit significand bits and is within half an ulp
    x = np.random.default_rng(0).normal(0, 10, 10000)
    r = mlp.bf16(x)
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * (1 + 1e-6))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p = _net(1)
    x = rng.normal(0, 1, (7, 48))
    y = rng.uniform(0, 1, (7, 2))
    _, g = mlp.loss_and_grad(p, x, y, rounding=False)
    idx = np.concatenate([rng.choice(np.arange(0, 6144), 12, replace=False),          # W1
                          np.arange(6144, 6144 + 4),                                    # b1
                          rng.choice(np.arange(6272, 6272 + 16384), 12, replace=False), # W2
                          rng.choice(np.arange(22784, 22784 + 16384), 12, replace=False),
                          np.arange(39296, 39296 + 256, 37),                            # W4
                          [39552, 39553]])                                              # b4
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        lp = mlp.bce_loss(mlp.forward(p + e, x, False)[0], y)
        lm = mlp.bce_loss(mlp.forward(p - e, x, False)[0], y)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_identity_network_has_closed_form_output():
    # W1 copies the 48 features into units 0..47, W2 = W3 = I, W4 picks unit 0
    # for the first logit and minus unit 1 for the second: for x >= 0 the
    # logits are x0 + b and -x1 + c
    d = {k: np.zeros(s) for k, s in mlp.SHAPES}
    d["W1"][:48, :48] = np.eye(48)
    d["W2"][:] = np.eye(128)
    d["W3"][:] = np.eye(128)
    d["W4"][0, 0] = 1.0
    d["W4"][1, 1] = -1.0
    d["b4"][:] = [0.25, -0.5]
    x = np.abs(np.random.default_rng(2).normal(0, 1, (5, 48)))
    for rounding in (False, True):
        z, _ = mlp.forward(mlp.pack(d), x, rounding)
        xr = mlp.bf16(x) if rounding else x
        assert np.allclose(z[:, 0], xr[:, 0] + 0.25, rtol=0, atol=1e-15)
        assert np.allclose(z[:, 1], -xr[:, 1] - 0.5, rtol=0, atol=1e-15)
    # negative inputs are cut by the first ReLU
    z, _ = mlp.forward(mlp.pack(d), -x, False)
    assert np.allclose(z, [[0.25, -0.5]] * 5, atol=0)


def test_loss_at_zero_logits_is_log2_and_its_gradient():
    # with all weights zero, z = b4 = 0: loss = log 2 for any soft label and
    # dL/db4_o = mean over samples of (1/2 - y_o) / 2
    p = np.zeros(mlp.N_PARAMS)
    y = np.random.default_rng(3).uniform(0, 1, (9, 2))
    loss, g = mlp.loss_and_grad(p, np.ones((9, 48)), y)
    assert loss == pytest.approx(np.log(2.0), rel=1e-15)
    assert np.allclose(g[-2:], (0.5 - y).sum(0) / 18.0, atol=1e-16)
    assert np.all(g[:-2] == 0)


def test_sigmoid_is_stable_and_correct():
    z = np.array([-800.0, -30.0, 0.0, 2.0, 800.0])
    s = mlp.sigmoid(z)
    assert s[0] == 0.0 and s[-1] == 1.0 and s[2] == 0.5
    assert s[3] == pytest.approx(1 / (1 + np.exp(-2.0)), rel=1e-15)
    assert s[1] == pytest.approx(np.exp(-30.0) / (1 + np.exp(-30.0)), rel=1e-14)


def test_first_adam_step_is_lr_times_sign():
    # after one step m_hat = g and v_hat = g^2, so the step is lr g / (|g| + eps)
    g = np.array([1e-3, -2.0, 0.5, 0.0])
    opt = mlp.Adam(4, lr=0.01)
    p1 = opt.step(np.zeros(4), g)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    for _ in range(5):
        p1 = opt.step(p1, g)
    assert np.allclose(p1, -6 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)


def test_rounded_gradient_is_close_to_exact_one():
    # the straight-through bfloat16 gradient differs from the exact float64
    # one by the rounding of the stored values only (a few times 2^-8)
    rng = np.random.default_rng(7)
    p = _net(9, 0.15)
    x = rng.normal(0, 1, (64, 48))
    y = rng.uniform(0, 1, (64, 2))
    _, g0 = mlp.loss_and_grad(p, x, y, rounding=False)
    _, g1 = mlp.loss_and_grad(p, x, y, rounding=True)
    assert np.linalg.norm(g1 - g0) <= 0.05 * np.linalg.norm(g0)
