"""Pins of the learned error-rate heuristic's oracle (Sec. 5.1; CPU only): the
network's likelihood gradient against central finite differences, the constant
predictor in closed form (its gradient vanishes at the sample mean and standard
deviation, the maximum-likelihood fit of a Gaussian), the first Adam step, the
weighted nearest-neighbour map against a k-d tree and hand-made cases, and the
grid levels of mapped rates by hand."""
import numpy as np
import pytest

from oracle import errnet as E


def _params(rng, scale=0.6):
    d = {name: rng.normal(0, scale, shape) for name, shape in E.SHAPES}
    return E.pack(d)


def _data(rng, n):
    X = np.concatenate([rng.uniform(-1, 1, (n, 6)), rng.integers(0, 25, (n, 1))], 1)
    r = rng.normal(0.02, 0.01, n)
    return X, r


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    X, r = _data(rng, 64)
    L, g = E.loss_and_grad(p, X, r)
    assert L == pytest.approx(E.loss(p, X, r), rel=1e-14)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (E.loss(p + e, X, r) - E.loss(p - e, X, r)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())
    # every layer is exercised: some units active, some not
    _, _, (_, a1, _, a2, _, _) = E.forward(p, X)
    assert 0 < (a1 > 0).mean() < 1 and 0 < (a2 > 0).mean() < 1


def test_constant_predictor_closed_form_and_mle():
    """With every weight zero the network predicts mean b3_0 and standard
    deviation softplus(b3_1) + SIGMA_MIN for every input; its likelihood is
    maximised by the sample mean and the (population) standard deviation."""
    rng = np.random.default_rng(2)
    X, r = _data(rng, 500)
    d = {name: np.zeros(shape) for name, shape in E.SHAPES}
    m, s = float(r.mean()), float(r.std())
    d["b3"] = np.array([m, np.log(np.expm1(s - E.SIGMA_MIN))])     # softplus^-1(s - SIGMA_MIN)
    p = E.pack(d)
    mu, sd, _ = E.forward(p, X)
    np.testing.assert_allclose(mu, m, rtol=1e-15)
    np.testing.assert_allclose(sd, s, rtol=1e-12)
    L, g = E.loss_and_grad(p, X, r)
    assert L == pytest.approx(np.log(s) + 0.5, rel=1e-12)     # mean (r - m)^2 = s^2
    np.testing.assert_allclose(E.unpack(g)["b3"], 0.0, atol=1e-10)
    # away from the fit the bias gradients have the closed form
    d["b3"] = np.array([m + 0.01, 0.3])
    p = E.pack(d)
    L, g = E.loss_and_grad(p, X, r)
    sd0 = np.log1p(np.exp(0.3)) + E.SIGMA_MIN
    e = r - (m + 0.01)
    assert E.unpack(g)["b3"][0] == pytest.approx(-np.mean(e) / sd0 ** 2, rel=1e-12)
    want = np.mean(1 / sd0 - e ** 2 / sd0 ** 3) / (1 + np.exp(-0.3))
    assert E.unpack(g)["b3"][1] == pytest.approx(want, rel=1e-12)


def test_first_adam_step_is_signed_learning_rate():
    rng = np.random.default_rng(3)
    p = _params(rng)
    g = rng.normal(0, 1, p.size)
    opt = E.Adam(p.size, lr=1e-3)
    # lr g / (|g| + eps) differs from lr sign(g) by lr eps / |g| at most
    np.testing.assert_allclose(opt.step(p, g), p - 1e-3 * np.sign(g), rtol=0, atol=1e-3 * 1e-8 / np.abs(g).min())


def test_knn_without_yaw_matches_kdtree():
    scipy_spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(4)
    M = np.concatenate([rng.uniform(0, 1, (400, 3)), rng.uniform(-1, 1, (400, 3)), rng.uniform(-3, 3, (400, 1))], 1)
    Q = np.concatenate([rng.uniform(0, 1, (50, 3)), rng.uniform(-1, 1, (50, 3)), rng.uniform(-3, 3, (50, 1))], 1)
    vals = rng.normal(0, 1, (400, 2))
    w = (4.0, 0.25, 0.0)
    got, idx, dist = E.knn_map(M, vals, Q, 8, w)
    scale = np.sqrt([w[0]] * 3 + [w[1]] * 3)
    tree = scipy_spatial.cKDTree(M[:, :6] * scale)
    td, ti = tree.query(Q[:, :6] * scale, k=8)
    np.testing.assert_allclose(dist, td, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(np.sort(idx, 1), np.sort(ti, 1))
    wt = 1 / (td + E.KNN_EPS)
    np.testing.assert_allclose(got, (wt[:, :, None] * vals[ti]).sum(1) / wt.sum(1)[:, None], rtol=1e-12)


def test_knn_hand_cases():
    # yaw wraps around: headings just either side of +-pi are neighbours
    M = np.zeros((3, 7))
    M[0, 6] = np.pi - 0.01
    M[1, 6] = 0.5
    M[2, 6] = -0.4
    q = np.zeros((1, 7))
    q[0, 6] = -np.pi + 0.01
    vals = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    _, idx, dist = E.knn_map(M, vals, q, 1, (1.0, 1.0, 1.0))
    assert idx[0, 0] == 0 and dist[0, 0] == pytest.approx(0.02, rel=1e-9)
    # a query on a mapped state returns (almost exactly) its value
    got, _, _ = E.knn_map(M, vals, M[1:2], 3, (1.0, 1.0, 1.0))
    np.testing.assert_allclose(got[0], vals[1], rtol=1e-5)
    # a constant map interpolates to that constant; ties go to the lower index
    got, idx, _ = E.knn_map(np.zeros((5, 7)), np.tile([0.3, 0.1], (5, 1)), np.ones((2, 7)), 3, (1.0, 1.0, 1.0))
    np.testing.assert_allclose(got, [[0.3, 0.1]] * 2, rtol=1e-15)
    np.testing.assert_array_equal(idx, [[0, 1, 2]] * 2)


def test_levels_by_hand():
    mu_ref, nf, K = 0.02, 12, 24
    got = E.levels_from_rate([0.0, 0.02, -0.02, 0.01, 0.03, -0.05], mu_ref, nf, K)
    assert list(got) == [12, 0, 24, 6, 0, 24]
    # halves round up: 8 (1 - 3/16) = 6.5 -> 7
    assert list(E.levels_from_rate([0.1875, 0.25], 1.0, 8, 24)) == [7, 6]
    c = E.cell_centers(2, 2)
    np.testing.assert_array_equal(c[:, :2], [[0.25, 0.25], [0.75, 0.25], [0.25, 0.75], [0.75, 0.75]])
    assert E.cell_centers(4, 3).shape == (64, 3)
