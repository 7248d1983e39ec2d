"""GPU parity of the learned error-rate heuristic (Sec. 5.1) against the float64
oracle: forward pass, likelihood gradient (element by element), Adam steps,
training on synthetic observations, the weighted nearest-neighbour map and the
grid levels of mapped rates.  The GPU computes in binary32; tolerances follow
from that (relative 1e-4 for values, 1e-3 of each tensor's largest gradient
entry for sums over thousands of samples)."""
import numpy as np
import pytest

import scenegen
from oracle import errnet as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def _params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.normal(0, scale, int(np.prod(s))) for _, s in E.SHAPES]).astype(np.float32)


@pytest.mark.parametrize("n", [1, 255, 256, 1000, 5000])
def test_forward_matches_oracle(mp, n):
    net = mp.ErrNet(seed=1, max_batch=8192)
    p = _params(10 + n)
    net.set_params(p)
    X, _ = scenegen.vio_samples(n, n)
    got = net.forward(X)
    mu, sd, _ = E.forward(p.astype(np.float64), X)
    np.testing.assert_allclose(got[:, 0], mu, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(got[:, 1], sd, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("n", [37, 256, 4000])
def test_gradient_matches_oracle(mp, n):
    net = mp.ErrNet(seed=2, max_batch=8192)
    p = _params(20 + n, 0.3)
    net.set_params(p)
    X, r = scenegen.vio_samples(n, 100 + n)
    loss, g = net.train_step(X, r, lr=0.0, apply=False, want_grads=True)
    lo, go = E.loss_and_grad(p.astype(np.float64), X, r)
    assert loss == pytest.approx(lo, rel=1e-4, abs=1e-5)
    gd, od = E.unpack(g.astype(np.float64)), E.unpack(go)
    for k, _ in E.SHAPES:
        tol = 1e-3 * np.max(np.abs(od[k])) + 1e-7
        err = np.abs(gd[k] - od[k])
        assert err.max() <= tol, (k, err.max(), tol)
    # apply = False leaves the parameters alone
    np.testing.assert_array_equal(net.get_params(), p)


def test_adam_steps_match_oracle(mp):
    net = mp.ErrNet(seed=3, max_batch=4096)
    p = _params(5, 0.3).astype(np.float64)
    net.set_params(p.astype(np.float32))
    opt = E.Adam(E.N_PARAMS, lr=2e-3)
    for step in range(3):
        X, r = scenegen.vio_samples(2000, 300 + step)
        _, g = net.train_step(X, r, lr=2e-3, apply=True, want_grads=True)
        p = opt.step(p, g.astype(np.float64))       # Adam on the device's own gradient
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - p)) <= 1e-6 + 1e-5 * np.max(np.abs(p)), step
        p = got


def test_training_learns_the_rate_model(mp):
    """Maximum-likelihood training on the synthetic observations: the loss falls
    from its start to near the noise model's own negative log-likelihood, and
    the predicted mean follows the feature count (fewer features, larger rate)."""
    net = mp.ErrNet(seed=4, max_batch=1 << 15)
    X, r = scenegen.vio_samples(200000, 7)
    rng = np.random.default_rng(0)
    first = None
    for t in range(1500):
        idx = rng.integers(0, len(X), 8192)
        loss, _ = net.train_step(X[idx], r[idx], lr=3e-3)
        first = loss if first is None else first
    Xt, rt = scenegen.vio_samples(20000, 8)
    out = net.forward(Xt)
    fit = float(np.mean(np.log(out[:, 1]) + (rt - out[:, 0]) ** 2 / (2 * out[:, 1] ** 2)))
    sv, sw, nv = np.linalg.norm(Xt[:, :3], axis=1), np.linalg.norm(Xt[:, 3:6], axis=1), Xt[:, 6]
    true_sd = 0.004 * (1 + sv) + 0.002 * sw
    true_mu = 0.02 * (1 + 0.5 * sv + 0.3 * sw) * (1 - nv / 12.0)
    ideal = float(np.mean(np.log(true_sd) + (rt - true_mu) ** 2 / (2 * true_sd ** 2)))
    assert fit < first - 1.0
    assert fit < ideal + 0.25        # the float64 oracle on this schedule: ideal + 0.11
    assert np.corrcoef(out[:, 0], true_mu)[0, 1] > 0.95


def _map(seed, N):
    M = scenegen.mapped_states(N, seed)
    rng = np.random.default_rng(seed)
    V = np.stack([rng.normal(0.0, 0.02, N), rng.uniform(0.002, 0.01, N)], 1).astype(np.float32)
    return M, V


@pytest.mark.parametrize("N,Q,k", [(1, 10, 1), (300, 500, 8), (3000, 2000, 16), (5000, 777, 5)])
def test_knn_map_matches_oracle(mp, N, Q, k):
    M, V = _map(N, N)
    q = scenegen.mapped_states(Q, 1000 + N)
    w = (4.0, 1.0, 0.25)
    got = mp.errmap_query(M, V, q, k=k, w=w)
    want, _, _ = E.knn_map(M, V, q, k, w)
    # skip queries whose k-th and (k+1)-th oracle distances nearly tie
    d2 = np.sort(E.knn_dist2(M, q, w), 1)
    kk = min(k, N)
    robust = np.ones(Q, bool) if kk == N else (np.sqrt(d2[:, kk]) - np.sqrt(d2[:, kk - 1])) > 1e-4
    assert robust.mean() > 0.95
    np.testing.assert_allclose(got[robust], want[robust], rtol=1e-4, atol=1e-7)


def test_knn_map_device_arrays(mp):
    import torch
    M, V = _map(9, 2000)
    q = scenegen.mapped_states(700, 99)
    a = mp.errmap_query(M, V, q, k=8)
    b = mp.errmap_query(torch.from_numpy(M).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(q).cuda(),
                        k=8).cpu().numpy()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dim,G", [(2, 16), (3, 8), (6, 8)])
def test_levels_match_oracle(mp, dim, G):
    M, V = _map(40 + G, 4000)
    vel, yaw, mu_ref, w = (0.3, -0.2, 0.1), 0.7, 0.02, (4.0, 1.0, 0.25)
    got = mp.errmap_levels(M, V, dim, G, vel=vel, yaw=yaw, mu_ref=mu_ref, k=8, w=w)
    dp = 2 if dim == 2 else 3
    c = E.cell_centers(G, dp).astype(np.float32)
    q = np.concatenate([c, np.tile(np.array(vel + (yaw,), np.float32), (len(c), 1))], 1)
    mu, _, _ = E.knn_map(M, V, q, 8, w)
    want = E.levels_from_rate(mu[:, 0], mu_ref)
    x = 12 * (1 - mu[:, 0] / mu_ref) + 0.5
    robust = np.abs(x - np.round(x)) > 1e-3
    assert robust.mean() > 0.95 and len(set(want.tolist())) > 3
    np.testing.assert_array_equal(got[robust], want[robust])
