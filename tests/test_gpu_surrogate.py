"""GPU parity of the surrogate path: candidate export (P_candidates, Alg. 3 final
lines) and trajectory features bit-exact against the oracle; the tensor-core MLP
forward pass, its back-propagated gradients and the Adam step against the float64
oracle with the same bfloat16 rounding points."""
import numpy as np
import pytest

import scenegen
from _gpu import BIG
from _search_ref import random_graph
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.fixture(scope="module")
def ws(mp):
    return mp.Workspace(40000, front_cap=2048, max_plans=1 << 23)


def _same_candidates(g, o):
    assert g["total"] == o["total"]
    assert len(g["paths"]) == len(o["paths"])
    np.testing.assert_array_equal(g["cost"], o["cost"])
    np.testing.assert_array_equal(g["h"], o["h"])
    for a, b in zip(g["paths"], o["paths"]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("seed", range(12))
def test_candidates_random_graphs(mp, orc, ws, seed):
    rng = np.random.default_rng(900 + seed)
    V = int(rng.integers(3, 30))
    g = random_graph(rng, V, p_edge=float(rng.uniform(0.15, 0.5)), dmax=int(rng.integers(1, 5)))
    ro = orc.roadmap_from_csr(*g)
    rg = mp.roadmap_from_csr(*g)
    for stop in (True, False):
        for cap in (1, 5, 300):
            a = orc.explore(ro, BIG, 2, goal_termination=stop, candidates=cap)
            b = mp.search(ws, rg, BIG, group_width_q=2, goal_stop=stop)
            assert b.status == a.status
            if a.status != 0:
                continue
            _same_candidates(mp.search_candidates(ws, 0, cap=cap), a.candidates)


@pytest.mark.parametrize("name,seed,n", [("2d", 1, 1000), ("2d", 6, 1000), ("3d", 2, 2500),
                                         ("6d", 1, 3000), ("6d", 4, 3000)])
def test_candidates_and_features_on_scenes(mp, orc, ws, name, seed, n):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    r = sc.cfg.r if name != "6d" else 18.0
    ro = orc.build_roadmap(sc, n=n, r=r)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    beta = orc.beta_percentile(ro)
    for stop in (True, False):
        a = orc.explore(ro, beta, orc.group_width(0.5, r), goal_termination=stop, candidates=64)
        b = mp.search(ws, rg, beta, lam=0.5, goal_stop=stop)
        assert b.status == a.status == 0
        cand = mp.search_candidates(ws, 0, cap=64)
        _same_candidates(cand, a.candidates)
        np.testing.assert_array_equal(cand["paths"][0], b.path)
        fg = mp.plan_features(rg, cand["paths"])
        fo = orc.plan_features(ro, cand["paths"])
        assert fg.shape == (len(cand["paths"]), 48)
        np.testing.assert_array_equal(fg, fo)


def test_candidates_reject_unfinished_query(mp, ws):
    g = (np.array([0, 0, 0], np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.int32),
         np.zeros(0, np.int32), np.zeros(0, np.int32), np.array([0, 1], np.uint8))
    rg = mp.roadmap_from_csr(*g)
    r = mp.search(ws, rg, BIG, group_width_q=1)
    assert r.status == 1
    with pytest.raises(mp.MpapError) as e:
        mp.search_candidates(ws, 0, cap=4)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG


def _features(rng, n):
    x = np.empty((n, 48), np.float32)
    x[:, :32] = rng.uniform(0, 1, (n, 32))
    x[:, 32:] = rng.uniform(-1, 1, (n, 16))
    return x


@pytest.mark.parametrize("n", [1, 127, 128, 300, 1000, 4096])
def test_mlp_forward_matches_oracle(mp, n):
    rng = np.random.default_rng(n)
    net = mp.Mlp(seed=11, max_batch=4096)
    p = net.get_params().astype(np.float64)
    # non-zero biases so that every bias path is exercised
    d = omlp.unpack(p)
    for b in ("b1", "b2", "b3", "b4"):
        d[b] = rng.normal(0, 0.1, d[b].shape)
    p = omlp.pack(d).astype(np.float32)
    net.set_params(p)
    x = _features(rng, n)
    got = net.forward(x)
    z, _ = omlp.forward(p.astype(np.float64), x, rounding=True)
    want = omlp.sigmoid(z)
    assert got.shape == (n, 2)
    assert np.max(np.abs(got - want)) <= 1e-3


def test_mlp_forward_device_arrays(mp):
    import torch
    rng = np.random.default_rng(3)
    net = mp.Mlp(seed=2, max_batch=512)
    x = _features(rng, 300)
    a = net.forward(x)
    b = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n", [64, 333, 2048])
def test_mlp_gradients_match_oracle(mp, n):
    rng = np.random.default_rng(100 + n)
    net = mp.Mlp(seed=5, max_batch=4096)
    p = net.get_params().astype(np.float64)
    x = _features(rng, n)
    y = rng.uniform(0, 1, (n, 2)).astype(np.float32)
    loss, g = net.train_step(x, y, lr=0.0, apply=False, want_grads=True)
    lo, go = omlp.loss_and_grad(p, x, y, rounding=True)
    assert loss == pytest.approx(lo, rel=1e-4, abs=1e-6)
    gd, od = omlp.unpack(g.astype(np.float64)), omlp.unpack(go)
    # element by element: every entry of every parameter gradient within
    # 1e-2 of that tensor's largest oracle magnitude (fp32 accumulation in
    # another order can move a bfloat16 rounding of an activation by one unit,
    # 2^-8 relative, which reaches the gradients through the layers above)
    for k, _ in omlp.SHAPES:
        tol = 1e-2 * np.max(np.abs(od[k])) + 1e-6
        err = np.abs(gd[k] - od[k])
        worst = np.unravel_index(np.argmax(err), err.shape)
        assert err[worst] <= tol, (k, worst, gd[k][worst], od[k][worst], tol)
    # apply = False leaves the parameters alone
    np.testing.assert_array_equal(net.get_params(), p.astype(np.float32))


def test_adam_step_matches_oracle(mp):
    rng = np.random.default_rng(8)
    net = mp.Mlp(seed=9, max_batch=1024)
    p = net.get_params().astype(np.float64)
    opt = omlp.Adam(omlp.N_PARAMS, lr=3e-3)
    for step in range(3):
        x = _features(rng, 500)
        y = rng.uniform(0, 1, (500, 2)).astype(np.float32)
        _, g = net.train_step(x, y, lr=3e-3, apply=True, want_grads=True)
        p = opt.step(p, g.astype(np.float64))      # Adam on the device's own gradient
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - p)) <= 1e-6 + 1e-5 * np.max(np.abs(p)), step
        p = got


def test_mlp_learns_a_separable_rule(mp):
    """A rule the network can represent (failure iff the mean of the first 16
    features exceeds 0.5): the training loss falls well below log 2."""
    rng = np.random.default_rng(21)
    net = mp.Mlp(seed=1, max_batch=1024)
    losses = []
    for _ in range(300):
        x = _features(rng, 1024)
        t = (x[:, :16].mean(1) > 0.5).astype(np.float32)
        y = np.stack([t, 1 - t], 1)
        loss, _ = net.train_step(x, y, lr=3e-3)
        losses.append(loss)
    assert losses[0] > 0.6 and np.mean(losses[-20:]) < 0.2


def test_mlp_rejects_oversized_batch(mp):
    net = mp.Mlp(seed=0, max_batch=128)
    with pytest.raises(mp.MpapError) as e:
        net.forward(np.zeros((129, 48), np.float32))
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG


def test_batched_candidates_and_features_match_single_calls(mp, orc):
    """mpap_search_candidates_batch / mpap_plan_features_batch (one launch for a
    whole batch) give exactly what the per-query calls give."""
    specs = [("2d", 2, 600), ("6d", 1, 2500), ("2d", 1, 600), ("3d", 2, 1500), ("6d", 4, 2500)]
    rms, qs = [], []
    for name, seed, n in specs:
        sc = scenegen.make_scene(name, seed, query_id=seed)
        r = sc.cfg.r if name != "6d" else 18.0
        ro = orc.build_roadmap(sc, n=n, r=r)
        rms.append(mp.build_roadmap_for_scene(sc, n=n, r=r))
        qs.append(mp.make_query(orc.beta_percentile(ro), 0.5, goal_stop=False))
    wsb = mp.Workspace(sum(rg.V for rg in rms), front_cap=1024, max_plans=1 << 23)
    res = mp.search_batch(wsb, rms, qs)
    batch = mp.search_candidates_batch(wsb, len(rms), cap=40)
    assert any(c is None for c in batch) or all(r.status == 0 for r in res)
    for i, (r, c) in enumerate(zip(res, batch)):
        if r.status != 0:
            assert c is None
            continue
        _same_candidates(c, mp.search_candidates(wsb, i, cap=40))
    feats = mp.plan_features_batch(rms, [c["paths"] if c else [] for c in batch])
    for rg, c, f in zip(rms, batch, feats):
        if c:
            np.testing.assert_array_equal(f, mp.plan_features(rg, c["paths"]))
        else:
            assert f.shape == (0, 48)


def test_screen_matches_single_certifications(mp):
    """mpap_surrogate_screen against direct calls: its predicted failure is the
    network's forward pass combined as 1 - (1 - p_coll)(1 - p_loc) in binary32;
    its order puts the candidates predicted at most tau first (each group in
    solution order); and its lock-step selection equals certifying each query's
    candidates one by one in that order (call id base + j) until one passes.
    Features computed by the screen equal the ones given to it."""
    from paper_1705_02408_gb300 import surrogate as S
    cfg = scenegen.surrogate_config(3000)
    scs = [scenegen.make_scene(cfg, s, query_id=s) for s in (1, 2, 3, 4, 5)]
    rms = mp.build_roadmaps([mp.scene_spec(sc) for sc in scs])
    wsb = mp.Workspace(sum(r.V for r in rms), front_cap=128, max_plans=1 << 22)
    res = mp.search_batch(wsb, rms, [mp.make_query(BIG, 0.5, goal_stop=False) for _ in scs])
    cands = S.collect_candidates(wsb, res, 16)
    assert sum(1 for c in cands if c) >= 4
    feats = S.candidate_features(rms, cands)
    mcs = [(256, sc.mc_seed, 5, sc.delta_fx, sc.sigma_fx * 3, sc.shift) for sc in scs]
    net = mp.Mlp(seed=7, max_batch=512)
    eps, tau = 0.05, 0.5
    one = np.float32(1)
    for use_net in (False, True):
        sel = S.screen(net, rms, cands, mcs, eps, tau, use_net=use_net, feats=feats if use_net else None)
        for i, c in enumerate(cands):
            k = len(c["paths"]) if c else 0
            order = list(range(k))
            if use_net and k:
                P = net.forward(feats[i])
                pf = one - (one - P[:, 0]) * (one - P[:, 1])
                np.testing.assert_array_equal(sel.p_fail[i], pf)
                order = [j for j in range(k) if pf[j] <= np.float32(tau)] + \
                        [j for j in range(k) if pf[j] > np.float32(tau)]
            want, calls = -1, 0
            for j in order:
                ro, seed, base, d, sig, sh = mcs[i]
                ct = mp.certify(rms[i], c["paths"][j], ro, seed, base + j, d, sig, sh)
                calls += 1
                if ct["hits_any"] <= eps * ct["rollouts"]:
                    want = j
                    break
            assert (int(sel.chosen[i]), int(sel.mc_calls[i])) == (want, calls), (use_net, i)
        assert sel.rounds == int(max(sel.mc_calls))
    # features computed inside the screen give the same decisions
    a = S.screen(net, rms, cands, mcs, eps, tau, use_net=True, feats=feats)
    b = S.screen(net, rms, cands, mcs, eps, tau, use_net=True)
    np.testing.assert_array_equal(a.chosen, b.chosen)
    for x, y in zip(a.p_fail, b.p_fail):
        np.testing.assert_array_equal(x, y)
    # at most one call per query
    c1 = S.screen(net, rms, cands, mcs, eps, tau, use_net=True, feats=feats, max_calls=1)
    assert int(c1.mc_calls.max()) <= 1 and c1.rounds <= 1
