"""What the trained surrogate gains over the method without it.

Training data come from the method itself: candidate goal plans of 256 seeded
6D queries (6000 samples, twice the 6D Monte Carlo noise), labelled by
1024-rollout Monte Carlo, train the network on the GPU.  On 64 held-out queries
the plain procedure certifies candidates in cost order until one passes a 5%
failure bound; the screened one tries the candidates the network predicts to
pass first.  Both return only Monte Carlo-certified plans (equal certified
failure bound, the same set of solved queries); the screen must need clearly
fewer Monte Carlo calls, at a small cost premium."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu

BIG = 1 << 62
EPS, TAU = 0.05, 0.1


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


def _batch(mp, S, ws, cfg, seeds, rollouts, call_base):
    scs = [scenegen.make_scene(cfg, s, query_id=s) for s in seeds]
    rms = mp.build_roadmaps([mp.scene_spec(sc) for sc in scs])
    res = mp.search_batch(ws, rms, [mp.make_query(BIG, 0.5, goal_stop=False) for _ in scs])
    cands = S.collect_candidates(ws, res, 64)
    feats = S.candidate_features(rms, cands)
    mcs = [(rollouts, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx, sc.shift) for sc in scs]
    return rms, cands, feats, mcs


def test_screen_needs_fewer_monte_carlo_calls(mp):
    from paper_1705_02408_gb300 import surrogate as S
    n, B = 6000, 32
    cfg = scenegen.surrogate_config(n)
    ws = mp.Workspace(B * (n + 2), front_cap=128, max_plans=1 << 24)
    X, Y = [], []
    for o in range(0, 256, B):
        rms, cands, feats, mcs = _batch(mp, S, ws, cfg, range(1001 + o, 1001 + o + B), 1024, 10000)
        for f, r in zip(feats, S.mc_rates(rms, cands, mcs, call_base=10000)):
            X.append(f)
            Y.append(r[:, :2])
    X, Y = np.concatenate(X), np.concatenate(Y)
    assert len(X) > 3000 and 0.05 < Y[:, 0].mean() < 0.5
    net = mp.Mlp(seed=3, max_batch=4096)
    losses = S.train(net, X, Y, steps=600, batch=4096, lr=2e-3)
    assert losses[-50:].mean() < 0.75 * losses[:5].mean()

    calls_plain = calls_screen = 0
    costs = []
    for o in range(0, 64, B):
        rms, cands, feats, mcs = _batch(mp, S, ws, cfg, range(1 + o, 1 + o + B), 1024, 0)
        # both procedures through the library's screened certification
        # (mpap_surrogate_screen): solution order, and the network's order
        a = S.screen(None, rms, cands, mcs, EPS, use_net=False)
        b = S.screen(net, rms, cands, mcs, EPS, TAU, use_net=True, feats=feats)
        # the screen's order: candidates predicted at most TAU first
        assert sum(int((p <= np.float32(TAU)).sum()) for p in b.p_fail) > 0
        np.testing.assert_array_equal(a.chosen >= 0, b.chosen >= 0)
        # every returned plan is certified: re-check both selections by Monte Carlo
        for sel in (a, b):
            for i in np.nonzero(sel.chosen >= 0)[0]:
                j = int(sel.chosen[i])
                ro, seed, _, d, sig, sh = mcs[i]
                c = mp.certify(rms[i], cands[i]["paths"][j], ro, seed, j, d, sig, sh)
                assert c["hits_any"] <= EPS * ro
        calls_plain += int(a.mc_calls.sum())
        calls_screen += int(b.mc_calls.sum())
        costs += [cands[i]["cost"][b.chosen[i]] / cands[i]["cost"][a.chosen[i]]
                  for i in range(len(cands)) if a.chosen[i] >= 0]
    print(f"Monte Carlo calls: plain {calls_plain}, screened {calls_screen}; "
          f"cost ratio mean {np.mean(costs):.4f}")
    assert len(costs) >= 48
    assert calls_screen <= 0.9 * calls_plain
    assert np.mean(costs) <= 1.1 and min(costs) >= 1.0
