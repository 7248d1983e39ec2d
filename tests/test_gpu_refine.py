"""GPU perception-bound refinement (Alg. 1 step 4, Sec. 3) against the oracle's:
every round's bound, outcome, plan cost and hit count, and the final plan and
certificate, identical; lock-step batches give what single queries give."""
import numpy as np
import pytest

import scenegen
from oracle import refine as orf

pytestmark = pytest.mark.gpu

CASES = [  # name, seed, n, r, noise scale, max_hits of 512 rollouts
    ("2d", 4, 600, None, 2, 25),      # pass, fail, bisection
    ("2d", 5, 600, None, 2, 25),      # fail, tighten past "no plan", pass
    ("3d", 2, 1500, None, 2, 40),
    ("6d", 1, 2500, 18.0, 3, 40),
    ("6d", 4, 2500, 18.0, 1, 5),
]


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.fixture(scope="module")
def setup(mp, orc):
    out = []
    for name, seed, n, r, scale, mh in CASES:
        sc = scenegen.make_scene(name, seed, query_id=seed)
        rr = sc.cfg.r if r is None else r
        ro = orc.build_roadmap(sc, n=n, r=rr)
        rg = mp.build_roadmap_for_scene(sc, n=n, r=rr)
        mc = (512, sc.mc_seed, 0, sc.delta_fx, sc.sigma_fx * scale, sc.shift)
        out.append((sc, rr, ro, rg, mc, mh, orc.beta_percentile(ro)))
    return out


def _oracle(orc, sc, rr, ro, mc, mh, b0, rounds):
    return orf.refine(ro, b0, orc.group_width(0.5, rr), mh, rounds, rollouts=mc[0], seed=mc[1],
                      delta_fx=mc[3], sigma_fx=mc[4], shift=mc[5])


def _same(g, o):
    assert g.history == o.history
    assert (g.certified, g.beta, g.cost, g.h, g.rounds) == (o.certified, o.beta, o.cost, o.h, o.rounds)
    np.testing.assert_array_equal(g.path, o.path)
    assert g.cert == o.cert


def test_refine_batch_matches_oracle(mp, orc, setup):
    from paper_1705_02408_gb300.refine import refine_batch
    ws = mp.Workspace(sum(s[3].V for s in setup), front_cap=1024, max_plans=1 << 23)
    got = refine_batch(ws, [s[3] for s in setup], [s[6] for s in setup], [s[4] for s in setup],
                       [s[5] for s in setup], max_rounds=10)
    outcomes = set()
    for s, g in zip(setup, got):
        o = _oracle(orc, *[s[k] for k in (0, 1, 2, 4, 5, 6)], 10)
        _same(g, o)
        outcomes |= {h[1] for h in g.history}
    # the batch exercises every branch of the bounds
    assert {"pass", "fail", "none"} <= outcomes
    assert any(g.certified for g in got)


def test_lock_step_equals_single_queries(mp, setup):
    from paper_1705_02408_gb300.refine import refine_batch
    ws = mp.Workspace(sum(s[3].V for s in setup), front_cap=1024, max_plans=1 << 23)
    batch = refine_batch(ws, [s[3] for s in setup], [s[6] for s in setup], [s[4] for s in setup],
                         [s[5] for s in setup], max_rounds=7)
    for s, b in zip(setup, batch):
        one = refine_batch(ws, [s[3]], [s[6]], [s[4]], s[5], max_rounds=7)[0]
        _same(one, b)
