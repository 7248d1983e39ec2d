"""Oracle pins of the perception-bound refinement (Alg. 1 step 4, Sec. 3): the
bracket against closed-form thresholds, and on real scenes against plain
explore/certify calls and the unconstrained optimum."""
import numpy as np
import pytest

import scenegen
from oracle import refine as orf


def _synthetic(nu, theta, kappa, c0=10_000):
    """search: no plan below nu, else a plan whose cost falls with beta until
    kappa; certify: passes exactly for beta <= theta (one fake hit per unit)."""
    state = {}

    def search(beta):
        state["beta"] = beta
        if beta < nu:
            return 1, 0, 0, np.zeros(0, np.uint32)
        return 0, c0 - min(beta, kappa), 0, np.array([0, 1], np.uint32)

    def certify(path, call_id):
        return {"hits_any": 0 if state["beta"] <= theta else 1, "call_id": call_id}

    return search, certify


@pytest.mark.parametrize("beta0,nu,theta,kappa", [
    (100, 0, 337, 5000),        # passes at beta0, loosens, bisects down to theta
    (100, 0, 37, 5000),         # fails at beta0, tightens, bisects up to theta
    (100, 250, 1000, 5000),     # no plan at beta0, loosens through "no plan" first
    (1, 0, 0, 5000),            # theta = 0
    (5000, 10, 4321, 6000),
])
def test_bracket_finds_the_exact_threshold(beta0, nu, theta, kappa):
    s, c = _synthetic(nu, theta, kappa)
    r = orf.refine_with(s, c, beta0, max_hits=0, max_rounds=64)
    assert r.certified and r.beta == theta
    assert r.cost == 10_000 - min(theta, kappa)
    # round t certifies with call_id t, and the kept certificate is the pass at theta
    t = [h[0] for h in r.history].index(theta)
    assert r.cert["call_id"] == t
    assert all(o in (orf.PASS, orf.FAIL, orf.NONE) for _, o, _, _ in r.history)


def test_bracket_stops_when_loosening_no_longer_helps():
    # every plan passes; the cost stops falling at kappa = 40
    s, c = _synthetic(0, 1 << 40, 40)
    r = orf.refine_with(s, c, 3, max_hits=0, max_rounds=64)
    assert r.certified and r.cost == 10_000 - 40
    betas = [h[0] for h in r.history]
    assert betas == [3, 7, 15, 31, 63, 127]          # stops at the first pass without a cheaper plan
    assert r.beta == 127


def test_bracket_without_any_pass():
    s, c = _synthetic(50, 20, 5000)                  # passing betas all lie below nu: no plan there
    r = orf.refine_with(s, c, 100, max_hits=0, max_rounds=64)
    assert not r.certified and r.beta == -1
    outcomes = [h[1] for h in r.history]
    assert orf.PASS not in outcomes and orf.NONE in outcomes and orf.FAIL in outcomes
    # the last two bounds tried are adjacent: 49 (no plan) and 50 (fail)
    assert sorted(h[0] for h in r.history)[:2] == [49, 50]


def test_round_budget():
    s, c = _synthetic(0, 12345, 1 << 30)
    r = orf.refine_with(s, c, 1, max_hits=0, max_rounds=5)
    assert r.rounds == 5 and len(r.history) == 5


@pytest.fixture(scope="module")
def scene2d(orc):
    sc = scenegen.make_scene("2d", 4, query_id=4)
    ro = orc.build_roadmap(sc, n=600)
    return sc, ro


def _mc(sc, scale=1):
    return dict(rollouts=512, seed=sc.mc_seed, delta_fx=sc.delta_fx, sigma_fx=sc.sigma_fx * scale,
                shift=sc.shift)


def test_refined_plan_is_the_explored_and_certified_plan(orc, scene2d):
    sc, ro = scene2d
    lam = orc.group_width(0.5, sc.cfg.r)
    beta0 = orc.beta_percentile(ro)
    m = _mc(sc, 2)
    r = orf.refine(ro, beta0, lam, 25, 10, **m)
    outcomes = [h[1] for h in r.history]
    assert r.certified and orf.FAIL in outcomes and outcomes.count(orf.PASS) >= 2
    e = orc.explore(ro, r.beta, lam)
    assert (e.status, e.cost, e.h) == (0, r.cost, r.h)
    np.testing.assert_array_equal(e.path, r.path)
    t = [h[0] for h in r.history].index(r.beta)
    assert r.cert == orc.certify(ro, r.path, m["rollouts"], m["seed"], t, m["delta_fx"], m["sigma_fx"], m["shift"])
    assert r.cert["hits_any"] <= 25


def test_no_failure_bound_reaches_the_unconstrained_optimum(orc, scene2d):
    sc, ro = scene2d
    lam = orc.group_width(0.5, sc.cfg.r)
    m = _mc(sc)
    r = orf.refine(ro, 1, lam, m["rollouts"], 64, **m)      # every plan passes
    best = orc.explore(ro, orc.INT64_MAX, lam)
    assert r.certified and r.cost == best.cost


def test_unreachable_failure_bound(orc, scene2d):
    sc, ro = scene2d
    lam = orc.group_width(0.5, sc.cfg.r)
    r = orf.refine(ro, orc.beta_percentile(ro), lam, -1, 6, **_mc(sc))
    assert not r.certified and r.rounds <= 6
    assert all(o != orf.PASS for _, o, _, _ in r.history)
