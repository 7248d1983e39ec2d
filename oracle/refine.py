"""Oracle of the perception-bound refinement -- TEST INFRASTRUCTURE ONLY.

Alg. 1 certifies the plan Explore returns for a bound beta by Monte Carlo and
then, per Sec. 3, loosens beta (more aggressive plans) or tightens it (more
conservative ones) and explores again until a robust plan is found.  The paper
gives no update rule; this is the reading both sides implement:

  * a plan at beta passes when its Monte Carlo any-failure count is at most
    max_hits (an integer fixed by the caller from the failure bound);
  * beta values that passed, failed or gave no plan bound the search: with no
    failure seen yet the bound doubles (2 beta + 1) after a pass or after "no
    plan", and stops once a pass brings no cheaper plan than the previous pass;
    with failures but no pass yet it halves towards the largest beta known to
    give no plan; with both it bisects between the largest passing and the
    smallest failing beta; it stops when no integer lies strictly between the
    bounds or after max_rounds explorations;
  * round t (0-based) certifies with call_id t;
  * the result is the plan of the largest passing beta.

Each step is a plain call of this package's explore() and certify(); the rounds
of one query run one after another.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BETA_CAP = 1 << 62

PASS, FAIL, NONE = "pass", "fail", "none"


@dataclass
class RefineResult:
    certified: bool
    beta: int                 # the largest passing beta (-1 without a pass)
    cost: int
    h: int
    path: np.ndarray
    cert: dict
    rounds: int
    history: list = field(default_factory=list)   # (beta, outcome, cost, hits_any) per round


def next_beta(beta, outcome, cost, lo, lo_cost, hi, none):
    """One step of the bracket: the updated (lo, lo_cost, hi, none) and the next
    beta, or None to stop.  lo/hi/none are None while unknown."""
    improved = False
    if outcome == PASS:
        improved = lo is None or cost < lo_cost
        lo, lo_cost = beta, cost
    elif outcome == FAIL:
        hi = beta
    else:
        none = beta
    if hi is None:
        # no failure yet: loosen, unless a pass stopped improving the plan
        if outcome == PASS and not improved:
            return lo, lo_cost, hi, none, None
        nb = min(2 * beta + 1, BETA_CAP)
        return lo, lo_cost, hi, none, (nb if nb > beta else None)
    if lo is None:
        # failures only: tighten towards the largest beta known to give no plan
        floor = -1 if none is None else none
        nb = (floor + hi) // 2
        return lo, lo_cost, hi, none, (nb if nb > floor else None)
    nb = (lo + hi) // 2
    return lo, lo_cost, hi, none, (nb if nb > lo else None)


def refine_with(search, certify, beta0: int, max_hits: int, max_rounds: int) -> RefineResult:
    """The refinement with explore/certify supplied as functions:
    search(beta) -> (status, cost, h, path); certify(path, call_id) -> cert dict."""
    lo = lo_cost = hi = none = None
    best = None
    history = []
    beta = int(beta0)
    t = 0
    while beta is not None and t < max_rounds:
        status, cost, h, path = search(beta)
        if status != 0:
            outcome, hits = NONE, -1
            cost = -1
        else:
            cert = certify(path, t)
            hits = cert["hits_any"]
            outcome = PASS if hits <= max_hits else FAIL
            if outcome == PASS:
                best = (beta, cost, h, np.asarray(path, np.uint32).copy(), cert)
        history.append((beta, outcome, int(cost), int(hits)))
        lo, lo_cost, hi, none, beta = next_beta(beta, outcome, cost, lo, lo_cost, hi, none)
        t += 1
    if best is None:
        return RefineResult(False, -1, -1, -1, np.zeros(0, np.uint32), {}, t, history)
    b, cost, h, path, cert = best
    return RefineResult(True, b, cost, h, path, cert, t, history)


def refine(rm, beta0: int, Lambda: int, max_hits: int, max_rounds: int, rollouts: int, seed: int,
           delta_fx: int, sigma_fx, shift) -> RefineResult:
    """The refinement on an oracle roadmap with Alg. 3 Explore (goal termination)
    and the Monte Carlo certifier."""
    import oracle

    def search(beta):
        r = oracle.explore(rm, beta, Lambda)
        return r.status, r.cost, r.h, r.path

    def certify(path, call_id):
        return oracle.certify(rm, path, rollouts, seed, call_id, delta_fx, sigma_fx, shift)

    return refine_with(search, certify, beta0, max_hits, max_rounds)
