"""Perception-bound refinement on the GPU (Alg. 1 step 4, Sec. 3).

Alg. 1 certifies the plan that Explore returns for a bound beta and, from the
Monte Carlo outcome, loosens beta (more aggressive plans) or tightens it (more
conservative ones) and explores again until a robust plan is found.  The paper
leaves the update open; the rule here:

  * a plan passes when its any-failure count is at most max_hits;
  * with no failure seen yet, beta becomes 2 beta + 1 after a pass or after "no
    plan", and the query stops once a pass brings no cheaper plan than the
    previous pass; with failures but no pass yet, beta halves towards the largest
    bound known to give no plan; with both, it bisects between the largest
    passing and the smallest failing bound; a query stops when no integer lies
    strictly between its bounds, or after max_rounds explorations;
  * the round-t certification uses call_id t;
  * a query's answer is the plan of its largest passing bound.

All queries advance in lock step: round t is one mpap_search_batch over the
queries still refining, each with its own bound, and one mpap_certify_batch of
the plans found.  This module only sequences those calls and keeps the bounds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import MPAP_NO_SOLUTION, MPAP_OK, certify_batch, make_query, search_batch

BETA_CAP = 1 << 62
PASS, FAIL, NONE, ERROR = "pass", "fail", "none", "error"


@dataclass
class Refined:
    certified: bool
    beta: int                 # largest passing bound (-1 without a pass)
    cost: int
    h: int
    path: np.ndarray
    cert: dict
    rounds: int
    history: list = field(default_factory=list)   # (beta, outcome, cost, hits_any) per round


@dataclass
class _Bounds:
    lo: int = None            # largest bound that passed
    lo_cost: int = None
    hi: int = None            # smallest bound that failed
    none: int = None          # largest bound without a plan

    def advance(self, beta, outcome, cost):
        """Records the outcome at beta and returns the next bound (None: stop)."""
        cheaper = False
        if outcome == PASS:
            cheaper = self.lo is None or cost < self.lo_cost
            self.lo, self.lo_cost = beta, cost
        elif outcome == FAIL:
            self.hi = beta
        else:
            self.none = beta
        if self.hi is None:
            if outcome == PASS and not cheaper:
                return None
            nb = min(2 * beta + 1, BETA_CAP)
            return nb if nb > beta else None
        if self.lo is None:
            below = -1 if self.none is None else self.none
            nb = (below + self.hi) // 2
            return nb if nb > below else None
        nb = (self.lo + self.hi) // 2
        return nb if nb > self.lo else None


def refine_batch(ws, rms, beta0, mcs, max_hits, max_rounds=8, lam=0.5, group_width_q=0,
                 path_cap=4096, stream=None):
    """Refines the bound of every query of the batch.

    rms: roadmaps; beta0: initial bounds; mcs: per query (rollouts, seed, _,
    delta_fx, sigma_fx, shift) (the call id is the round); max_hits: per query or
    one value.  Returns one Refined per query."""
    n = len(rms)
    hits_cap = list(max_hits) if np.ndim(max_hits) else [int(max_hits)] * n
    bounds = [_Bounds() for _ in range(n)]
    beta = [int(b) for b in beta0]
    best = [None] * n
    hist = [[] for _ in range(n)]
    active = list(range(n))
    t = 0
    while active and t < max_rounds:
        res = search_batch(ws, [rms[i] for i in active],
                           [make_query(beta[i], lam, group_width_q) for i in active],
                           path_cap=path_cap, stream=stream, check=False)
        found = [k for k, r in enumerate(res) if r.status == MPAP_OK]
        certs = {}
        if found:
            jobs = [active[k] for k in found]
            out = certify_batch([rms[i] for i in jobs], [res[k].path for k in found],
                                [(mcs[i][0], mcs[i][1], t, mcs[i][3], mcs[i][4], mcs[i][5]) for i in jobs],
                                stream=stream)
            certs = dict(zip(found, out))
        nxt = []
        for k, (i, r) in enumerate(zip(active, res)):
            if r.status == MPAP_OK:
                hits = certs[k]["hits_any"]
                outcome = PASS if hits <= hits_cap[i] else FAIL
                if outcome == PASS:
                    best[i] = (beta[i], r.cost, r.h, r.path, certs[k])
                hist[i].append((beta[i], outcome, int(r.cost), int(hits)))
            elif r.status == MPAP_NO_SOLUTION:
                outcome = NONE
                hist[i].append((beta[i], outcome, -1, -1))
            else:
                # a search error (capacity, iteration bound) ends this query's refinement
                hist[i].append((beta[i], ERROR, -1, int(r.status)))
                continue
            nb = bounds[i].advance(beta[i], outcome, r.cost)
            if nb is not None:
                beta[i] = nb
                nxt.append(i)
        active = nxt
        t += 1
    out = []
    for i in range(n):
        if best[i] is None:
            out.append(Refined(False, -1, -1, -1, np.zeros(0, np.uint32), {}, len(hist[i]), hist[i]))
        else:
            b, cost, h, path, cert = best[i]
            out.append(Refined(True, b, int(cost), int(h), path, cert, len(hist[i]), hist[i]))
    return out
