"""Perception-bound refinement (Alg. 1 step 4, Sec. 3): marshalling for
mpap_refine_batch and mpap_refine_advance.

Alg. 1 certifies the plan that Explore returns for a bound beta and, from the
Monte Carlo outcome, loosens beta (more aggressive plans) or tightens it (more
conservative ones) and explores again until a robust plan is found.  The library
implements the rule (include/mpap.h, mpap_refine_advance) and the lock-step
batched driver (mpap_refine_batch: per round one batched search over the queries
still refining and one batched certification with call id = round); this module
only converts arguments and results.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import (MPAP_REFINE_ERROR, MPAP_REFINE_FAIL, MPAP_REFINE_NONE, MPAP_REFINE_PASS, _as, _check, _mc_array,
               _stream, lib, make_query, mpap_mc_params, mpap_query, mpap_refine_bounds, mpap_refine_result,
               mpap_refine_round)

BETA_CAP = 1 << 62
PASS, FAIL, NONE, ERROR = "pass", "fail", "none", "error"
_NAMES = {MPAP_REFINE_PASS: PASS, MPAP_REFINE_FAIL: FAIL, MPAP_REFINE_NONE: NONE, MPAP_REFINE_ERROR: ERROR}
_CODES = {PASS: MPAP_REFINE_PASS, FAIL: MPAP_REFINE_FAIL, NONE: MPAP_REFINE_NONE}


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


class Bounds:
    """One query's bounds, advanced by the library's rule (mpap_refine_advance)."""

    def __init__(self):
        self.b = mpap_refine_bounds(-1, 0, -1, -1)

    def advance(self, beta, outcome, cost):
        """Records the outcome ("pass", "fail", "none") at beta and returns the
        next bound, None to stop."""
        nxt = C.c_int64()
        _check(lib().mpap_refine_advance(C.byref(self.b), int(beta), _CODES[outcome], int(cost), C.byref(nxt)),
               "mpap_refine_advance")
        return None if nxt.value < 0 else nxt.value

    @property
    def state(self):
        """(lo, lo_cost, hi, none) with None for unknown bounds."""
        f = lambda v: None if v < 0 else v
        return f(self.b.lo), (self.b.lo_cost if self.b.lo >= 0 else None), f(self.b.hi), f(self.b.none)


def refine_batch(ws, rms, beta0, mcs, max_hits, max_rounds=8, lam=0.5, group_width_q=0,
                 path_cap=4096, stream=None):
    """mpap_refine_batch: refines the bound of every query of the batch.

    rms: roadmaps; beta0: initial bounds; mcs: per query (rollouts, seed, _,
    delta_fx, sigma_fx, shift) (the call id is the round); max_hits: per query or
    one value.  Returns one Refined per query."""
    n = len(rms)
    hits_cap = np.ascontiguousarray(list(max_hits) if np.ndim(max_hits) else [int(max_hits)] * n, np.uint32)
    hs = (C.c_void_p * n)(*[rm.h for rm in rms])
    qs = (mpap_query * n)(*[make_query(int(b), lam, group_width_q) for b in beta0])
    ms, keep = _mc_array(mcs)
    paths = np.zeros((max(n, 1), path_cap), np.uint32)
    hist = (mpap_refine_round * (max(n, 1) * max_rounds))()
    outs = (mpap_refine_result * max(n, 1))()
    for i in range(n):
        outs[i].path_cap = path_cap
        outs[i].path = paths[i].ctypes.data_as(C.POINTER(C.c_uint32))
        outs[i].hist_cap = max_rounds
        outs[i].history = C.cast(C.addressof(hist) + i * max_rounds * C.sizeof(mpap_refine_round),
                                 C.POINTER(mpap_refine_round))
    _check(lib().mpap_refine_batch(ws.h, hs, qs, _as(ms, mpap_mc_params), hits_cap.ctypes.data_as(C.c_void_p),
                                   n, int(max_rounds), outs, _stream(stream)), "mpap_refine_batch")
    out = []
    for i in range(n):
        o = outs[i]
        h = []
        for t in range(min(o.rounds, max_rounds)):
            r = hist[i * max_rounds + t]
            h.append((int(r.beta), _NAMES[r.outcome], int(r.cost), int(r.hits)))
        if not o.certified:
            out.append(Refined(False, -1, -1, -1, np.zeros(0, np.uint32), {}, int(o.rounds), h))
            continue
        if o.status != 0:
            raise RuntimeError(f"refine_batch: query {i}'s plan needs more than path_cap = {path_cap} nodes")
        cert = dict(hits_loc=o.cert.hits_loc, hits_coll=o.cert.hits_coll, hits_any=o.cert.hits_any,
                    rollouts=o.cert.rollouts)
        out.append(Refined(True, int(o.beta), int(o.cost), int(o.h), paths[i, :o.path_len].copy(), cert,
                           int(o.rounds), h))
    return out
