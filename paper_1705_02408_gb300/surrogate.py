"""Screening candidate plans with the learned certification surrogate.

Alg. 1 certifies the plan Explore returns by Monte Carlo and, when it fails,
refines the perception bound and searches again.  Explore's own candidate set
P_candidates (Alg. 3 final lines: every plan stored at a goal node) already holds
the alternatives, so the plain GPU procedure here certifies candidates in cost
order, one Monte Carlo call per candidate, until one passes (hit rate <= eps).
The screened procedure first runs the MLP surrogate on every candidate's 48
trajectory features and certifies, in cost order, the candidates it predicts to
pass before the others.  Monte Carlo still decides every returned plan, so both
procedures meet the same certified failure bound; the screen only changes how
many Monte Carlo calls (and lock-step rounds over a batch of queries) that takes.

Every computation runs in libmpap kernels (search, candidate back-tracing,
features, MLP, Monte Carlo); the screened certification itself, ordering and
lock-step rounds included, is one library call (mpap_surrogate_screen).  This
module marshals arguments and sequences the training steps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import ctypes as C

from . import (Mlp, _check, _mc_array, _stream, certify_batch, lib, mpap_mc_params,
               plan_features_batch, search_candidates_batch)


def collect_candidates(ws, results, cap=64, path_cap=1 << 14):
    """P_candidates (up to cap, in solution order) of every query of the last
    mpap_search_batch on ws, in one launch; None for a query without a solution."""
    return search_candidates_batch(ws, len(results), cap=cap, path_cap=path_cap)


def candidate_features(rms, cands):
    """[k_i, 48] float32 features per query (k_i = number of candidates), in one launch."""
    return plan_features_batch(rms, [c["paths"] if c else [] for c in cands])


def mc_rates(rms, cands, mcs, call_base=0):
    """Monte Carlo hit rates of every candidate of every query in one batched
    certification: per query an array [k_i, 3] of (collision, localisation, any)
    failure fractions.  mcs[i] = (rollouts, seed, call_id, delta_fx, sigma_fx,
    shift); candidate j of query i uses call_id call_base + j."""
    jobs_rm, jobs_path, jobs_mc, where = [], [], [], []
    for i, (rm, c) in enumerate(zip(rms, cands)):
        if not c:
            continue
        ro, seed, _, delta, sig, sh = mcs[i]
        for j, p in enumerate(c["paths"]):
            jobs_rm.append(rm)
            jobs_path.append(p)
            jobs_mc.append((ro, seed, call_base + j, delta, sig, sh))
            where.append((i, j))
    out = [np.zeros((len(c["paths"]) if c else 0, 3)) for c in cands]
    if jobs_rm:
        certs = certify_batch(jobs_rm, jobs_path, jobs_mc)
        for (i, j), ct in zip(where, certs):
            r = float(ct["rollouts"])
            out[i][j] = (ct["hits_coll"] / r, ct["hits_loc"] / r, ct["hits_any"] / r)
    return out


def train(net: Mlp, X, Y, steps=1000, batch=4096, lr=1e-3, seed=0, log_every=0):
    """Minibatch Adam on (X [n,48], Y [n,2] soft labels), batches drawn uniformly
    with replacement; returns the per-step losses."""
    X = np.ascontiguousarray(X, np.float32)
    Y = np.ascontiguousarray(Y, np.float32)
    rng = np.random.default_rng(seed)
    b = min(batch, net.max_batch, len(X))
    losses = []
    for t in range(steps):
        idx = rng.integers(0, len(X), b)
        loss, _ = net.train_step(X[idx], Y[idx], lr=lr)
        losses.append(loss)
        if log_every and (t + 1) % log_every == 0:
            print(f"  step {t + 1}: loss {np.mean(losses[-log_every:]):.4f}", flush=True)
    return np.array(losses)


@dataclass
class Selection:
    chosen: np.ndarray      # per query: candidate index that passed, -1 if none did
    mc_calls: np.ndarray    # per query: Monte Carlo certifications spent
    rounds: int             # lock-step rounds (batched certification launches)
    p_fail: list = None     # per query: predicted any-failure probability of each candidate


def screen(net, rms, cands, mcs, eps, tau=0.1, use_net=True, feats=None, max_calls=0, stream=None):
    """mpap_surrogate_screen: certifies the candidates of every query in lock-step
    rounds until one passes (any-failure fraction <= eps), in the network's
    screened order (predicted any-failure <= tau first) when use_net, else in
    index (solution) order.  cands: per query a dict with "paths" (or None);
    mcs[i] = (rollouts, seed, call_base, delta_fx, sigma_fx, shift), candidate j
    certified with call id call_base + j; feats: per query [k_i, 48] float32, or
    None to compute them on the GPU."""
    nq = len(rms)
    counts = [len(c["paths"]) if c else 0 for c in cands]
    cand_ptr = np.zeros(nq + 1, np.uint32)
    cand_ptr[1:] = np.cumsum(counts)
    paths = [p for c in cands if c for p in c["paths"]]
    total = len(paths)
    path_ptr = np.zeros(total + 1, np.uint32)
    path_ptr[1:] = np.cumsum([len(p) for p in paths])
    flat = np.ascontiguousarray(np.concatenate(paths) if paths else np.zeros(1), np.uint32)
    fx = None
    if feats is not None and use_net and total:
        fx = np.ascontiguousarray(np.concatenate([f for f in feats if len(f)]), np.float32)
    ms, keep = _mc_array(mcs)
    chosen = np.zeros(max(nq, 1), np.int32)
    calls = np.zeros(max(nq, 1), np.uint32)
    pf = np.zeros(max(total, 1), np.float32)
    rounds = C.c_uint32()
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib().mpap_surrogate_screen(net.h if (use_net and net is not None) else None,
                                       (C.c_void_p * max(nq, 1))(*[rm.h for rm in rms]), nq, vp(cand_ptr),
                                       vp(path_ptr), vp(flat), vp(fx) if fx is not None else None,
                                       ms.ctypes.data_as(C.POINTER(mpap_mc_params)), float(eps), float(tau),
                                       1 if use_net else 0, int(max_calls), vp(chosen), vp(calls),
                                       C.byref(rounds), vp(pf), _stream(stream)), "mpap_surrogate_screen")
    split = [pf[cand_ptr[i]:cand_ptr[i + 1]].copy() for i in range(nq)]
    return Selection(chosen[:nq].astype(np.int64), calls[:nq].astype(np.int64), int(rounds.value), split)
