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
features, MLP, Monte Carlo); this module sequences the calls.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Mlp, certify_batch, plan_features_batch, search_candidates_batch


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


def predicted_failure(net: Mlp, feats):
    """Predicted probability of any failure, 1 - (1 - p_coll)(1 - p_loc), per
    candidate of every query (one batched forward pass)."""
    sizes = [len(f) for f in feats]
    if sum(sizes) == 0:
        return [np.zeros(0) for _ in feats]
    X = np.concatenate([f for f in feats if len(f)])
    P = np.concatenate([net.forward(X[o:o + net.max_batch]) for o in range(0, len(X), net.max_batch)])
    pa = 1.0 - (1.0 - P[:, 0]) * (1.0 - P[:, 1])
    out, o = [], 0
    for s in sizes:
        out.append(pa[o:o + s])
        o += s
    return out


def screened_order(p_fail, tau):
    """Candidates predicted to pass (p_fail <= tau) first, then the rest; each
    group keeps the cost order."""
    idx = np.arange(len(p_fail))
    return np.concatenate([idx[p_fail <= tau], idx[p_fail > tau]]).astype(np.int64)


@dataclass
class Selection:
    chosen: np.ndarray      # per query: candidate index that passed, -1 if none did
    mc_calls: np.ndarray    # per query: Monte Carlo certifications spent
    rounds: int             # lock-step rounds (batched certification launches)


def certify_in_order(rms, cands, mcs, orders, eps, max_calls=None):
    """Lock-step over the batch: in round t every unresolved query certifies the
    t-th candidate of its order (one batched launch per round) and is resolved by
    the first candidate whose any-failure fraction is at most eps.  Candidate j of
    query i always uses call_id j, so a candidate's certificate does not depend on
    the order it is tried in."""
    nq = len(rms)
    chosen = np.full(nq, -1, np.int64)
    calls = np.zeros(nq, np.int64)
    live = [i for i in range(nq) if cands[i]]
    rounds = 0
    t = 0
    while live:
        batch = [i for i in live if t < len(orders[i]) and (max_calls is None or t < max_calls)]
        if not batch:
            break
        jobs = []
        for i in batch:
            j = int(orders[i][t])
            ro, seed, _, delta, sig, sh = mcs[i]
            jobs.append((i, j, (ro, seed, j, delta, sig, sh)))
        certs = certify_batch([rms[i] for i, _, _ in jobs], [cands[i]["paths"][j] for i, j, _ in jobs],
                              [m for _, _, m in jobs])
        rounds += 1
        done = set()
        for (i, j, _), ct in zip(jobs, certs):
            calls[i] += 1
            if ct["hits_any"] <= eps * ct["rollouts"]:
                chosen[i] = j
                done.add(i)
        live = [i for i in live if i not in done and t + 1 < len(orders[i])]
        t += 1
    return Selection(chosen, calls, rounds)
