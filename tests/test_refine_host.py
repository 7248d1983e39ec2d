"""Host logic of the GPU refinement driver (no GPU): its bound bookkeeping takes
the same steps as the oracle's on random outcome sequences, and the lock-step
driver sequences library calls as the oracle's loop does, with the searches and
certifications replaced by deterministic fakes."""
import numpy as np

from oracle import refine as orf


def _gpu_bounds():
    from paper_1705_02408_gb300.refine import _Bounds
    return _Bounds()


def test_bounds_follow_the_oracle_rule():
    rng = np.random.default_rng(5)
    for trial in range(300):
        b = _gpu_bounds()
        lo = lo_cost = hi = none = None
        beta = int(rng.integers(0, 1 << int(rng.integers(1, 40))))
        cost = 10 ** 9
        for step in range(40):
            outcome = rng.choice([orf.PASS, orf.FAIL, orf.NONE], p=[0.45, 0.4, 0.15])
            if outcome == orf.PASS:
                cost -= int(rng.integers(0, 3))
            got = b.advance(beta, outcome, cost)
            lo, lo_cost, hi, none, want = orf.next_beta(beta, outcome, cost, lo, lo_cost, hi, none)
            assert got == want, (trial, step)
            assert (b.lo, b.lo_cost, b.hi, b.none) == (lo, lo_cost, hi, none)
            if want is None:
                break
            beta = want


def test_lock_step_driver_with_fake_library(monkeypatch):
    """refine_batch against the oracle's sequential loop, with searches and
    certifications replaced by deterministic functions of (query, beta, call)."""
    import paper_1705_02408_gb300 as mp
    from paper_1705_02408_gb300 import refine as gref

    class R:
        def __init__(self, status, cost, h, path):
            self.status, self.cost, self.h, self.path = status, cost, h, path

    def fake_search(q, beta):
        if beta < 3 * q:
            return R(mp.MPAP_NO_SOLUTION, 0, 0, np.zeros(0, np.uint32))
        cost = 1000 - min(beta, 200 + 50 * q)
        return R(mp.MPAP_OK, cost, beta // 2, np.array([q, beta % 7], np.uint32))

    def fake_cert(q, path, call_id):
        beta_rt = int(path[1])
        hits = (q * 7 + call_id * 3 + beta_rt) % 11
        return {"hits_loc": hits, "hits_coll": 0, "hits_any": hits, "rollouts": 10}

    nq = 6
    rms = [object() for _ in range(nq)]
    qid = {id(r): i for i, r in enumerate(rms)}

    def search_batch(ws, rr, queries, path_cap=4096, stream=None, check=True):
        return [fake_search(qid[id(r)], q.beta) for r, q in zip(rr, queries)]

    def certify_batch(rr, paths, mcs, stream=None):
        return [fake_cert(qid[id(r)], p, m[2]) for r, p, m in zip(rr, paths, mcs)]

    monkeypatch.setattr(gref, "search_batch", search_batch)
    monkeypatch.setattr(gref, "certify_batch", certify_batch)
    beta0 = [10, 50, 3, 400, 0, 77]
    mcs = [(10, 1, 0, 1, None, None)] * nq
    got = gref.refine_batch(None, rms, beta0, mcs, 5, max_rounds=9)
    for q in range(nq):
        def s(beta, q=q):
            r = fake_search(q, beta)
            return r.status, r.cost, r.h, r.path

        def c(path, call_id, q=q):
            return fake_cert(q, path, call_id)

        want = orf.refine_with(s, c, beta0[q], 5, 9)
        g = got[q]
        assert g.history == want.history
        assert (g.certified, g.beta, g.cost, g.h, g.rounds) == (want.certified, want.beta, want.cost, want.h,
                                                                 want.rounds)
        np.testing.assert_array_equal(g.path, want.path)
        assert g.cert == want.cert
