"""Host logic of the library's refinement (no GPU): its bound rule
(mpap_refine_advance, the step mpap_refine_batch takes after every
certification) takes the same steps as the oracle's on random outcome sequences
and at the edges of the integer range, and the batch entry point rejects bad
arguments before touching a device."""
import ctypes as C

import numpy as np
import pytest

from oracle import refine as orf


@pytest.fixture(scope="module")
def gref():
    from paper_1705_02408_gb300 import build
    build.build()
    from paper_1705_02408_gb300 import refine
    return refine


def _walk(gref, beta, outcomes, costs):
    b = gref.Bounds()
    lo = lo_cost = hi = none = None
    for outcome, cost in zip(outcomes, costs):
        got = b.advance(beta, outcome, cost)
        lo, lo_cost, hi, none, want = orf.next_beta(beta, outcome, cost, lo, lo_cost, hi, none)
        assert got == want, (beta, outcome, cost)
        assert b.state == (lo, lo_cost, hi, none)
        if want is None:
            return
        beta = want


def test_bounds_follow_the_oracle_rule(gref):
    rng = np.random.default_rng(5)
    for trial in range(300):
        beta = int(rng.integers(0, 1 << int(rng.integers(1, 40))))
        outcomes = rng.choice([orf.PASS, orf.FAIL, orf.NONE], size=40, p=[0.45, 0.4, 0.15])
        costs = 10 ** 9 - np.cumsum(rng.integers(0, 3, 40))
        _walk(gref, beta, list(outcomes), [int(c) for c in costs])


def test_bounds_at_the_edges(gref):
    """Loosening saturates at 2^62 (2 beta + 1 would overflow 64 bits near it);
    tightening from a failure at 0 stops (floor((-1 + 0) / 2) = -1 leaves no
    integer in between); bisection of bounds near 2^62 does not overflow."""
    cap = 1 << 62
    for beta in (cap // 2 - 1, cap // 2, cap // 2 + 1, cap - 1, cap):
        _walk(gref, beta, [orf.NONE, orf.NONE], [0, 0])
    _walk(gref, 0, [orf.FAIL], [0])
    _walk(gref, 5, [orf.FAIL, orf.NONE, orf.FAIL, orf.NONE], [0] * 4)
    _walk(gref, cap - 3, [orf.PASS, orf.PASS], [10, 9])
    _walk(gref, cap - 3, [orf.PASS, orf.FAIL, orf.PASS, orf.FAIL], [10, 0, 9, 0])


def test_advance_rejects_bad_arguments(gref):
    import paper_1705_02408_gb300 as mp
    b = mp.mpap_refine_bounds(-1, 0, -1, -1)
    nxt = C.c_int64()
    assert mp.lib().mpap_refine_advance(C.byref(b), -1, mp.MPAP_REFINE_PASS, 0, C.byref(nxt)) == \
        mp.MPAP_ERR_INVALID_ARG
    assert mp.lib().mpap_refine_advance(C.byref(b), 5, mp.MPAP_REFINE_ERROR, 0, C.byref(nxt)) == \
        mp.MPAP_ERR_INVALID_ARG
    assert mp.lib().mpap_refine_advance(None, 5, mp.MPAP_REFINE_PASS, 0, C.byref(nxt)) == mp.MPAP_ERR_INVALID_ARG
    # a batch without a workspace is rejected on the host
    assert mp.lib().mpap_refine_batch(None, None, None, None, None, 1, 4, None, None) == mp.MPAP_ERR_INVALID_ARG
    assert mp.lib().mpap_surrogate_screen(None, None, 1, None, None, None, None, None, 0.05, 0.1, 0, 0, None,
                                          None, None, None, None) == mp.MPAP_ERR_INVALID_ARG
