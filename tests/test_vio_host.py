"""Host-side parameters of the closed-loop VIO model: the library's LQR gains
(mpap_vio_lqr_gains, a Riccati fixed point in double) against the oracle's
(pinned against scipy's Riccati solver), and argument checks.  No GPU needed."""
import pytest

import oracle.vio as ov


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.mark.parametrize("w", [ov.LQR_WEIGHTS, (1.0, 1.0, 1.0), (5.0, 0.1, 0.3), (0.0, 1.0, 2.0), (1e-3, 0.0, 50.0)])
def test_lqr_gains_match_the_oracle(mp, w):
    kp, kw, _ = ov.lqr_gain(*w)
    got = mp.vio_lqr_gains(*w)
    assert abs(got[0] - ov.q16(kp)) <= 1 and abs(got[1] - ov.q16(kw)) <= 1


@pytest.mark.parametrize("w", [(-1.0, 1.0, 1.0), (1.0, -0.5, 1.0), (1.0, 1.0, 0.0), (1.0, 1.0, float("nan"))])
def test_lqr_gains_reject_bad_weights(mp, w):
    with pytest.raises(mp.MpapError) as e:
        mp.vio_lqr_gains(*w)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG
