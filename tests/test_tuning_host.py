"""The launch-shape table of the library (host side only; no GPU needed)."""
import pytest


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    m.tuning_clear()
    yield m
    m.tuning_clear()


DEFAULT = dict(edge_warps=8, wave_blocks_per_sm=8, plan_lanes_from=8, front_cap=64, grid_merge_from=2048)


def test_defaults_and_buckets(mp):
    mp.tuning_clear()
    assert mp.tuning_get(6, 16002) == DEFAULT
    mp.tuning_set(6, 16002, edge_warps=4, wave_blocks_per_sm=2, plan_lanes_from=8, front_cap=128)
    want = dict(edge_warps=4, wave_blocks_per_sm=2, plan_lanes_from=8, front_cap=128, grid_merge_from=2048)
    # the key is (dimension, floor(log2 V)): 8192 <= V < 16384 share bucket 13
    assert mp.tuning_get(6, 8192) == want and mp.tuning_get(6, 16383) == want
    assert mp.tuning_get(6, 16384) == DEFAULT and mp.tuning_get(6, 8191) == DEFAULT
    assert mp.tuning_get(3, 16002) == DEFAULT and mp.tuning_get(0, 16002) == DEFAULT
    assert mp.tuning_export() == [(6, 13, want)]
    mp.tuning_set(0, 40000, wave_blocks_per_sm=4)
    assert [(d, b) for d, b, _ in mp.tuning_export()] == [(0, 15), (6, 13)]
    mp.tuning_clear()
    assert mp.tuning_export() == []


@pytest.mark.parametrize("bad", [dict(edge_warps=6), dict(edge_warps=16), dict(wave_blocks_per_sm=0),
                                 dict(plan_lanes_from=65), dict(front_cap=0), dict(grid_merge_from=32),
                                 dict(grid_merge_from=(1 << 30) + 1)])
def test_invalid_shapes_are_rejected(mp, bad):
    with pytest.raises(mp.MpapError) as e:
        mp.tuning_set(2, 1000, **bad)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG


def test_invalid_dimension_is_rejected(mp):
    with pytest.raises(mp.MpapError):
        mp.tuning_set(4, 1000)
