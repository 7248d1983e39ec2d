"""GPU roadmap construction (Alg. 2 + per-edge transfers) vs the oracle: the
node states and the whole CSR, bit for bit."""
import numpy as np
import pytest

import scenegen
from _gpu import assert_reverse_is_transpose, assert_same_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_1705_02408_gb300 import build
    build.build()
    import paper_1705_02408_gb300 as m
    return m


@pytest.mark.parametrize("name,seed,n,r", [
    ("2d", 1, 1000, None), ("2d", 2, 1000, None), ("2d", 3, 257, 0.2),
    ("3d", 1, 2000, None), ("3d", 4, 777, 0.2),
    ("6d", 1, 2000, None), ("6d", 5, 1500, 20.0),
    ("2d", 6, 2000, 0.2),    # mean degree ~250: rows overflow the 128-edge scratch rows
    ("3d", 8, 3000, 0.3),
])
def test_roadmap_matches_oracle(mp, orc, name, seed, n, r):
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r)
    ro = orc.build_roadmap(sc, n=n, r=r)
    assert_same_graph(rg.export(), ro.graph())
    assert_reverse_is_transpose(rg)


def test_roadmap_device_inputs(mp, orc):
    sc = scenegen.make_scene("3d", 9)
    rg = mp.build_roadmap_for_scene(sc, n=1200, device_inputs=True)
    ro = orc.build_roadmap(sc, n=1200)
    assert_same_graph(rg.export(), ro.graph())


def test_roadmap_from_points(mp, orc):
    rng = np.random.default_rng(3)
    sc = scenegen.make_scene("2d", 4)
    x = np.zeros((6, 300), np.float32)
    x[:2] = rng.random((2, 300)).astype(np.float32)
    x[:2, 0] = 0.05; x[:2, 1] = 0.95
    ro = orc.build_roadmap_from_points(2, sc.box_lo, sc.box_hi, sc.grid, 64, x, r=0.15)
    rg = mp.build_roadmap_from_points(2, sc.box_lo, sc.box_hi, sc.grid, 64, x, r=0.15)
    assert_same_graph(rg.export(), ro.graph())


def test_roadmap_edge_cases(mp, orc):
    # no obstacles, tiny n, ragged tiles (n + 2 not a multiple of 256 or 8)
    sc = scenegen.make_scene("2d", 1)
    sc.box_lo = np.zeros((0, 3), np.float32); sc.box_hi = np.zeros((0, 3), np.float32)
    sc.cfg = scenegen.config("2d", nb=0)
    for n in (1, 7, 255, 263):
        rg = mp.build_roadmap_for_scene(sc, n=n, r=0.3)
        ro = orc.build_roadmap(sc, n=n, r=0.3)
        assert_same_graph(rg.export(), ro.graph())
        assert_reverse_is_transpose(rg)
    # radius too small for any edge
    rg = mp.build_roadmap_for_scene(sc, n=50, r=1e-6)
    assert rg.E == 0
    assert_reverse_is_transpose(rg)


def test_roadmap_full_size_6d(mp, orc):
    """The 6D double-integrator roadmap at full size (16000 samples), as timed by
    the benchmark, compared edge for edge."""
    sc = scenegen.make_scene("6d", 1, query_id=1)
    rg = mp.build_roadmap_for_scene(sc)
    ro = orc.build_roadmap(sc)
    assert_same_graph(rg.export(), ro.graph())
    assert_reverse_is_transpose(rg)


def test_batched_build_and_handle_reuse(mp, orc):
    """mpap_build_roadmaps: mixed dimensions in one call, then a rebuild of the
    same handles with other scenes and sizes (smaller and larger)."""
    first = [("2d", 1, 1000, None), ("3d", 2, 1500, None), ("6d", 3, 2000, None), ("2d", 4, 300, 0.2)]
    second = [("6d", 5, 2500, None), ("2d", 6, 200, 0.2), ("3d", 7, 3000, None), ("6d", 8, 700, 20.0)]
    rms = None
    for batch in (first, second):
        scenes = [scenegen.make_scene(nm, sd, query_id=sd) for nm, sd, _, _ in batch]
        specs = [mp.scene_spec(sc, n=n, r=r) for sc, (_, _, n, r) in zip(scenes, batch)]
        rms = mp.build_roadmaps(specs, rms=rms)
        for sc, rg, (_, _, n, r) in zip(scenes, rms, batch):
            assert_same_graph(rg.export(), orc.build_roadmap(sc, n=n, r=r).graph())
            assert_reverse_is_transpose(rg)


def test_reverse_csr_of_a_given_graph(mp, orc):
    """mpap_roadmap_from_csr derives the reverse CSR with its own kernels
    (in-degree count, scan, fill): also the exact transpose."""
    from _search_ref import random_graph
    rng = np.random.default_rng(77)
    for V in (1, 5, 40, 300):
        g = random_graph(rng, V, p_edge=0.3 if V < 100 else 0.05, dmax=4)
        assert_reverse_is_transpose(mp.roadmap_from_csr(*g))


@pytest.mark.parametrize("name,seed,n,r,M", [
    # M inc max(n_f, K - n_f) >= 2^31: 64-bit transfer sums
    ("6d", 1, 1200, None, 44),    # one edge's S is exactly -2^31
    ("6d", 2, 1200, None, 44),
    ("2d", 2, 800, 0.3, 40),      # transfers up to 2.04e9
    # below the bound: 32-bit sums
    ("3d", 3, 1200, None, 8),
    ("6d", 3, 1200, None, 16),
    # 6D checkpoint levels packed by the collision test (m = 1..16 below M)
    ("6d", 3, 1200, None, 1),     # no interior checkpoint
    ("6d", 3, 1200, None, 5),
    ("6d", 3, 1200, None, 17),    # all 16 packed, the endpoint computed
])
def test_transfer_sums_both_widths(mp, orc, name, seed, n, r, M):
    """The per-edge transfer runs in 32-bit integers only where its partial sums
    provably fit; either width gives the oracle's 64-bit values, up to the int32
    limits of the stored fields."""
    sc = scenegen.make_scene(name, seed, query_id=seed)
    rg = mp.build_roadmap_for_scene(sc, n=n, r=r, M=M)
    g = orc.build_roadmap(sc, n=n, r=r, M=M).graph()
    assert_same_graph(rg.export(), g)
    np.testing.assert_array_equal(np.stack(rg.peaks()), np.stack([g.Smax, g.Cmax]))


@pytest.mark.parametrize("name,seed,n,r,M", [("6d", 4, 1200, None, 44), ("2d", 2, 800, 0.3, 64)])
def test_transfer_beyond_int32_fails_like_the_oracle(mp, orc, name, seed, n, r, M):
    """An edge whose transfer does not fit the int32 fields fails the build
    (MPAP_ERR_CAPACITY) exactly where the oracle's construction fails."""
    sc = scenegen.make_scene(name, seed, query_id=seed)
    with pytest.raises(RuntimeError):
        orc.build_roadmap(sc, n=n, r=r, M=M)
    with pytest.raises(mp.MpapError) as e:
        mp.build_roadmap_for_scene(sc, n=n, r=r, M=M)
    assert e.value.status == mp.MPAP_ERR_CAPACITY


def test_level_above_K_is_rejected(mp):
    """Quality levels lie in 0..K: a grid cell at K + 1 fails the build with
    MPAP_ERR_INVALID_ARG; the top level K itself is accepted."""
    sc = scenegen.make_scene("6d", 3, query_id=3)
    K = 24
    sc.grid = sc.grid.copy()
    sc.grid.reshape(-1)[777] = K
    mp.build_roadmap_for_scene(sc, n=300)
    sc.grid.reshape(-1)[777] = K + 1
    with pytest.raises(mp.MpapError) as e:
        mp.build_roadmap_for_scene(sc, n=300)
    assert e.value.status == mp.MPAP_ERR_INVALID_ARG


@pytest.mark.parametrize("name,nb,seed,n", [("2d", 33, 3, 900), ("3d", 40, 5, 1500), ("6d", 48, 6, 1500),
                                            ("6d", 32, 7, 1500), ("3d", 1, 8, 1200)])
def test_box_counts_around_the_prefilter_limit(mp, orc, name, nb, seed, n):
    """Scenes of at most 32 boxes take the collision prefilter table, larger ones
    the pass over every box: the edge set is the oracle's either way."""
    sc = scenegen.make_scene(scenegen.config(name, nb=nb), seed, query_id=seed)
    assert len(sc.box_lo) == nb
    rg = mp.build_roadmap_for_scene(sc, n=n)
    assert_same_graph(rg.export(), orc.build_roadmap(sc, n=n).graph())
    assert_reverse_is_transpose(rg)
