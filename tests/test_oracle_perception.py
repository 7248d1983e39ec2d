"""Oracle pins of the visible-feature perception levels (the feature count behind
the Sec. 4.1 heuristic): range, horizontal field of view, occlusion by a box
and the cap at K, each against hand-computed tables."""
import numpy as np

import scenegen

NOBOX = np.zeros((0, 3), np.float32)


def test_unobstructed_full_view_counts_every_feature(orc):
    rng = np.random.default_rng(1)
    for F, K, want in ((10, 24, 10), (40, 24, 24), (40, 5, 5), (0, 24, 0)):
        f = np.zeros((F, 3), np.float32)
        f[:, :2] = rng.random((F, 2))
        lv = orc.feature_levels(2, NOBOX, NOBOX, f, 8, range_=2.0, K=K)
        assert lv.shape == (1, 64) and (lv == want).all()


def test_a_wall_box_hides_the_features_behind_it(orc):
    lo = np.array([[0.45, 0.0, 0.0]], np.float32)
    hi = np.array([[0.55, 1.0, 1.0]], np.float32)
    f = np.array([[0.8, y, 0.0] for y in (0.1, 0.3, 0.5, 0.7, 0.9)], np.float32)
    lv = orc.feature_levels(2, lo, hi, f, 8, range_=2.0).reshape(8, 8)   # [y][x]
    xc = (2 * np.arange(8) + 1) / 16.0
    want = np.where(xc > 0.55, 5, 0)
    for row in lv:
        np.testing.assert_array_equal(row, want)
    # 3D: the same wall spanning the cube
    f3 = np.array([[0.8, 0.5, z] for z in (0.2, 0.5, 0.8)], np.float32)
    lv3 = orc.feature_levels(3, lo, hi, f3, 4, range_=2.0).reshape(4, 4, 4)   # [z][y][x]
    xc4 = (2 * np.arange(4) + 1) / 8.0
    assert (lv3 == np.where(xc4 > 0.55, 3, 0)[None, None, :]).all()


def test_field_of_view_and_range():
    import oracle as orc
    f = np.array([[0.9, 0.5, 0.0]], np.float32)
    heads = np.array([[1, 0], [0, 1], [-1, 0]], np.float32)
    # G = 2: cell centres (0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)
    lv = orc.feature_levels(2, NOBOX, NOBOX, f, 2, heads, np.float32(np.cos(np.pi / 6)), 2.0)
    np.testing.assert_array_equal(lv[0], [1, 0, 1, 0])      # 21 deg off the x axis in, 59 deg out
    np.testing.assert_array_equal(lv[2], [0, 0, 0, 0])      # looking away
    lv = orc.feature_levels(2, NOBOX, NOBOX, f, 2, heads, np.float32(0.5), 2.0)
    np.testing.assert_array_equal(lv[1], [0, 1, 0, 0])      # 31 deg off +y in, 69 deg out, behind out
    # range 0.3: only the cells 0.29 away see the feature
    lv = orc.feature_levels(2, NOBOX, NOBOX, f, 2, range_=0.3)
    np.testing.assert_array_equal(lv[0], [0, 1, 0, 1])
    # a 90-degree half-angle keeps the half-plane ahead, boundary included
    g = np.array([[0.25, 0.9, 0.0]], np.float32)          # straight above cell (0.25, 0.25)
    lv = orc.feature_levels(2, NOBOX, NOBOX, g, 2, heads[:1], np.float32(0.0), 2.0)
    assert lv[0, 0] == 1 and lv[0, 1] == 0


def test_features_sit_off_their_surfaces(orc):
    sc = scenegen.make_scene("3d", 4, query_id=4)
    f = scenegen.feature_points(sc, 200)
    assert f.shape == (200, 3) and f.dtype == np.float32
    assert ((f >= 0) & (f <= 1)).all()
    inside = ((f[:, None, :] > sc.box_lo[None]) & (f[:, None, :] < sc.box_hi[None])).all(-1)
    assert not inside.any()
    np.testing.assert_array_equal(f, scenegen.feature_points(sc, 200))     # seeded
    h = scenegen.yaw_headings(8)
    np.testing.assert_allclose((h.astype(np.float64) ** 2).sum(1), 1.0, atol=1e-6)


def test_field_of_view_in_3d_is_horizontal(orc):
    """The field of view is a horizontal cone: a feature straight above a cell
    centre (no horizontal offset) passes every heading; one off to the side counts
    only for headings within the half-angle of its horizontal direction, whatever
    its height; range uses the full 3D distance."""
    import oracle
    heads = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], np.float32)
    narrow = np.float32(np.cos(np.radians(10)))
    above = np.array([[0.25, 0.25, 0.95]], np.float32)       # over cell (0.25, 0.25, 0.25)
    lv = oracle.feature_levels(3, NOBOX, NOBOX, above, 2, heads, narrow, 2.0)
    assert (lv[:, 0] == 1).all()
    side = np.array([[0.95, 0.25, 0.75]], np.float32)        # +x of cell 0, 45 deg up
    lv = oracle.feature_levels(3, NOBOX, NOBOX, side, 2, heads, narrow, 2.0)
    np.testing.assert_array_equal(lv[:, 0], [1, 0, 0, 0])
    # |d| = sqrt(0.7^2 + 0.5^2) = 0.86: out at range 0.8, in at range 0.9
    assert oracle.feature_levels(3, NOBOX, NOBOX, side, 2, heads[:1], narrow, 0.8)[0, 0] == 0
    assert oracle.feature_levels(3, NOBOX, NOBOX, side, 2, heads[:1], narrow, 0.9)[0, 0] == 1
