"""Pins of the watershed oracle -- the marker-controlled watershed by
flooding that Section 1 names as an IWPP algorithm, defined here as the
image foresting transform with the highest-value path cost, plateau
distances and least-label ties -- against facts that do not come from the
oracle's code: threshold decomposition of the flooding levels (connected
components per level), relaxation of the plateau distances to a fixpoint,
per-label reachability along optimal edges, the closed form on a constant
relief (Chebyshev distance to the markers), profiles worked out by hand and
structural invariants of the partition."""
import numpy as np
import pytest

import oracle

IMAX = np.iinfo(np.int32).max


def _markers(rng, h, w, k, labels=5):
    m = np.zeros((h, w), np.int32)
    for _ in range(k):
        m[rng.integers(0, h), rng.integers(0, w)] = rng.integers(1, labels + 1)
    return m


@pytest.mark.parametrize("levels", [2, 4, 256])
def test_matches_independent_restatements(levels):
    rng = np.random.default_rng(levels)
    for _ in range(60):
        h, w = (int(v) for v in rng.integers(1, 22, 2))
        f = rng.integers(0, levels, (h, w)).astype(np.uint8)
        m = _markers(rng, h, w, int(rng.integers(1, 7)))
        label, level, pdist = oracle.watershed(f, m, with_pdist=True)
        t = oracle.watershed_levels_threshold(f, m)
        np.testing.assert_array_equal(level.astype(np.int64), t)
        pr = oracle.watershed_pdist_relax(t, m)
        np.testing.assert_array_equal(pdist.astype(np.int64), pr)
        np.testing.assert_array_equal(label, oracle.watershed_labels_reach(t, pr, m))


def test_int32_relief_full_range():
    rng = np.random.default_rng(11)
    for _ in range(40):
        h, w = (int(v) for v in rng.integers(1, 18, 2))
        f = rng.choice(np.array([np.iinfo(np.int32).min, -5, 0, 7, IMAX], np.int32), (h, w))
        m = _markers(rng, h, w, int(rng.integers(1, 5)), labels=1000)
        label, level, pdist = oracle.watershed(f, m, with_pdist=True)
        t = oracle.watershed_levels_threshold(f, m)
        np.testing.assert_array_equal(level.astype(np.int64), t)
        pr = oracle.watershed_pdist_relax(t, m)
        np.testing.assert_array_equal(label, oracle.watershed_labels_reach(t, pr, m))


def test_constant_relief_is_chebyshev_voronoi():
    # one level everywhere: the entry set is the markers, the plateau
    # distance is the Chebyshev distance to the nearest marker, and a pixel
    # takes the least label among the markers at that distance
    rng = np.random.default_rng(3)
    for h, w in ((1, 30), (17, 1), (25, 31), (40, 40)):
        f = np.full((h, w), 9, np.uint8)
        m = _markers(rng, h, w, 6, labels=4)
        yy, xx = np.mgrid[0:h, 0:w]
        ys, xs = np.nonzero(m)
        cheb = np.maximum(np.abs(yy[..., None] - ys), np.abs(xx[..., None] - xs))
        dmin = cheb.min(axis=-1)
        lab = np.where(cheb == dmin[..., None], m[ys, xs], np.iinfo(np.int32).max).min(axis=-1)
        label, level, pdist = oracle.watershed(f, m, with_pdist=True)
        assert (level == 9).all()
        np.testing.assert_array_equal(pdist, dmin)
        np.testing.assert_array_equal(label, np.where(m != 0, m, lab))


@pytest.mark.parametrize("f, m, exp_label, exp_level", [
    # a plateau between two basins is split at its middle; the middle pixel
    # (equally far from both entries) takes the smaller label
    ([0, 5, 5, 5, 5, 5, 0], [1, 0, 0, 0, 0, 0, 2], [1, 1, 1, 1, 2, 2, 2], [0, 5, 5, 5, 5, 5, 0]),
    # an even plateau splits evenly
    ([0, 5, 5, 5, 5, 0], [3, 0, 0, 0, 0, 4], [3, 3, 3, 4, 4, 4], [0, 5, 5, 5, 5, 0]),
    # a ridge pixel reached from both sides at once takes the smaller label
    ([0, 5, 9, 5, 0], [2, 0, 0, 0, 1], [2, 2, 1, 1, 1], [0, 5, 9, 5, 0]),
    # a basin without a marker floods to its spill level and is split like
    # a plateau
    ([0, 3, 1, 3, 0], [1, 0, 0, 0, 2], [1, 1, 1, 2, 2], [0, 3, 3, 3, 0]),
    # each basin keeps its own marker's label below the pass; the pass
    # pixel, entered from both sides, takes the smaller label
    ([2, 1, 0, 6, 4, 4], [0, 0, 7, 0, 0, 5], [7, 7, 7, 5, 5, 5], [2, 1, 0, 6, 4, 4]),
    # the higher marker floods nothing below it
    ([0, 1, 8, 1, 0], [0, 0, 9, 0, 0], [9, 9, 9, 9, 9], [8, 8, 8, 8, 8]),
])
def test_profiles_worked_by_hand(f, m, exp_label, exp_level):
    f = np.array([f], np.uint8)
    m = np.array([m], np.int32)
    label, level = oracle.watershed(f, m)
    np.testing.assert_array_equal(label[0], exp_label)
    np.testing.assert_array_equal(level[0], exp_level)
    # the same profile as a column
    label_t, level_t = oracle.watershed(f.T.copy(), m.T.copy())
    np.testing.assert_array_equal(label_t[:, 0], exp_label)
    np.testing.assert_array_equal(level_t[:, 0], exp_level)


def test_two_basins_in_two_dimensions():
    # two cones with a ridge along the middle column; each marker owns its
    # half, the ridge (equal level from both sides) goes to the smaller label
    yy, xx = np.mgrid[0:9, 0:11]
    f = np.minimum(np.abs(xx - 2), np.abs(xx - 8)).astype(np.uint8)
    m = np.zeros_like(f, np.int32)
    m[4, 2] = 6
    m[4, 8] = 3
    label, level = oracle.watershed(f, m)
    assert (label[:, :5] == 6).all() and (label[:, 6:] == 3).all()
    assert (label[:, 5] == 3).all()
    np.testing.assert_array_equal(level, f)


def test_without_markers_and_degenerate():
    f = np.arange(12, dtype=np.uint8).reshape(3, 4)
    label, level, pdist = oracle.watershed(f, np.zeros((3, 4), np.int32), with_pdist=True)
    assert (label == 0).all() and (level == 255).all() and (pdist == IMAX).all()
    label, level = oracle.watershed(f.astype(np.int32), np.zeros((3, 4), np.int32))
    assert (level == IMAX).all()
    # one pixel
    label, level = oracle.watershed(np.array([[4]], np.uint8), np.array([[8]], np.int32))
    assert label[0, 0] == 8 and level[0, 0] == 4
    # every pixel a marker: nothing changes
    rng = np.random.default_rng(5)
    m = rng.integers(1, 9, (6, 7)).astype(np.int32)
    f = rng.integers(0, 256, (6, 7)).astype(np.uint8)
    label, level = oracle.watershed(f, m)
    np.testing.assert_array_equal(label, m)
    np.testing.assert_array_equal(level, f)


def test_partition_invariants():
    from scipy import ndimage

    rng = np.random.default_rng(9)
    noise = ndimage.gaussian_filter(rng.random((160, 190)), 3)
    f = np.round(255 * (noise - noise.min()) / (noise.max() - noise.min())).astype(np.uint8)
    m = _markers(rng, 160, 190, 40, labels=25)
    label, level = oracle.watershed(f, m)
    assert (level >= f).all()
    np.testing.assert_array_equal(level[m != 0], f[m != 0])
    np.testing.assert_array_equal(label[m != 0], m[m != 0])
    assert (label != 0).all()
    # every region is 8-connected and holds a marker of its label: each
    # connected piece of {label == L} contains a marker pixel of value L
    for L in np.unique(label):
        pieces, n = ndimage.label(label == L, structure=np.ones((3, 3), bool))
        has = np.zeros(n + 1, bool)
        has[pieces[(m == L)]] = True
        assert has[1:].all(), L
    # a single marker floods everything
    one = np.zeros_like(m)
    one[80, 90] = 4
    assert (oracle.watershed(f, one)[0] == 4).all()
