"""Pins of the influence-zone / SKIZ oracle -- the skeleton by influence
zones that Section 1 names among the IWPP algorithms, defined here as the
geodesic SKIZ of labelled sources inside a mask with the shortest-path
metric (8 moves, cost 5 / 7) -- against facts that do not come from the
oracle's code: one distance map per label by relaxation to a fixpoint, the
closed form of the chamfer distance on an open grid, cases worked out by
hand, and invariants."""
import numpy as np
import pytest

import oracle

IMAX = np.iinfo(np.int32).max


def chamfer(dy, dx):
    a, b = np.abs(dy), np.abs(dx)
    return 7 * np.minimum(a, b) + 5 * (np.maximum(a, b) - np.minimum(a, b))


def _labels(rng, h, w, k, values=5):
    lab = np.zeros((h, w), np.int32)
    for _ in range(k):
        lab[rng.integers(0, h), rng.integers(0, w)] = rng.integers(1, values + 1)
    return lab


@pytest.mark.parametrize("density", [0.0, 0.2, 0.45])
def test_matches_per_label_distance_maps(density):
    rng = np.random.default_rng(int(density * 100) + 1)
    for _ in range(40):
        h, w = (int(v) for v in rng.integers(1, 20, 2))
        m = (rng.random((h, w)) >= density).astype(np.uint8)
        lab = _labels(rng, h, w, int(rng.integers(0, 7)))
        z, s, d = oracle.skiz(m, lab)
        z2, s2, d2 = oracle.skiz_per_label(m, lab)
        np.testing.assert_array_equal(d, d2)
        np.testing.assert_array_equal(z, z2)
        np.testing.assert_array_equal(s, s2)


def test_open_grid_closed_form():
    rng = np.random.default_rng(2)
    for h, w in ((1, 30), (23, 1), (19, 27), (40, 33)):
        lab = _labels(rng, h, w, 6, values=4)
        yy, xx = np.mgrid[0:h, 0:w]
        ys, xs = np.nonzero(lab)
        vals = np.unique(lab[ys, xs])
        per = np.stack([np.min(np.stack([chamfer(yy - y, xx - x) for y, x in zip(ys, xs) if lab[y, x] == L]),
                               axis=0) for L in vals])
        best = per.min(axis=0)
        reach = per == best
        z, s, d = oracle.skiz(np.ones((h, w), np.uint8), lab)
        np.testing.assert_array_equal(d, best)
        np.testing.assert_array_equal(z, vals[np.argmax(reach, axis=0)])
        np.testing.assert_array_equal(s, (reach.sum(axis=0) >= 2).astype(np.uint8))


def test_worked_by_hand():
    # two sources on a row: the midpoint is equally near both
    m = np.ones((1, 9), np.uint8)
    lab = np.zeros((1, 9), np.int32)
    lab[0, 0], lab[0, 8] = 1, 2
    z, s, d = oracle.skiz(m, lab)
    np.testing.assert_array_equal(z[0], [1, 1, 1, 1, 1, 2, 2, 2, 2])
    np.testing.assert_array_equal(s[0], [0, 0, 0, 0, 1, 0, 0, 0, 0])
    np.testing.assert_array_equal(d[0], [0, 5, 10, 15, 20, 15, 10, 5, 0])
    # a wall down column 5 with one gap in the bottom row: zones follow the
    # geodesic distance, and the gap is equally near both sources
    m = np.ones((7, 11), np.uint8)
    m[:6, 5] = 0
    lab = np.zeros((7, 11), np.int32)
    lab[0, 0], lab[0, 10] = 4, 3
    z, s, d = oracle.skiz(m, lab)
    assert (z[:, :5] == 4).all() and (z[:, 6:] == 3).all()
    assert z[6, 5] == 3 and s[6, 5] == 1 and s.sum() == 1
    assert d[6, 5] == 5 * 7 + 5  # from (0, 0): five diagonal steps and one straight
    assert (z[:6, 5] == 0).all() and (d[:6, 5] == IMAX).all()


def test_degenerate_and_invariants():
    m = np.ones((5, 6), np.uint8)
    z, s, d = oracle.skiz(m, np.zeros((5, 6), np.int32))
    assert (z == 0).all() and (s == 0).all() and (d == IMAX).all()
    # a label on an obstacle is no source
    lab = np.zeros((5, 6), np.int32)
    lab[2, 2] = 7
    m0 = m.copy()
    m0[2, 2] = 0
    z, s, d = oracle.skiz(m0, lab)
    assert (z == 0).all()
    rng = np.random.default_rng(9)
    m = (rng.random((60, 70)) >= 0.3).astype(np.uint8)
    lab = _labels(rng, 60, 70, 25, values=9)
    z, s, d = oracle.skiz(m, lab)
    src = (m != 0) & (lab != 0)
    np.testing.assert_array_equal(z[src], lab[src])
    assert (s[src] == 0).all() and (z[m == 0] == 0).all() and (s[m == 0] == 0).all()
    assert ((z == 0) == (d == IMAX)).all()
