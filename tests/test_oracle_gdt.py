"""Pins of the shortest-path (geodesic) distance oracle -- Section 1's
shortest paths on a grid with obstacles, with this build's 8-move 5-7 costs
-- against facts that do not come from the oracle itself: the closed form of
the 5-7 chamfer distance on an open grid, brute-force relaxation to a
fixpoint (Bellman-Ford) on small grids with obstacles, a detour worked out
by hand, and the shortest-path optimality conditions."""
import numpy as np
import pytest

import oracle

IMAX = np.iinfo(np.int32).max


def chamfer(dy, dx):
    a, b = np.abs(dy), np.abs(dx)
    return 7 * np.minimum(a, b) + 5 * (np.maximum(a, b) - np.minimum(a, b))


def test_open_grid_closed_form():
    rng = np.random.default_rng(1)
    for h, w in ((1, 1), (1, 40), (37, 1), (23, 31), (64, 65)):
        m = np.ones((h, w), np.uint8)
        yy, xx = np.mgrid[0:h, 0:w]
        seeds = np.zeros((h, w), np.uint8)
        pts = [(0, 0), (h - 1, w - 1), (int(rng.integers(h)), int(rng.integers(w)))]
        exp = np.full((h, w), np.iinfo(np.int64).max)
        for y, x in pts:
            seeds[y, x] = 1
            exp = np.minimum(exp, chamfer(yy - y, xx - x))
        np.testing.assert_array_equal(oracle.gdt(m, seeds), exp)


@pytest.mark.parametrize("density", [0.1, 0.3, 0.5])
def test_matches_bellman_ford_with_obstacles(density):
    rng = np.random.default_rng(int(density * 100))
    for _ in range(25):
        h, w = (int(v) for v in rng.integers(1, 24, 2))
        m = (rng.random((h, w)) >= density).astype(np.uint8)
        s = (rng.random((h, w)) < 0.03).astype(np.uint8)
        np.testing.assert_array_equal(oracle.gdt(m, s), oracle.gdt_bellman_ford(m, s))


def test_detour_around_a_wall():
    # a vertical wall in column 5 with one gap at row 9; source at (0, 0)
    m = np.ones((10, 11), np.uint8)
    m[:9, 5] = 0
    s = np.zeros_like(m)
    s[0, 0] = 1
    d = oracle.gdt(m, s)
    # to the gap (9, 5): 5 diagonal + 4 straight steps = 5*7 + 4*5
    assert d[9, 5] == 55
    # just across the wall at (0, 6): from the gap 1 diagonal step to (8, 6),
    # then 8 straight steps up: 55 + 7 + 8*5
    assert d[0, 6] == 55 + 7 + 40
    assert (d[:9, 5] == IMAX).all()


def test_obstacles_unreachable_and_optimality():
    rng = np.random.default_rng(7)
    h, w = 120, 150
    m = (rng.random((h, w)) >= 0.3).astype(np.uint8)
    m[:, 70] = 0  # a full wall: the right part has no source
    s = np.zeros((h, w), np.uint8)
    s[rng.integers(0, h, 5), rng.integers(0, 60, 5)] = 1
    d = oracle.gdt(m, s).astype(np.int64)
    free = m != 0
    assert (d[~free] == IMAX).all()
    assert (d[:, 71:] == IMAX).all()
    assert (d[(s != 0) & free] == 0).all()
    fin = d < IMAX
    tight = (s != 0) & free
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            cost = 7 if dy and dx else 5
            # q = p + (dy, dx): no edge can still improve, and record which
            # finite pixels are reached exactly through some neighbour
            p = d[max(-dy, 0):h + min(-dy, 0), max(-dx, 0):w + min(-dx, 0)]
            q = d[max(dy, 0):h + min(dy, 0), max(dx, 0):w + min(dx, 0)]
            qf = free[max(dy, 0):h + min(dy, 0), max(dx, 0):w + min(dx, 0)]
            pf = fin[max(-dy, 0):h + min(-dy, 0), max(-dx, 0):w + min(-dx, 0)]
            assert not (qf & pf & (p + cost < q)).any()
            sub = tight[max(dy, 0):h + min(dy, 0), max(dx, 0):w + min(dx, 0)]
            sub |= qf & pf & (p + cost == q)
    assert (tight == fin).all()


def test_stats_count_the_work():
    m = np.ones((50, 50), np.uint8)
    s = np.zeros_like(m)
    s[25, 25] = 1
    st = {}
    oracle.gdt(m, s, stats=st)
    assert st["pops"] >= 2500 and st["improvements"] >= 2499
