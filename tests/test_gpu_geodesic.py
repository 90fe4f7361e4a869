"""Shortest paths on a grid with obstacles (iwpp_geodesic), the further IWPP
use of Section 1, on the GPU through the C ABI against the Dijkstra oracle:
distances are exact integers, so every comparison is bit-exact -- random
obstacle fields of ragged sizes spanning many tiles, a serpentine maze whose
single path crosses every tile row many times, the open grid, degenerate
cases, and every sweep / queue setting."""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import IWPPError

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
IMAX = np.iinfo(np.int32).max


def run(ctx, mask, seeds, **opts):
    if opts:
        old = ctx.options()
        ctx.set_options(**opts)
    try:
        d = ctx.geodesic(torch.from_numpy(np.ascontiguousarray(mask)).to(DEV),
                         torch.from_numpy(np.ascontiguousarray(seeds)).to(DEV))
        torch.cuda.synchronize()
        return d.cpu().numpy()
    finally:
        if opts:
            ctx.set_options(**old)


def field(rng, h, w, density, nseeds):
    m = (rng.random((h, w)) >= density).astype(np.uint8)
    s = np.zeros((h, w), np.uint8)
    s[rng.integers(0, h, nseeds), rng.integers(0, w, nseeds)] = 1
    return m, s


def serpentine(h, w, pitch=6):
    """Horizontal walls every `pitch` rows, each open at alternating ends:
    one path snakes through the whole image."""
    m = np.ones((h, w), np.uint8)
    for k, r in enumerate(range(pitch, h, pitch)):
        m[r, :] = 0
        if k % 2 == 0:
            m[r, w - 2:] = 1
        else:
            m[r, :2] = 1
    s = np.zeros((h, w), np.uint8)
    s[0, 0] = 1
    return m, s


def test_small_random_fields(cuda_ctx):
    rng = np.random.default_rng(90)
    for _ in range(40):
        h, w = (int(v) for v in rng.integers(1, 200, 2))
        m, s = field(rng, h, w, float(rng.uniform(0, 0.5)), int(rng.integers(0, 6)))
        np.testing.assert_array_equal(run(cuda_ctx, m, s), oracle.gdt(m, s))


@pytest.mark.parametrize("density", [0.0, 0.25, 0.4])
def test_many_tiles_ragged(cuda_ctx, density):
    rng = np.random.default_rng(int(density * 100) + 1)
    m, s = field(rng, 1111, 1333, density, 7)
    np.testing.assert_array_equal(run(cuda_ctx, m, s), oracle.gdt(m, s))


def test_long_valid_call_outlasts_the_wait_bound(cuda_ctx):
    """The device-side bound (timeout_ms) is on a wait that sees no progress,
    not on the work: a 2048^2 serpentine maze, whose one corridor is walked
    by thousands of tile visits in sequence, runs about ten times longer than
    timeout_ms = 50 and still completes with the exact result."""
    import time

    m, s = serpentine(2048, 2048)
    ref = oracle.gdt(m, s)
    old = cuda_ctx.options()
    cuda_ctx.set_options(timeout_ms=50)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = run(cuda_ctx, m, s)
        elapsed = time.perf_counter() - t0
    finally:
        cuda_ctx.set_options(**old)
    assert elapsed > 0.05
    np.testing.assert_array_equal(got, ref)


def test_serpentine_maze_crosses_every_tile_repeatedly(cuda_ctx):
    m, s = serpentine(700, 900)
    ref = oracle.gdt(m, s)
    assert 100000 < ref[m != 0].max() < IMAX  # every free pixel on one long path
    np.testing.assert_array_equal(run(cuda_ctx, m, s), ref)


def test_open_grid_closed_form(cuda_ctx):
    h, w = 300, 410
    m = np.ones((h, w), np.uint8)
    s = np.zeros((h, w), np.uint8)
    s[123, 321] = 1
    yy, xx = np.mgrid[0:h, 0:w]
    a, b = np.abs(yy - 123), np.abs(xx - 321)
    np.testing.assert_array_equal(run(cuda_ctx, m, s),
                                  7 * np.minimum(a, b) + 5 * (np.maximum(a, b) - np.minimum(a, b)))


def test_degenerate_cases(cuda_ctx):
    m = np.ones((150, 170), np.uint8)
    assert (run(cuda_ctx, m, np.zeros_like(m)) == IMAX).all()  # no source
    z = np.zeros((150, 170), np.uint8)
    assert (run(cuda_ctx, z, np.ones_like(z)) == IMAX).all()  # all obstacles
    one = np.ones((1, 1), np.uint8)
    assert run(cuda_ctx, one, one)[0, 0] == 0
    # a source on an obstacle is no source
    s = np.zeros_like(m)
    s[5, 5] = 1
    m2 = m.copy()
    m2[5, 5] = 0
    d = run(cuda_ctx, m2, s)
    assert (d == IMAX).all()


@pytest.mark.parametrize("sweeps,revisit_min,mode", [(0, 0, 0), (1, 0, 1), (3, 1 << 20, 2), (12, 16, 3)])
def test_settings_do_not_change_the_result(cuda_ctx, sweeps, revisit_min, mode):
    rng = np.random.default_rng(95)
    m, s = field(rng, 520, 610, 0.3, 4)
    ref = oracle.gdt(m, s)
    got = run(cuda_ctx, m, s, gdt_sweeps=sweeps, gdt_revisit_sweep_min=revisit_min, queue_mode=mode)
    np.testing.assert_array_equal(got, ref)


def test_invalid_arguments(cuda_ctx):
    a = torch.ones((8, 8), dtype=torch.uint8, device=DEV)
    with pytest.raises(IWPPError):
        cuda_ctx.geodesic(a, torch.ones((8, 9), dtype=torch.uint8, device=DEV))
    with pytest.raises(IWPPError):
        cuda_ctx.geodesic(a.to(torch.int32), a)
    with pytest.raises(IWPPError):
        cuda_ctx.geodesic(torch.ones((0, 8), dtype=torch.uint8, device=DEV),
                          torch.ones((0, 8), dtype=torch.uint8, device=DEV))


@pytest.mark.slow
def test_4096_random_obstacles(cuda_ctx):
    rng = np.random.default_rng(97)
    m, s = field(rng, 4096, 4096, 0.3, 20)
    np.testing.assert_array_equal(run(cuda_ctx, m, s), oracle.gdt(m, s))
