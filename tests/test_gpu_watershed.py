"""Watershed from markers (iwpp_watershed), the IWPP use of Section 1, on the
GPU through the C ABI against the oracle (Dijkstra flooding, breadth-first
plateau distances, per-label search): labels and flooding levels are
unique, so every comparison is bit-exact -- uint8 and int32 reliefs of
ragged sizes spanning many tiles, reliefs with few levels (wide plateaus
crossing tile borders), a serpentine plateau, constant reliefs, pitched and
unaligned inputs, degenerate cases and every sweep / queue setting."""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import IWPPError, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
IMAX = np.iinfo(np.int32).max


def run(ctx, relief, markers, **opts):
    if opts:
        old = ctx.options()
        ctx.set_options(**opts)
    try:
        f = torch.from_numpy(np.ascontiguousarray(relief)).to(DEV)
        m = torch.from_numpy(np.ascontiguousarray(markers)).to(DEV)
        lab, lev = ctx.watershed(f, m, with_levels=True)
        torch.cuda.synchronize()
        return lab.cpu().numpy(), lev.cpu().numpy()
    finally:
        if opts:
            ctx.set_options(**old)


def random_markers(rng, h, w, k, labels=50):
    m = np.zeros((h, w), np.int32)
    m[rng.integers(0, h, k), rng.integers(0, w, k)] = rng.integers(1, labels + 1, k)
    return m


def check(ctx, relief, markers, **opts):
    lab, lev = run(ctx, relief, markers, **opts)
    elab, elev = oracle.watershed(relief, markers)
    np.testing.assert_array_equal(lev, elev)
    np.testing.assert_array_equal(lab, elab)


@pytest.mark.parametrize("levels", [2, 5, 256])
def test_small_random_u8(cuda_ctx, levels):
    rng = np.random.default_rng(100 + levels)
    for _ in range(25):
        h, w = (int(v) for v in rng.integers(1, 230, 2))
        f = rng.integers(0, levels, (h, w)).astype(np.uint8)
        check(cuda_ctx, f, random_markers(rng, h, w, int(rng.integers(1, 12))))


def test_blurred_relief_ragged(cuda_ctx):
    for k, (h, w) in enumerate(((333, 517), (64, 64), (65, 129), (1, 700), (700, 1), (257, 255))):
        f = synth.blurred_noise_u8(h, w, 4.0, 110 + k)
        check(cuda_ctx, f, synth.grid_markers(h, w, 37, 120 + k))


def test_int32_relief(cuda_ctx):
    rng = np.random.default_rng(130)
    for _ in range(10):
        h, w = (int(v) for v in rng.integers(1, 200, 2))
        f = rng.choice(np.array([np.iinfo(np.int32).min, -7, 0, 3, 1 << 20, IMAX], np.int32), (h, w))
        check(cuda_ctx, f, random_markers(rng, h, w, int(rng.integers(1, 8)), labels=1 << 30))
    f = (synth.blurred_noise_u8(300, 280, 3.0, 131).astype(np.int32) - 128) * 1000003
    check(cuda_ctx, f, synth.grid_markers(300, 280, 25, 132))


def test_constant_relief_plateau_across_tiles(cuda_ctx):
    rng = np.random.default_rng(140)
    f = np.full((300, 410), 17, np.uint8)
    check(cuda_ctx, f, random_markers(rng, 300, 410, 7, labels=4))
    # a single marker: one label, and the plateau spans every tile
    m = np.zeros((300, 410), np.int32)
    m[299, 0] = 9
    lab, lev = run(cuda_ctx, f, m)
    assert (lab == 9).all() and (lev == 17).all()


def test_serpentine_plateau(cuda_ctx):
    # low corridors (value 10) behind high walls (200) that open at
    # alternating ends: one winding plateau whose breadth-first distance
    # crosses every tile row many times; markers at both ends of the path
    h, w = 260, 200
    f = np.full((h, w), 10, np.uint8)
    for k, r in enumerate(range(5, h, 5)):
        f[r, :] = 200
        if k % 2 == 0:
            f[r, w - 2:] = 10
        else:
            f[r, :2] = 10
    m = np.zeros((h, w), np.int32)
    m[0, 0] = 1
    m[h - 1, 0 if len(range(5, h, 5)) % 2 == 1 else w - 1] = 2  # the far end of the path
    check(cuda_ctx, f, m)


def test_pitched_and_unaligned(cuda_ctx):
    rng = np.random.default_rng(150)
    big = synth.blurred_noise_u8(301, 333, 3.0, 151)
    bigm = random_markers(rng, 301, 333, 40)
    f = torch.from_numpy(big).to(DEV)[1:, 3:330]  # odd offset: plain staging
    m = torch.from_numpy(bigm).to(DEV)[1:, 3:330]
    lab, lev = cuda_ctx.watershed(f, m, with_levels=True)
    elab, elev = oracle.watershed(big[1:, 3:330].copy(), bigm[1:, 3:330].copy())
    np.testing.assert_array_equal(lev.cpu().numpy(), elev)
    np.testing.assert_array_equal(lab.cpu().numpy(), elab)
    # labels only (no levels output)
    lab2 = cuda_ctx.watershed(f, m)
    np.testing.assert_array_equal(lab2.cpu().numpy(), elab)


def test_degenerate(cuda_ctx):
    f = synth.blurred_noise_u8(90, 70, 2.0, 160)
    lab, lev = run(cuda_ctx, f, np.zeros((90, 70), np.int32))
    assert (lab == 0).all() and (lev == 255).all()
    lab, lev = run(cuda_ctx, f.astype(np.int32), np.zeros((90, 70), np.int32))
    assert (lab == 0).all() and (lev == IMAX).all()
    check(cuda_ctx, np.array([[3]], np.uint8), np.array([[5]], np.int32))
    every = np.arange(1, 90 * 70 + 1, dtype=np.int32).reshape(90, 70)
    lab, lev = run(cuda_ctx, f, every)
    np.testing.assert_array_equal(lab, every)
    np.testing.assert_array_equal(lev, f)
    # negative labels are labels too
    rng = np.random.default_rng(161)
    m = random_markers(rng, 90, 70, 9) - 30
    m[m == -30] = 0
    check(cuda_ctx, f, m)


@pytest.mark.parametrize("opts", [dict(ws_sweeps=0), dict(ws_sweeps=1), dict(ws_sweeps=16),
                                  dict(ws_revisit_sweep_min=8), dict(ws_revisit_sweep_min=10 ** 6),
                                  dict(queue_mode=1), dict(queue_mode=2), dict(queue_mode=3),
                                  dict(spill_cap=0), dict(blocks_per_sm=1)])
def test_settings(cuda_ctx, opts):
    f = synth.blurred_noise_u8(400, 380, 3.0, 170)
    f = (f // 16).astype(np.uint8)  # 16 levels: wide plateaus
    check(cuda_ctx, f, synth.grid_markers(400, 380, 45, 171), **opts)


def test_invalid_arguments(cuda_ctx):
    f = torch.zeros((10, 10), dtype=torch.uint8, device=DEV)
    m = torch.zeros((10, 10), dtype=torch.int32, device=DEV)
    with pytest.raises(IWPPError):
        cuda_ctx.watershed(f, m.to(torch.uint8))
    with pytest.raises(IWPPError):
        cuda_ctx.watershed(f, torch.zeros((10, 11), dtype=torch.int32, device=DEV))
    with pytest.raises(IWPPError):
        cuda_ctx.watershed(f, m, labels=m)  # labels alias the markers


@pytest.mark.slow
def test_4096_blurred(cuda_ctx):
    f = synth.blurred_noise_u8(4096, 4096, 8.0, 180)
    check(cuda_ctx, f, synth.grid_markers(4096, 4096, 64, 181))


def _shift(x, dy, dx, fill):
    """out[y, x] = x[y + dy, x + dx]; fill outside the image."""
    h, w = x.shape
    out = torch.full_like(x, fill)
    out[max(-dy, 0):h + min(-dy, 0), max(-dx, 0):w + min(-dx, 0)] = \
        x[max(dy, 0):h + min(dy, 0), max(dx, 0):w + min(dx, 0)]
    return out


OFF8 = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dy or dx]


def test_separates_touching_disks(cuda_ctx):
    """The use the paper's distance transform serves (Section 2.2): split
    overlapping disks by a watershed of the negated distance map, from
    markers at the distance maxima.  The relief comes from the library's
    own distance transform; labels and levels must equal the oracle's on
    that relief."""
    from scipy import ndimage

    b, _ = synth.disks_binary(384, 320, 6, 20, 0.3, 240)
    sq, _ = cuda_ctx.edt(torch.from_numpy(b).to(DEV), feature_nonzero=False)
    torch.cuda.synchronize()
    d = sq.cpu().numpy()
    relief = np.where(b != 0, -d, 0).astype(np.int32)
    peaks = (b != 0) & (d == ndimage.maximum_filter(d, size=5)) & (d > 4)
    markers, n = ndimage.label(peaks, structure=np.ones((3, 3), bool))
    markers = markers.astype(np.int32)
    markers[b == 0] = n + 1  # the background is one more basin
    lab, lev = run(cuda_ctx, relief, markers)
    elab, elev = oracle.watershed(relief, markers)
    np.testing.assert_array_equal(lev, elev)
    np.testing.assert_array_equal(lab, elab)
    assert len(np.unique(lab[b != 0])) >= n // 2  # the disks are split into many regions


@pytest.mark.slow
def test_16384_certificates(cuda_ctx):
    """Full size, the bench's workload shape (16384^2 blurred relief, one
    marker per 64x64 cell), through certificates that have one solution
    each, checked with torch on the device:
    - levels: level = relief at markers, and elsewhere level = max(relief,
      least neighbour level), whose only solution is the flooding level;
    - plateau distances, computed here by Jacobi iteration: 0 at entry
      pixels, else 1 + least equal-level neighbour distance;
    - labels: markers keep theirs, every other pixel holds the least label
      of its optimal in-neighbours (the optimal edges raise (level,
      plateau distance), so this recursion has one solution)."""
    side = 16384
    f = torch.from_numpy(synth.blurred_noise_u8(side, side, 16.0, 190)).to(DEV)
    m = torch.from_numpy(synth.grid_markers(side, side, 64, 191)).to(DEV)
    lab, lev = cuda_ctx.watershed(f, m, with_levels=True)
    torch.cuda.synchronize()
    big = 1 << 30
    c, fi, mk = lev.to(torch.int32), f.to(torch.int32), m != 0
    del lev
    assert bool((c >= fi).all()) and bool((c[mk] == fi[mk]).all())
    least = torch.full_like(c, big)
    for dy, dx in OFF8:
        torch.minimum(least, _shift(c, dy, dx, big), out=least)
    assert bool((c == torch.where(mk, fi, torch.maximum(fi, least))).all())
    entry = mk | (least < c)
    del least, fi
    d = torch.where(entry, 0, big).to(torch.int32)
    same = [_shift(c, dy, dx, -1) == c for dy, dx in OFF8]
    for _ in range(side * side):
        best = d.clone()
        for (dy, dx), s in zip(OFF8, same):
            torch.minimum(best, torch.where(s, _shift(d, dy, dx, big) + 1, big), out=best)
        if torch.equal(best, d):
            break
        d = best
    del same
    assert int(d.max()) < big  # every pixel reached
    want = torch.full_like(lab, np.iinfo(np.int32).max)
    for dy, dx in OFF8:
        nc = _shift(c, dy, dx, big)
        opt = ((nc < c) & (d == 0)) | ((nc == c) & (_shift(d, dy, dx, -2) + 1 == d))
        torch.minimum(want, torch.where(opt, _shift(lab, dy, dx, 0), np.iinfo(np.int32).max), out=want)
    want = torch.where(mk, m, want)
    assert torch.equal(lab, want)
