"""Influence zones and their skeleton (iwpp_skiz), an IWPP use of Section 1,
on the GPU through the C ABI against the oracle (Dijkstra, then per-label
searches along shortest-path edges): zones, skeleton and distances are
unique, so every comparison is bit-exact -- random obstacle fields of
ragged sizes, the open grid, a serpentine corridor, pitched inputs,
degenerate cases and every sweep / queue setting."""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import IWPPError

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
IMAX = np.iinfo(np.int32).max


def run(ctx, mask, labels, **opts):
    if opts:
        old = ctx.options()
        ctx.set_options(**opts)
    try:
        z, s, d = ctx.skiz(torch.from_numpy(np.ascontiguousarray(mask)).to(DEV),
                           torch.from_numpy(np.ascontiguousarray(labels)).to(DEV), with_dist=True)
        torch.cuda.synchronize()
        return z.cpu().numpy(), s.cpu().numpy(), d.cpu().numpy()
    finally:
        if opts:
            ctx.set_options(**old)


def check(ctx, mask, labels, **opts):
    z, s, d = run(ctx, mask, labels, **opts)
    ez, es, ed = oracle.skiz(mask, labels)
    np.testing.assert_array_equal(d, ed)
    np.testing.assert_array_equal(z, ez)
    np.testing.assert_array_equal(s, es)
    return z, s


def field(rng, h, w, density, k, values=20):
    m = (rng.random((h, w)) >= density).astype(np.uint8)
    lab = np.zeros((h, w), np.int32)
    lab[rng.integers(0, h, k), rng.integers(0, w, k)] = rng.integers(1, values + 1, k)
    return m, lab


def test_small_random_fields(cuda_ctx):
    rng = np.random.default_rng(200)
    for _ in range(40):
        h, w = (int(v) for v in rng.integers(1, 220, 2))
        check(cuda_ctx, *field(rng, h, w, float(rng.uniform(0, 0.45)), int(rng.integers(1, 12))))


def test_open_grid_many_ties(cuda_ctx):
    # an even grid of sources: many pixels lie equally near two or more
    h, w = 300, 333
    m = np.ones((h, w), np.uint8)
    lab = np.zeros((h, w), np.int32)
    k = 1
    for y in range(5, h, 40):
        for x in range(7, w, 40):
            lab[y, x] = k
            k += 1
    z, s = check(cuda_ctx, m, lab)
    assert s.sum() > 0


def test_serpentine_corridor(cuda_ctx):
    h, w = 250, 190
    m = np.ones((h, w), np.uint8)
    for k, r in enumerate(range(6, h, 6)):
        m[r, :] = 0
        if k % 2 == 0:
            m[r, w - 2:] = 1
        else:
            m[r, :2] = 1
    lab = np.zeros((h, w), np.int32)
    lab[0, 0], lab[h - 1, 0], lab[120, 90] = 3, 1, 2
    check(cuda_ctx, m, lab)


def test_pitched_and_negative_labels(cuda_ctx):
    rng = np.random.default_rng(210)
    m, lab = field(rng, 301, 333, 0.25, 30)
    lab = np.where(lab != 0, lab - 10, 0).astype(np.int32)  # includes negative labels
    dm = torch.from_numpy(m).to(DEV)[1:, 3:330]
    dl = torch.from_numpy(lab).to(DEV)[1:, 3:330]
    z, s, d = cuda_ctx.skiz(dm, dl, with_dist=True)
    ez, es, ed = oracle.skiz(m[1:, 3:330].copy(), lab[1:, 3:330].copy())
    np.testing.assert_array_equal(d.cpu().numpy(), ed)
    np.testing.assert_array_equal(z.cpu().numpy(), ez)
    np.testing.assert_array_equal(s.cpu().numpy(), es)
    z2, s2 = cuda_ctx.skiz(dm, dl)  # without the distance output
    np.testing.assert_array_equal(z2.cpu().numpy(), ez)


def test_degenerate(cuda_ctx):
    m = np.ones((70, 90), np.uint8)
    z, s, d = run(cuda_ctx, m, np.zeros((70, 90), np.int32))
    assert (z == 0).all() and (s == 0).all() and (d == IMAX).all()
    z, s, d = run(cuda_ctx, np.zeros((70, 90), np.uint8), np.ones((70, 90), np.int32))
    assert (z == 0).all() and (s == 0).all() and (d == IMAX).all()
    check(cuda_ctx, np.ones((1, 1), np.uint8), np.array([[5]], np.int32))
    every = np.arange(1, 70 * 90 + 1, dtype=np.int32).reshape(70, 90)
    z, s, d = run(cuda_ctx, m, every)
    np.testing.assert_array_equal(z, every)
    assert (s == 0).all() and (d == 0).all()


@pytest.mark.parametrize("opts", [dict(ws_sweeps=0), dict(ws_sweeps=2), dict(gdt_sweeps=1),
                                  dict(ws_revisit_sweep_min=16), dict(gdt_revisit_sweep_min=0),
                                  dict(queue_mode=3), dict(spill_cap=0)])
def test_settings(cuda_ctx, opts):
    rng = np.random.default_rng(220)
    check(cuda_ctx, *field(rng, 400, 390, 0.3, 60), **opts)


def test_invalid_arguments(cuda_ctx):
    m = torch.ones((10, 10), dtype=torch.uint8, device=DEV)
    lab = torch.zeros((10, 10), dtype=torch.int32, device=DEV)
    with pytest.raises(IWPPError):
        cuda_ctx.skiz(m, lab.to(torch.uint8))
    with pytest.raises(IWPPError):
        cuda_ctx.skiz(m.to(torch.int32), lab)
    with pytest.raises(IWPPError):
        cuda_ctx.skiz(m, torch.zeros((10, 11), dtype=torch.int32, device=DEV))


@pytest.mark.slow
def test_4096_field(cuda_ctx):
    rng = np.random.default_rng(230)
    check(cuda_ctx, *field(rng, 4096, 4096, 0.3, 512, values=400))
