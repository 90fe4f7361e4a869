"""The exact distance transform on the GPU (iwpp_edt_exact: separable
column and row passes) against the definition: squared distances
bit-identical to brute force on small images and to the oracle's exact
transform (Meijster et al.) at every size up to the 16384^2 workload; the
nearest index must be a feature at exactly that squared distance (ties
may pick any equally near feature)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import IWPPError, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
IMAX = np.iinfo(np.int32).max


def run(ctx, b, fnz=False):
    sq, nn = ctx.edt(torch.from_numpy(np.ascontiguousarray(b)).to(DEV), feature_nonzero=fnz, exact=True)
    torch.cuda.synchronize()
    return sq.cpu().numpy(), nn.cpu().numpy()


def check_nearest(b, sq, nn, fnz, sample=None):
    """nearest is a feature, at exactly the returned squared distance (on a
    seeded sample of pixels when `sample` is given)."""
    h, w = b.shape
    assert ((nn == -1) == (sq == IMAX)).all()
    if sample is None:
        yy, xx = np.nonzero(sq != IMAX)
    else:
        rng = np.random.default_rng(5)
        yy, xx = rng.integers(0, h, sample), rng.integers(0, w, sample)
        keep = sq[yy, xx] != IMAX
        yy, xx = yy[keep], xx[keep]
    idx = nn[yy, xx].astype(np.int64)
    fy, fx = idx // w, idx % w
    feat = (b != 0) if fnz else (b == 0)
    assert feat[fy, fx].all()
    assert np.array_equal((yy - fy) ** 2 + (xx - fx) ** 2, sq[yy, xx].astype(np.int64))


@pytest.mark.parametrize("fnz", [False, True])
def test_small_random_vs_bruteforce(cuda_ctx, fnz):
    rng = np.random.default_rng(700 + fnz)
    for _ in range(60):
        h, w = (int(v) for v in rng.integers(1, 90, 2))
        b = (rng.random((h, w)) < rng.random()).astype(np.uint8)
        sq, nn = run(cuda_ctx, b, fnz)
        np.testing.assert_array_equal(sq, oracle.edt_bruteforce(b, fnz))
        check_nearest(b, sq, nn, fnz)


def test_special_cases(cuda_ctx):
    sq, nn = run(cuda_ctx, np.ones((70, 300), np.uint8))  # no feature
    assert (sq == IMAX).all() and (nn == -1).all()
    sq, nn = run(cuda_ctx, np.zeros((40, 50), np.uint8))  # every pixel a feature
    assert (sq == 0).all() and (nn == np.arange(2000).reshape(40, 50)).all()
    b = np.ones((300, 257), np.uint8)
    b[299, 0] = 0  # one feature in a corner: the farthest pixel is the opposite corner
    sq, nn = run(cuda_ctx, b)
    yy, xx = np.mgrid[0:300, 0:257]
    np.testing.assert_array_equal(sq, (yy - 299) ** 2 + xx ** 2)
    assert (nn == 299 * 257).all()


@pytest.mark.parametrize("fnz", [False, True])
def test_config_4096_and_ragged(cuda_ctx, fnz):
    wl = synth.config_workload("edt4096")
    for b in (wl.binary, np.ascontiguousarray(wl.binary[:4001, :3999])):
        sq, nn = run(cuda_ctx, b, fnz)
        np.testing.assert_array_equal(sq, oracle.edt_exact(b, fnz))
        check_nearest(b, sq, nn, fnz)


def test_never_above_propagation_and_equal_off_departures(cuda_ctx):
    """The propagation result is never below the exact one and equals it
    except at its departure pixels."""
    b = synth.config_workload("edt4096", size=1500).binary
    sq_e, _ = run(cuda_ctx, b)
    sq_p, _ = cuda_ctx.edt(torch.from_numpy(b).to(DEV))
    sq_p = sq_p.cpu().numpy()
    assert (sq_p >= sq_e).all()
    assert (sq_p != sq_e).mean() < 1e-3


@pytest.mark.parametrize("fnz", [False, True])
def test_far_pixels_and_envelope_shapes(cuda_ctx, fnz):
    """Rows whose pixels lie thousands of columns from every site of the
    row: one feature in a corner (one site per row), a few scattered ones,
    a feature row far off (all sites equally far: every site is on the
    envelope), and a row band where the sites' distances vary along the
    row, with a 9000-column gap."""
    rng = np.random.default_rng(31 + fnz)
    cases = []
    b = np.zeros((600, 20000), np.uint8)
    b[599, 0] = 1
    cases.append(b)
    b = np.zeros((2000, 12000), np.uint8)
    for y, x in zip(rng.integers(0, 2000, 4), rng.integers(0, 12000, 4)):
        b[y, x] = 1
    cases.append(b)
    b = np.zeros((4400, 9001), np.uint8)
    b[0, :] = 1  # every column has a site; all at the same row offset
    cases.append(b)
    b = np.zeros((257, 16384), np.uint8)
    xs = np.arange(16384)
    ys = (128 + 120 * np.sin(xs / 900.0)).astype(int)
    keep = rng.random(16384) < 0.3
    b[ys[keep], xs[keep]] = 1
    b[:, 5000:14000] = 0  # a wide gap with no site
    cases.append(b)
    for b in cases:
        if not fnz:
            b = (1 - b).astype(np.uint8)  # features are the 0 pixels
        sq, nn = run(cuda_ctx, b, fnz)
        np.testing.assert_array_equal(sq, oracle.edt_exact(b, fnz))
        check_nearest(b, sq, nn, fnz, sample=200_000)


def test_largest_side_and_invalid(cuda_ctx):
    for shape in ((1, 32768), (32768, 1), (3, 32768)):
        rng = np.random.default_rng(sum(shape) + 1)
        b = (rng.random(shape) < 0.999).astype(np.uint8)
        b.flat[0] = 0
        sq, nn = run(cuda_ctx, b)
        np.testing.assert_array_equal(sq, oracle.edt_exact(b, False))
        check_nearest(b, sq, nn, False)
    for shape in ((1, 32769), (0, 4)):
        with pytest.raises(IWPPError):
            cuda_ctx.edt(torch.zeros(shape, dtype=torch.uint8, device=DEV), exact=True)


@pytest.mark.slow
@pytest.mark.parametrize("fnz", [False, True])
def test_full_16k(cuda_ctx, fnz):
    wl = synth.config_workload("edt16k")
    sq, nn = run(cuda_ctx, wl.binary, fnz)
    np.testing.assert_array_equal(sq, oracle.edt_exact(wl.binary, fnz))
    check_nearest(wl.binary, sq, nn, fnz, sample=2_000_000)
