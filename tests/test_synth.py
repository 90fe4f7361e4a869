"""The seeded input generators: deterministic, right shapes and value
ranges, coverage targets met."""
import numpy as np

from paper_1209_3314_gb300 import synth


def test_blurred_noise_deterministic_and_full_range():
    a = synth.blurred_noise_u8(200, 150, 4.0, seed=1)
    b = synth.blurred_noise_u8(200, 150, 4.0, seed=1)
    c = synth.blurred_noise_u8(200, 150, 4.0, seed=2)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.dtype == np.uint8 and a.min() == 0 and a.max() == 255


def test_threaded_blur_matches_single_strip():
    x = np.random.default_rng(0).random((1200, 1000))
    from scipy.ndimage import correlate1d

    k = synth._gauss_kernel(3.0)
    ref = correlate1d(correlate1d(x, k, axis=1, mode="reflect"), k, axis=0, mode="reflect")
    got = synth._blur_axis(synth._blur_axis(x, 3.0, 1), 3.0, 0)
    np.testing.assert_array_equal(got, ref)


def test_recon_inputs_marker_below_mask():
    marker, mask = synth.recon_inputs(64, 80, 2.0, 40, seed=3)
    assert (marker <= mask).all()
    np.testing.assert_array_equal(marker, np.maximum(mask.astype(int) - 40, 0))


def test_disks_coverage():
    img, n = synth.disks_binary(512, 512, 4, 40, 0.3, seed=4)
    assert set(np.unique(img)) <= {0, 1}
    assert 0.3 <= img.mean() < 0.32 and n > 10


def test_batched_workloads_shapes():
    wls = synth.batched_workloads(n=6, seed=9, smin=32, smax=64)
    assert [w.op for w in wls] == ["recon", "edt"] * 3
    for w in wls:
        assert 32 <= w.h <= 64 and 32 <= w.w <= 64


def test_tissue_region_coverage_and_shape():
    for h, w in ((1000, 777), (64, 5000)):
        for cov in (0.25, 0.5, 0.75):
            r = synth.tissue_region(h, w, cov, seed=11)
            assert r.shape == (h, w) and r.dtype == bool
            # cells are taken whole: the overshoot is below one cell's pixels
            cell_px = -(-h // 256) * -(-w // 256)
            assert cov * h * w <= r.sum() <= cov * h * w + cell_px
        assert synth.tissue_region(h, w, 1.0, seed=11).all()
    a = synth.tissue_region(512, 512, 0.5, seed=3)
    b = synth.tissue_region(512, 512, 0.5, seed=3)
    assert np.array_equal(a, b)
    # blob-shaped: most region pixels have their right neighbour in the region
    assert (a[:, 1:] & a[:, :-1]).sum() > 0.9 * a[:, 1:].sum()


def test_apply_tissue_zeroes_the_background():
    marker, mask = synth.recon_inputs(300, 200, 4.0, 40, seed=5)
    r = synth.tissue_region(300, 200, 0.5, seed=6)
    m2, k2 = synth.apply_tissue(marker, mask, r)
    assert m2.dtype == np.uint8 and k2.dtype == np.uint8
    assert (m2[~r] == 0).all() and (k2[~r] == 0).all()
    assert np.array_equal(m2[r], marker[r]) and np.array_equal(k2[r], mask[r])


def test_grid_markers():
    m = synth.grid_markers(130, 97, 32, 7)
    # one marker per 32x32 cell (clipped at the image edge), labels 1..k in
    # row-major cell order
    cells = ((130 + 31) // 32) * ((97 + 31) // 32)
    ys, xs = np.nonzero(m)
    assert len(ys) == cells and m.dtype == np.int32
    np.testing.assert_array_equal(np.sort(m[ys, xs]), np.arange(1, cells + 1))
    for y, x in zip(ys, xs):
        cy, cx = y // 32, x // 32
        assert m[y, x] == cy * ((97 + 31) // 32) + cx + 1
    np.testing.assert_array_equal(m, synth.grid_markers(130, 97, 32, 7))
