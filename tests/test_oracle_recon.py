"""Pins of the reconstruction oracle (Algorithm 2, FH) against things other
than itself: the Section 2.1 definition run by brute force, threshold
decomposition with connected-component labelling, invariants and special
cases with closed-form answers."""
import numpy as np
import pytest

import oracle
from paper_1209_3314_gb300 import synth


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("levels", [4, 8, 256])
def test_fh_equals_bruteforce_tiny_u8(conn, levels):
    rng = np.random.default_rng(100 + conn + levels)
    for _ in range(150):
        h, w = rng.integers(1, 17, 2)
        I = rng.integers(0, levels, (h, w)).astype(np.uint8)
        J = rng.integers(0, levels, (h, w)).astype(np.uint8)  # marker may exceed mask
        np.testing.assert_array_equal(oracle.fh(J, I, conn), oracle.recon_bruteforce(J, I, conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_fh_equals_bruteforce_tiny_i32_full_range(conn):
    rng = np.random.default_rng(7 + conn)
    lo, hi = np.iinfo(np.int32).min, np.iinfo(np.int32).max
    for _ in range(100):
        h, w = rng.integers(1, 13, 2)
        I = rng.integers(lo, hi, (h, w), dtype=np.int64, endpoint=True).astype(np.int32)
        J = (I.astype(np.int64) - rng.integers(0, 2**31, (h, w))).clip(lo, hi).astype(np.int32)
        np.testing.assert_array_equal(oracle.fh(J, I, conn), oracle.recon_bruteforce(J, I, conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_fh_equals_threshold_decomposition_512(conn):
    wl = synth.config_workload("recon512")
    out = oracle.fh(wl.marker, wl.mask, conn)
    np.testing.assert_array_equal(out, oracle.recon_threshold_decomposition(wl.marker, wl.mask, conn))


def test_fh_equals_threshold_decomposition_smooth_1024():
    marker, mask = synth.recon_inputs(1024, 768, 8.0, 60, seed=55)
    out = oracle.fh(marker, mask, 8)
    np.testing.assert_array_equal(out, oracle.recon_threshold_decomposition(marker, mask, 8))


@pytest.mark.parametrize("conn", [4, 8])
def test_invariants_and_idempotence(conn):
    marker, mask = synth.recon_inputs(300, 257, 4.0, 40, seed=9)
    out = oracle.fh(marker, mask, conn)
    assert (np.minimum(marker, mask) <= out).all() and (out <= mask).all()
    np.testing.assert_array_equal(oracle.fh(out, mask, conn), out)
    assert oracle.recon_unstable_pairs(out, mask, conn) == 0


def test_special_cases():
    rng = np.random.default_rng(3)
    mask = rng.integers(0, 256, (40, 33)).astype(np.uint8)
    # marker = mask -> mask
    np.testing.assert_array_equal(oracle.fh(mask, mask, 8), mask)
    # marker = 0 -> 0
    np.testing.assert_array_equal(oracle.fh(np.zeros_like(mask), mask, 8), np.zeros_like(mask))
    # constant mask c, marker below it with maximum m -> m everywhere
    m = np.full((25, 31), 200, np.uint8)
    j = rng.integers(0, 150, m.shape).astype(np.uint8)
    np.testing.assert_array_equal(oracle.fh(j, m, 4), np.full(m.shape, j.max(), np.uint8))
    # 1-D row: each pixel gets the largest marker value reachable through a
    # path whose mask stays at or above it (closed form via running minima)
    I = np.array([[5, 9, 3, 8, 8, 2, 7]], np.uint8)
    J = np.array([[0, 6, 0, 0, 7, 0, 1]], np.uint8)
    exp = np.array([[5, 6, 3, 7, 7, 2, 2]], np.uint8)
    np.testing.assert_array_equal(oracle.fh(J, I, 8), exp)


def test_diagonal_connectivity_matters():
    # a diagonal chain of bright mask pixels carries the marker only under
    # 8-connectivity
    I = np.zeros((5, 5), np.uint8)
    for k in range(5):
        I[k, k] = 100
    J = np.zeros_like(I)
    J[0, 0] = 90
    out8 = oracle.fh(J, I, 8)
    out4 = oracle.fh(J, I, 4)
    assert out8[4, 4] == 90 and out4[4, 4] == 0 and out4[0, 0] == 90


def test_queue_counters_reported():
    st = {}
    wl = synth.config_workload("recon512")
    oracle.fh(wl.marker, wl.mask, 8, stats=st)
    assert 0 < st["initial"] <= st["pushes"]
