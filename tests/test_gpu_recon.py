"""Reconstruction on the GPU through the C ABI, bit-exact against the CPU
oracle (Algorithm 2) on seeded inputs: tiny and ragged images, several
tiles, both connectivities, uint8 and int32, in place and pitched, forced
queue overflow / spill / rescan paths, and the full 16384^2 workload."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import IWPPError, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run(ctx, marker, mask, conn=8, **opts):
    if opts:
        old = ctx.options()
        ctx.set_options(**opts)
    try:
        out = ctx.recon(gpu(marker), gpu(mask), conn=conn)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        if opts:
            ctx.set_options(**old)


def test_golden_small_cases(cuda_ctx):
    with open(os.path.join(GOLDEN, "recon_small.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        I = np.array(c["mask"], np.uint8)
        J = np.array(c["marker"], np.uint8)
        np.testing.assert_array_equal(run(cuda_ctx, J, I, 8), np.array(c["out8"], np.uint8))
        np.testing.assert_array_equal(run(cuda_ctx, J, I, 4), np.array(c["out4"], np.uint8))


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("dtype", [np.uint8, np.int32])
@pytest.mark.parametrize("sweeps", [0, 1])
def test_random_ragged(cuda_ctx, conn, dtype, sweeps):
    rng = np.random.default_rng(1000 + conn + 7 * sweeps + (dtype == np.int32))
    for _ in range(12):
        h, w = (int(v) for v in rng.integers(1, 200, 2))
        if dtype == np.uint8:
            I = rng.integers(0, 256, (h, w)).astype(np.uint8)
            J = rng.integers(0, 256, (h, w)).astype(np.uint8)  # exceeds the mask in places
        else:
            I = rng.integers(-2**31, 2**31 - 1, (h, w), dtype=np.int64).astype(np.int32)
            J = (I.astype(np.int64) - rng.integers(0, 2**31, (h, w))).clip(-2**31, 2**31 - 1).astype(np.int32)
        np.testing.assert_array_equal(run(cuda_ctx, J, I, conn, sweeps=sweeps), oracle.fh(J, I, conn))


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_config_512(cuda_ctx, conn, sweeps):
    wl = synth.config_workload("recon512")
    np.testing.assert_array_equal(run(cuda_ctx, wl.marker, wl.mask, conn, sweeps=sweeps),
                                  oracle.fh(wl.marker, wl.mask, conn))


def test_config_4096_and_int32_variant(cuda_ctx):
    wl = synth.config_workload("recon4096")
    ref = oracle.fh(wl.marker, wl.mask, 8)
    np.testing.assert_array_equal(run(cuda_ctx, wl.marker, wl.mask, 8), ref)
    # int32: the same values widened and shifted into the negative range
    J = wl.marker.astype(np.int32) * 1000 - 70000
    I = wl.mask.astype(np.int32) * 1000 - 70000
    np.testing.assert_array_equal(run(cuda_ctx, J, I, 8), ref.astype(np.int32) * 1000 - 70000)


@pytest.mark.parametrize("sweeps,revisit_sweeps,revisit_min",
                         [(0, -1, 0), (1, -1, 0), (3, -1, 0), (3, 0, 0), (3, 1, 0), (2, 2, 1 << 20)])
def test_sweep_count_does_not_change_result(cuda_ctx, sweeps, revisit_sweeps, revisit_min):
    marker, mask = synth.recon_inputs(700, 513, 6.0, 50, seed=21)
    got = run(cuda_ctx, marker, mask, 8, sweeps=sweeps, revisit_sweeps=revisit_sweeps,
              revisit_sweep_min=revisit_min)
    np.testing.assert_array_equal(got, oracle.fh(marker, mask, 8))


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_queue_modes_give_the_same_result(cuda_ctx, mode):
    """The queue-ablation modes (per-thread atomics, global-only queue)
    change how items are queued, never the result; no sweeps, so the queue
    carries the whole propagation."""
    marker, mask = synth.recon_inputs(700, 513, 6.0, 50, seed=22)
    for conn in (4, 8):
        got = run(cuda_ctx, marker, mask, conn, queue_mode=mode, sweeps=0)
        np.testing.assert_array_equal(got, oracle.fh(marker, mask, conn))
    J = marker.astype(np.int32) * 7 - 900
    I = mask.astype(np.int32) * 7 - 900
    np.testing.assert_array_equal(run(cuda_ctx, J, I, 8, queue_mode=mode, sweeps=1),
                                  oracle.fh(marker, mask, 8).astype(np.int32) * 7 - 900)


def test_in_place_and_pitched(cuda_ctx):
    marker, mask = synth.recon_inputs(333, 301, 4.0, 40, seed=8)
    ref = oracle.fh(marker, mask, 8)
    m = gpu(marker)
    cuda_ctx.recon(m, gpu(mask), conn=8, out=m)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(m.cpu().numpy(), ref)
    # pitched views: rows of a wider buffer
    big_m = torch.zeros((333, 400), dtype=torch.uint8, device=DEV)
    big_k = torch.zeros((333, 352), dtype=torch.uint8, device=DEV)
    big_o = torch.full((333, 384), 7, dtype=torch.uint8, device=DEV)
    big_m[:, :301] = gpu(marker)
    big_k[:, 17:318] = gpu(mask)
    out = cuda_ctx.recon(big_m[:, :301], big_k[:, 17:318], conn=8, out=big_o[:, 50:351])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    assert (big_o[:, :50] == 7).all() and (big_o[:, 351:] == 7).all()


@pytest.mark.parametrize("dtype", [np.uint8, np.int32])
def test_tma_path_with_ragged_width(cuda_ctx, dtype):
    """Row pitches that meet TMA alignment (multiple of 16 bytes) with image
    widths that are not a multiple of the tile: boxes run past the image."""
    marker, mask = synth.recon_inputs(700, 1000, 6.0, 50, seed=31)
    if dtype == np.int32:
        marker, mask = marker.astype(np.int32) * 7 - 900, mask.astype(np.int32) * 7 - 900
    ref = oracle.fh(marker, mask, 8)
    pitch = 1008
    bm = torch.zeros((700, pitch), dtype=torch.from_numpy(marker).dtype, device=DEV)
    bk = torch.zeros_like(bm)
    bo = torch.zeros_like(bm)
    bm[:, :1000] = gpu(marker)
    bk[:, :1000] = gpu(mask)
    out = cuda_ctx.recon(bm[:, :1000], bk[:, :1000], conn=8, out=bo[:, :1000])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    assert (bo[:, 1000:] == 0).all()


def test_forced_tile_queue_overflow_relaunch(cuda_ctx):
    """Section 3.2 / 5.2.4: a queue too small to hold the work drops items;
    relaunching from the partial result gives the identical output."""
    marker, mask = synth.recon_inputs(1024, 1024, 8.0, 60, seed=5)
    ref = oracle.fh(marker, mask, 8)
    cuda_ctx.stats_reset()
    out = run(cuda_ctx, marker, mask, 8, queue_factor=1, max_relaunch=60)
    np.testing.assert_array_equal(out, ref)
    assert cuda_ctx.stats()["relaunches"] > 0


def test_overflow_limit_reports_error(cuda_ctx):
    marker, mask = synth.recon_inputs(1024, 1024, 8.0, 60, seed=5)
    old = cuda_ctx.options()
    cuda_ctx.set_options(queue_factor=1, max_relaunch=0)
    try:
        with pytest.raises(IWPPError) as e:
            cuda_ctx.recon(gpu(marker), gpu(mask), conn=8)
        assert e.value.code == -5
    finally:
        cuda_ctx.set_options(**old)
    # the context stays usable
    np.testing.assert_array_equal(run(cuda_ctx, marker, mask, 8), oracle.fh(marker, mask, 8))


def test_spill_and_rescan_paths(cuda_ctx):
    rng = np.random.default_rng(44)
    mask = rng.integers(0, 256, (256, 320)).astype(np.uint8)
    marker = np.maximum(mask.astype(np.int16) - 50, 0).astype(np.uint8)
    ref = oracle.fh(marker, mask, 8)
    for spill in (0, 64, 4096):
        cuda_ctx.stats_reset()
        np.testing.assert_array_equal(run(cuda_ctx, marker, mask, 8, sweeps=0, spill_cap=spill), ref)
        st = cuda_ctx.stats()
        if spill == 0:
            assert st["rescans"] > 0
        if spill == 64:
            assert st["spills"] > 0


def test_degenerate_shapes_and_values(cuda_ctx):
    rng = np.random.default_rng(2)
    for h, w in ((1, 1), (1, 97), (97, 1), (2, 2), (65, 1), (1, 65)):
        I = rng.integers(0, 256, (h, w)).astype(np.uint8)
        J = rng.integers(0, 256, (h, w)).astype(np.uint8)
        for conn in (4, 8):
            np.testing.assert_array_equal(run(cuda_ctx, J, I, conn), oracle.fh(J, I, conn))
    I = rng.integers(0, 256, (150, 170)).astype(np.uint8)
    np.testing.assert_array_equal(run(cuda_ctx, I, I, 8), I)
    np.testing.assert_array_equal(run(cuda_ctx, np.zeros_like(I), I, 8), np.zeros_like(I))
    c = np.full((150, 170), 200, np.uint8)
    j = rng.integers(0, 150, c.shape).astype(np.uint8)
    np.testing.assert_array_equal(run(cuda_ctx, j, c, 8), np.full(c.shape, j.max(), np.uint8))


def test_extreme_aspect_ratios(cuda_ctx):
    """One row or one column of thousands of tiles (ragged last tile)."""
    rng = np.random.default_rng(3)
    for h, w in ((1, 200_003), (200_003, 1), (3, 70_001)):
        I = rng.integers(0, 256, (h, w)).astype(np.uint8)
        J = np.maximum(I.astype(np.int16) - rng.integers(0, 60, (h, w)), 0).astype(np.uint8)
        for conn in (4, 8):
            np.testing.assert_array_equal(run(cuda_ctx, J, I, conn), oracle.fh(J, I, conn))


@pytest.mark.parametrize("cov", [0.25, 0.6])
def test_partial_tissue_coverage(cuda_ctx, cov):
    """Tissue-masked images (background 0 in marker and mask), the kind the
    coverage benchmark times."""
    marker, mask = synth.recon_inputs(1500, 1300, 8.0, 50, seed=31)
    marker, mask = synth.apply_tissue(marker, mask, synth.tissue_region(1500, 1300, cov, seed=32))
    for conn in (4, 8):
        np.testing.assert_array_equal(run(cuda_ctx, marker, mask, conn), oracle.fh(marker, mask, conn))


def test_device_wait_timeout_is_reported_and_the_context_stays_usable(cuda_ctx):
    """Failure detection without a fault: one initial tile-queue slot is left
    empty, so one claim waits until the (short) deadline runs out; every CTA
    ends within its own deadline, the call returns ETIMEOUT, and the next
    call on the same context is correct."""
    import time

    marker, mask = synth.recon_inputs(600, 700, 6.0, 50, seed=42)
    old = cuda_ctx.options()
    cuda_ctx.set_options(timeout_ms=200, test_empty_slot=1)
    try:
        t0 = time.perf_counter()
        with pytest.raises(IWPPError) as e:
            run(cuda_ctx, marker, mask, 8)
        assert e.value.code == -4
        assert time.perf_counter() - t0 < 30.0
    finally:
        cuda_ctx.set_options(**old)
    np.testing.assert_array_equal(run(cuda_ctx, marker, mask, 8), oracle.fh(marker, mask, 8))
    b = (synth.disks_binary(300, 300, 4, 20, 0.3, seed=43)[0])
    sq, nn = cuda_ctx.edt(torch.from_numpy(b).to(DEV))
    assert sq.cpu().numpy().max() > 0


def test_empty_images_are_rejected(cuda_ctx):
    for shape in ((0, 5), (5, 0), (0, 0)):
        a = torch.zeros(shape, dtype=torch.uint8, device=DEV)
        with pytest.raises(IWPPError) as e:
            cuda_ctx.recon(a, a.clone(), out=torch.zeros(shape, dtype=torch.uint8, device=DEV))
        assert e.value.code == -1


def test_invalid_arguments_raise(cuda_ctx):
    a = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    b = torch.zeros((8, 9), dtype=torch.uint8, device=DEV)
    with pytest.raises(IWPPError):
        cuda_ctx.recon(a, a.clone(), conn=6)
    with pytest.raises(IWPPError):
        cuda_ctx.recon(a, b)
    m = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    with pytest.raises(IWPPError):
        cuda_ctx.recon(a, m, out=m)
    with pytest.raises(IWPPError):
        cuda_ctx.recon(a, torch.zeros((8, 8), dtype=torch.int32, device=DEV))


def test_async_calls_then_sync(cuda_ctx):
    marker, mask = synth.recon_inputs(512, 600, 4.0, 40, seed=12)
    ref = oracle.fh(marker, mask, 8)
    outs = [cuda_ctx.recon(gpu(marker), gpu(mask), conn=8, sync=False) for _ in range(3)]
    cuda_ctx.sync()
    for o in outs:
        np.testing.assert_array_equal(o.cpu().numpy(), ref)


@pytest.mark.slow
def test_full_16k(cuda_ctx):
    """The 16384^2 workload in the configuration the benchmark times,
    compared pixel for pixel with the oracle (and its int32 variant)."""
    wl = synth.config_workload("recon16k")
    ref = oracle.fh(wl.marker, wl.mask, 8)
    np.testing.assert_array_equal(run(cuda_ctx, wl.marker, wl.mask, 8), ref)
    J = wl.marker.astype(np.int32) - 128
    I = wl.mask.astype(np.int32) - 128
    np.testing.assert_array_equal(run(cuda_ctx, J, I, 8), ref.astype(np.int32) - 128)
