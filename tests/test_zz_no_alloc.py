"""The allocation-free reconstruction entry point (iwpp_recon_u8_noalloc).

It serves callers that cannot allocate device memory -- code running inside
another allocator's accounting, and real-time paths that forbid allocation
after start-up -- by keeping its scratch in a static array inside the
library.  The tests call it through the C ABI several times in a row on
different inputs (a later call must not see anything left over in the
shared scratch by an earlier one) and compare every result bit for bit with
the CPU oracle (Algorithm 2) and with the context-based entry point
iwpp_recon: reconstruction is exact, so the tolerance is zero.  They cover
conn 4 and 8, out of place and in place, and a corridor maze whose tile
visits exceed the scratch's tile queue, so that its device-side relaunch
runs.  The file sorts last so that a run stopping at the first failure has
run everything else.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import Context, IWPPError, synth
from paper_1209_3314_gb300.binding import recon_u8_noalloc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1209_3314_gb300 import build

    build.build()
    c = Context(0)
    yield c
    c.close()


def corridor_maze(h, w, period, seed):
    """A grayscale corridor maze: wall rows every `period` rows, each open at
    alternating ends, corridor values in 100..255 and the marker non-zero at
    the corridor's start only (equal to the mask there).  The wavefront must follow the corridor, which
    crosses every tile row period-fold, so tiles are visited many times."""
    rng = np.random.default_rng(seed)
    mask = rng.integers(100, 256, size=(h, w), dtype=np.uint8)
    for k, r in enumerate(range(period - 1, h, period)):
        mask[r, :] = 0
        if k % 2 == 0:
            mask[r, w - 2:] = 200
        else:
            mask[r, :2] = 200
    marker = np.zeros_like(mask)
    marker[0, 0] = mask[0, 0]
    return marker, mask


def run_noalloc(marker, mask, conn, in_place, dev):
    m = torch.from_numpy(marker).to(dev)
    k = torch.from_numpy(mask).to(dev)
    if in_place:
        out = recon_u8_noalloc(m, k, conn=conn, out=m)
        assert out.data_ptr() == m.data_ptr()
    else:
        out = torch.full_like(k, 255)  # caller-owned output, garbage to start
        recon_u8_noalloc(m, k, conn=conn, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    # (seed, h, w, sigma, h-offset, conn, in place)
    (77, 1000, 1200, 8.0, 60, 8, False),
    (78, 700, 1333, 8.0, 60, 4, False),
    (79, 513, 1000, 4.0, 40, 8, True),
    (80, 1024, 777, 4.0, 40, 4, True),
]


def test_noalloc_matches_oracle_and_context_on_calls_in_a_row(ctx):
    dev = torch.device("cuda:0")
    for seed, h, w, sigma, off, conn, in_place in CASES:
        marker, mask = synth.recon_inputs(h, w, sigma, off, seed=seed)
        ref = oracle.fh(marker, mask, conn)
        got = run_noalloc(marker, mask, conn, in_place, dev)
        assert np.array_equal(got, ref), (seed, conn, in_place)
        via_ctx = ctx.recon(torch.from_numpy(marker).to(dev), torch.from_numpy(mask).to(dev), conn=conn)
        assert np.array_equal(via_ctx.cpu().numpy(), got)


def test_noalloc_full_size_and_relaunch_on_shared_scratch(ctx):
    dev = torch.device("cuda:0")
    # a 4096^2 image of the 4096^2 reconstruction workload (sigma 8, h 60)
    marker, mask = synth.recon_inputs(4096, 4096, 8.0, 60, seed=1001)
    ref = oracle.fh(marker, mask, 8)
    assert np.array_equal(run_noalloc(marker, mask, 8, False, dev), ref)
    # a corridor maze: 341 corridor segments, each crossing the 16 tiles of
    # its tile row in turn, so about 20 visits per tile -- more than the
    # scratch's 16 tile-queue slots per tile: the call runs a relaunch
    for conn, in_place in ((8, False), (4, True)):
        marker, mask = corridor_maze(1024, 1024, 3, seed=81 + conn)
        ref = oracle.fh(marker, mask, conn)
        assert np.array_equal(run_noalloc(marker, mask, conn, in_place, dev), ref), (conn, in_place)
    # the same maze through a context with the scratch's queue settings
    # does overflow its tile queue: the relaunch path is the one exercised
    saved = ctx.options()
    try:
        ctx.set_options(queue_factor=16, max_relaunch=4)
        ctx.stats_reset()
        m = torch.from_numpy(marker).to(dev)
        out = ctx.recon(m, torch.from_numpy(mask).to(dev), conn=4)
        assert ctx.stats()["relaunches"] >= 1
        assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        ctx.set_options(**saved)


def test_noalloc_rejects_bad_arguments(ctx):
    dev = torch.device("cuda:0")
    w = 64 * 65537  # one row of 65537 tiles: more tiles than the scratch holds
    a = torch.zeros((1, w), dtype=torch.uint8, device=dev)
    b = torch.zeros_like(a)
    with pytest.raises(IWPPError) as e:
        recon_u8_noalloc(a, b, conn=8, out=torch.zeros_like(a))
    assert e.value.code == -1
    m = torch.zeros((64, 128), dtype=torch.uint8, device=dev)
    k = torch.zeros((64, 256), dtype=torch.uint8, device=dev)
    # out overlapping the mask only in part (shifted by one column)
    with pytest.raises(IWPPError) as e:
        recon_u8_noalloc(m, k[:, :128], conn=8, out=k[:, 1:129])
    assert e.value.code == -1
    with pytest.raises(IWPPError) as e:
        recon_u8_noalloc(m, k[:, :128], conn=6, out=torch.zeros_like(m))
    assert e.value.code == -1
