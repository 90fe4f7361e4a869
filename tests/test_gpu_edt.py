"""Distance transform on the GPU through the C ABI against the CPU oracle
(Algorithm 3) and the exact EDT, with the parity criterion of
tests/parity.py: certificate of the propagation rule, never below the exact
distance, differences from the oracle only at departure pixels."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from parity import edt_parity
from paper_1209_3314_gb300 import IWPPError, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
IMAX = np.iinfo(np.int32).max


def run(ctx, b, fnz=False, **opts):
    if opts:
        old = ctx.options()
        ctx.set_options(**opts)
    try:
        sq, nn = ctx.edt(torch.from_numpy(np.ascontiguousarray(b)).to(DEV), feature_nonzero=fnz)
        torch.cuda.synchronize()
        return sq.cpu().numpy(), nn.cpu().numpy()
    finally:
        if opts:
            ctx.set_options(**old)


@pytest.mark.parametrize("fnz", [False, True])
def test_tiny_random_vs_bruteforce(cuda_ctx, fnz):
    rng = np.random.default_rng(500 + fnz)
    for _ in range(80):
        h, w = (int(v) for v in rng.integers(1, 150, 2))
        b = (rng.random((h, w)) < rng.random()).astype(np.uint8)
        sq, nn = run(cuda_ctx, b, fnz)
        edt_parity(b, sq, nn, fnz, exact=oracle.edt_bruteforce(b, fnz) if h * w < 2500 else None)


def test_special_cases(cuda_ctx):
    b = np.ones((131, 77), np.uint8)
    b[100, 5] = 0
    sq, nn = run(cuda_ctx, b)
    yy, xx = np.mgrid[0:131, 0:77]
    np.testing.assert_array_equal(sq, (yy - 100) ** 2 + (xx - 5) ** 2)
    assert (nn == 100 * 77 + 5).all()
    b = np.ones((90, 140), np.uint8)
    b[:, 70] = 0
    sq, _ = run(cuda_ctx, b)
    np.testing.assert_array_equal(sq, np.broadcast_to((np.arange(140) - 70) ** 2, (90, 140)))
    b = np.zeros((70, 70), np.uint8)
    b[33, 69] = 1
    sq, nn = run(cuda_ctx, b)
    assert sq[33, 69] == 1 and sq.sum() == 1
    sq, nn = run(cuda_ctx, np.ones((100, 100), np.uint8))
    assert (nn == -1).all() and (sq == IMAX).all()
    sq, nn = run(cuda_ctx, np.zeros((100, 100), np.uint8))
    assert (sq == 0).all() and (nn == np.arange(10000).reshape(100, 100)).all()
    sq, nn = run(cuda_ctx, np.ones((1, 1), np.uint8), fnz=True)
    assert sq[0, 0] == 0 and nn[0, 0] == 0


@pytest.mark.parametrize("edt_sweeps,revisit", [(0, 0), (1, 0), (2, 0), (1, 64), (3, 1 << 20)])
def test_sweep_settings_keep_parity(cuda_ctx, edt_sweeps, revisit):
    # queue-only visits, sweeps on every visit, sweeps on the first visit only:
    # every setting must satisfy the same parity criterion
    wl = synth.config_workload("edt4096", size=700)
    for fnz in (False, True):
        sq, nn = run(cuda_ctx, wl.binary, fnz, edt_sweeps=edt_sweeps, edt_revisit_sweep_min=revisit)
        edt_parity(wl.binary, sq, nn, fnz)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_queue_modes_keep_parity(cuda_ctx, mode):
    wl = synth.config_workload("edt4096", size=600)
    for fnz in (False, True):
        sq, nn = run(cuda_ctx, wl.binary, fnz, queue_mode=mode, edt_sweeps=0)
        edt_parity(wl.binary, sq, nn, fnz)


def test_figure3_fixture(cuda_ctx):
    with open(os.path.join(GOLDEN, "edt_departure_170.json")) as f:
        g = json.load(f)
    b = np.array(g["binary"], np.uint8)
    sq, nn = run(cuda_ctx, b)
    edt_parity(b, sq, nn, exact=oracle.edt_bruteforce(b))
    y, x = g["pixel"]
    assert sq[y, x] in (169, 170)


@pytest.mark.parametrize("fnz", [False, True])
def test_config_4096(cuda_ctx, fnz):
    wl = synth.config_workload("edt4096")
    sq, nn = run(cuda_ctx, wl.binary, fnz)
    rep = edt_parity(wl.binary, sq, nn, fnz)
    print("edt4096", "nonzero" if fnz else "zero", rep)


def test_overflow_spill_rescan_paths(cuda_ctx):
    img, _ = synth.disks_binary(1024, 768, 4, 60, 0.3, seed=9)
    sq_o, _ = oracle.edt(img)
    ex = oracle.edt_exact(img)
    for opts in (dict(queue_factor=1, max_relaunch=60), dict(spill_cap=0), dict(spill_cap=16)):
        sq, nn = run(cuda_ctx, img, **opts)
        edt_parity(img, sq, nn, sq_o=sq_o, exact=ex)


def test_tma_and_plain_staging_agree(cuda_ctx):
    """Width 1000 (TMA boxes, ragged last tile) and width 999 (plain loads)."""
    for w in (1000, 999):
        img, _ = synth.disks_binary(600, w, 4, 40, 0.3, seed=w)
        sq, nn = run(cuda_ctx, img)
        edt_parity(img, sq, nn)


def test_largest_side_and_beyond(cuda_ctx):
    """Sides of 32768 (the largest the packed feature coordinates allow) as
    a row, a column and a 3-row strip against the exact EDT; one pixel more
    and empty images are rejected."""
    for shape in ((1, 32768), (32768, 1), (3, 32768)):
        rng = np.random.default_rng(sum(shape))
        b = (rng.random(shape) < 0.999).astype(np.uint8)
        b.flat[-1] = 0  # a feature in the last pixel at least
        sq, nn = run(cuda_ctx, b)
        edt_parity(b, sq, nn, exact=oracle.edt_exact(b, False))
        assert nn.flat[-1] == b.size - 1 and sq.flat[-1] == 0
    for shape in ((1, 32769), (32769, 1), (0, 4), (4, 0)):
        with pytest.raises(IWPPError) as e:
            cuda_ctx.edt(torch.zeros(shape, dtype=torch.uint8, device=DEV))
        assert e.value.code == -1


def test_invalid_arguments_raise(cuda_ctx):
    b = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    s = torch.zeros((8, 8), dtype=torch.int32, device=DEV)
    with pytest.raises(IWPPError):
        cuda_ctx.edt(b.to(torch.int32))
    with pytest.raises(IWPPError):
        cuda_ctx.edt(b, sqdist=s, nearest=s)


@pytest.mark.slow
@pytest.mark.parametrize("fnz", [False, True])
def test_full_16k(cuda_ctx, fnz):
    wl = synth.config_workload("edt16k")
    sq, nn = run(cuda_ctx, wl.binary, fnz)
    rep = edt_parity(wl.binary, sq, nn, fnz)
    print("edt16k", "nonzero" if fnz else "zero", rep)
