"""The distance transform with IWPP_EDT_EXACT_PROPAGATION: the 8-neighbour
propagation (Algorithms 3 and 6) followed by a second wavefront whose window
widens with the distance (Section 2.2: a sufficiently large neighbourhood
makes the propagation exact).  Its squared distances must equal the exact
transform (brute force on small images, the oracle's Meijster transform up
to the 16384^2 workload) at every pixel -- zero departures -- in both
polarities, and nearest must be a feature at exactly that distance.  The
Figure 3 configuration, where the 8-neighbour rule gives 170 instead of
169, comes out exact."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1209_3314_gb300 import IWPPError, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
IMAX = np.iinfo(np.int32).max
HERE = os.path.dirname(os.path.abspath(__file__))


def run(ctx, b, fnz=False, **opts):
    old = ctx.options() if opts else None
    if opts:
        ctx.set_options(**opts)
    try:
        sq, nn = ctx.edt(torch.from_numpy(np.ascontiguousarray(b)).to(DEV), feature_nonzero=fnz,
                         exact_propagation=True)
        torch.cuda.synchronize()
        return sq.cpu().numpy(), nn.cpu().numpy()
    finally:
        if opts:
            ctx.set_options(**old)


def check_nearest(b, sq, nn, fnz):
    h, w = b.shape
    assert ((nn == -1) == (sq == IMAX)).all()
    yy, xx = np.nonzero(sq != IMAX)
    idx = nn[yy, xx].astype(np.int64)
    fy, fx = idx // w, idx % w
    feat = (b != 0) if fnz else (b == 0)
    assert feat[fy, fx].all()
    assert np.array_equal((yy - fy) ** 2 + (xx - fx) ** 2, sq[yy, xx].astype(np.int64))


def test_figure3_configuration_is_exact(cuda_ctx):
    g = json.load(open(os.path.join(HERE, "golden", "edt_departure_170.json")))
    b = np.array(g["binary"], dtype=np.uint8)
    sq_prop, _ = cuda_ctx.edt(torch.from_numpy(b).to(DEV))
    ex = oracle.edt_exact(b)
    assert (sq_prop.cpu().numpy() != ex).any()  # the 8-neighbour rule departs here
    sq, nn = run(cuda_ctx, b)
    np.testing.assert_array_equal(sq, ex)
    check_nearest(b, sq, nn, False)


@pytest.mark.parametrize("fnz", [False, True])
def test_small_random_vs_bruteforce(cuda_ctx, fnz):
    rng = np.random.default_rng(900 + fnz)
    for _ in range(40):
        h, w = (int(v) for v in rng.integers(1, 150, 2))
        b = (rng.random((h, w)) < rng.uniform(0.002, 0.5)).astype(np.uint8)
        sq, nn = run(cuda_ctx, b, fnz)
        np.testing.assert_array_equal(sq, oracle.edt_bruteforce(b, fnz))
        check_nearest(b, sq, nn, fnz)


@pytest.mark.parametrize("fnz", [False, True])
def test_disk_images_ragged(cuda_ctx, fnz):
    for k, (h, w, rmax, cov) in enumerate(((1000, 1300, 40, 0.3), (777, 2049, 80, 0.25), (1500, 999, 60, 0.1))):
        b, _ = synth.disks_binary(h, w, 4, rmax, cov, seed=910 + k)
        ex = oracle.edt_exact(b, fnz)
        sq_prop, _ = cuda_ctx.edt(torch.from_numpy(b).to(DEV), feature_nonzero=fnz)
        sq, nn = run(cuda_ctx, b, fnz)
        assert int((sq != ex).sum()) == 0, ("departures", int((sq != ex).sum()),
                                            "8-neighbour departures", int((sq_prop.cpu().numpy() != ex).sum()))
        check_nearest(b, sq, nn, fnz)


def test_degenerate_cases(cuda_ctx):
    sq, nn = run(cuda_ctx, np.ones((70, 300), np.uint8))  # no feature
    assert (sq == IMAX).all() and (nn == -1).all()
    sq, nn = run(cuda_ctx, np.zeros((40, 50), np.uint8))  # every pixel a feature
    assert (sq == 0).all()
    b = np.ones((513, 700), np.uint8)
    b[17, 600] = 0  # one feature far from most pixels
    sq, nn = run(cuda_ctx, b)
    np.testing.assert_array_equal(sq, oracle.edt_exact(b))
    b = np.ones((1, 999), np.uint8)
    b[0, 3] = 0
    sq, _ = run(cuda_ctx, b)
    np.testing.assert_array_equal(sq, oracle.edt_exact(b))


def test_batched_and_mixed_jobs_take_the_flag(cuda_ctx):
    jobs, refs = [], []
    for k in range(4):
        b, _ = synth.disks_binary(300 + 97 * k, 400 + 31 * k, 4, 40, 0.3, seed=930 + k)
        t = torch.from_numpy(b).to(DEV)
        jobs.append({"op": "edt", "binary": t, "feature_nonzero": k % 2 == 1, "exact_propagation": True,
                     "sqdist": torch.empty(b.shape, dtype=torch.int32, device=DEV),
                     "nearest": torch.empty(b.shape, dtype=torch.int32, device=DEV)})
        refs.append(oracle.edt_exact(b, k % 2 == 1))
    cuda_ctx.run_jobs(jobs)
    torch.cuda.synchronize()
    for j, ex in zip(jobs, refs):
        np.testing.assert_array_equal(j["sqdist"].cpu().numpy(), ex)


def test_unknown_flags_rejected(cuda_ctx):
    a = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    from paper_1209_3314_gb300.binding import image_of
    import ctypes
    im = image_of(a)
    sq = torch.empty((8, 8), dtype=torch.int32, device=DEV)
    nn = torch.empty_like(sq)
    rc = cuda_ctx.lib.iwpp_edt(cuda_ctx.h, ctypes.byref(im), ctypes.c_void_p(sq.data_ptr()),
                               ctypes.c_void_p(nn.data_ptr()), 4, None)
    assert rc == -1


@pytest.mark.slow
@pytest.mark.parametrize("fnz", [False, True])
def test_full_16k_zero_departures(cuda_ctx, fnz):
    """The 16384^2 distance-transform workload (disks r 4..80, 25 %
    foreground), both polarities: zero departures from the exact transform."""
    wl = synth.config_workload("edt16k")
    b = wl.binary
    sq, nn = run(cuda_ctx, b, fnz)
    ex = oracle.edt_exact(b, fnz)
    dep = int((sq != ex).sum())
    assert dep == 0, dep
    # nearest on a sample (the full check is memory heavy at this size)
    h, w = b.shape
    rng = np.random.default_rng(11)
    yy, xx = rng.integers(0, h, 1 << 20), rng.integers(0, w, 1 << 20)
    idx = nn[yy, xx].astype(np.int64)
    fy, fx = idx // w, idx % w
    feat = (b != 0) if fnz else (b == 0)
    assert feat[fy, fx].all()
    assert np.array_equal((yy - fy) ** 2 + (xx - fx) ** 2, sq[yy, xx].astype(np.int64))
