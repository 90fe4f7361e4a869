"""The batched and ticketed entry points of the C ABI, each checked against
the oracle: iwpp_recon_batched (bit-exact, Section 2.1), iwpp_edt_batched
(the departure-aware criterion of Section 2.2, both polarities), and
iwpp_submit / iwpp_poll / iwpp_wait on a context.  Images are ragged
(uneven, odd sizes) and partly pitched (views into wider buffers, whose
pitch rules out TMA staging and exercises the plain-load path)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity import edt_parity
from paper_1209_3314_gb300 import synth
from paper_1209_3314_gb300.binding import (IWPP_EDT_FEATURE_NONZERO, IWPP_EINVAL, IWPP_OK, Image, IWPPError,
                                           image_of)

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
SHAPES = [(37, 1000), (700, 64), (333, 517), (64, 64), (1, 900), (1025, 257), (129, 1100)]


def on_device(a, pitch_pad):
    """A device copy of `a`; with pitch_pad > 0 a view into a wider buffer."""
    t = torch.from_numpy(np.ascontiguousarray(a))
    if not pitch_pad:
        return t.to(DEV)
    h, w = a.shape
    buf = torch.zeros((h, w + pitch_pad), dtype=t.dtype, device=DEV)
    buf[:, :w] = t.to(DEV)
    return buf[:, :w]


@pytest.mark.parametrize("conn", [4, 8])
def test_recon_batched_through_the_c_abi(cuda_ctx, conn):
    lib = cuda_ctx.lib
    markers, masks, outs, refs = [], [], [], []
    for k, (h, w) in enumerate(SHAPES):
        marker, mask = synth.recon_inputs(h, w, 2.0 + k % 5, 20 + 9 * k, seed=500 + k + conn)
        if k % 3 == 2:  # int32 images, values below zero included
            marker, mask = marker.astype(np.int32) - 100, mask.astype(np.int32) - 100
        pad = (0, 5, 16)[k % 3]
        markers.append(on_device(marker, pad))
        masks.append(on_device(mask, (0, 16, 7)[k % 3]))
        outs.append(on_device(np.zeros_like(mask), (3, 0, 16)[k % 3]))
        refs.append(oracle.fh(marker, mask, conn))
    n = len(SHAPES)
    M = (Image * n)(*[image_of(t) for t in markers])
    K = (Image * n)(*[image_of(t) for t in masks])
    O = (Image * n)(*[image_of(t) for t in outs])
    rc = lib.iwpp_recon_batched(cuda_ctx.h, n, M, K, conn, O, None)
    assert rc == IWPP_OK, lib.iwpp_last_error(cuda_ctx.h).decode()
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("feature_nonzero", [False, True])
def test_edt_batched_through_the_c_abi(cuda_ctx, feature_nonzero):
    lib = cuda_ctx.lib
    bins, sqs, nns, host = [], [], [], []
    for k, (h, w) in enumerate(SHAPES):
        img, _ = synth.disks_binary(h, w, 4, 40, 0.1 + 0.05 * k, seed=600 + k)
        host.append(img)
        bins.append(on_device(img, (0, 9, 16)[k % 3]))
        sqs.append(torch.full((h, w), -5, dtype=torch.int32, device=DEV))
        nns.append(torch.full((h, w), -5, dtype=torch.int32, device=DEV))
    n = len(SHAPES)
    B = (Image * n)(*[image_of(t) for t in bins])
    S = (ctypes.c_void_p * n)(*[t.data_ptr() for t in sqs])
    N = (ctypes.c_void_p * n)(*[t.data_ptr() for t in nns])
    flags = IWPP_EDT_FEATURE_NONZERO if feature_nonzero else 0
    rc = lib.iwpp_edt_batched(cuda_ctx.h, n, B, S, N, flags, None)
    assert rc == IWPP_OK, lib.iwpp_last_error(cuda_ctx.h).decode()
    torch.cuda.synchronize()
    for img, sq, nn in zip(host, sqs, nns):
        edt_parity(img, sq.cpu().numpy(), nn.cpu().numpy(), feature_nonzero)


def test_batched_rejects_bad_arguments(cuda_ctx):
    lib = cuda_ctx.lib
    a = torch.zeros((10, 10), dtype=torch.uint8, device=DEV)
    b = torch.zeros((10, 11), dtype=torch.uint8, device=DEV)
    M = (Image * 2)(image_of(a), image_of(a))
    K = (Image * 2)(image_of(a), image_of(b))  # second pair: shapes differ
    O = (Image * 2)(image_of(torch.empty_like(a)), image_of(torch.empty_like(a)))
    assert lib.iwpp_recon_batched(cuda_ctx.h, 2, M, K, 8, O, None) == IWPP_EINVAL
    assert lib.iwpp_recon_batched(cuda_ctx.h, 0, M, K, 8, O, None) == IWPP_EINVAL


def test_submit_poll_wait(cuda_ctx):
    jobs, refs = [], []
    for k, (h, w) in enumerate(SHAPES[:5]):
        if k % 2 == 0:
            marker, mask = synth.recon_inputs(h, w, 4.0, 40, seed=700 + k)
            m, kk = on_device(marker, 16 * (k % 3 == 0)), on_device(mask, 0)
            jobs.append({"op": "recon", "marker": m, "mask": kk, "out": torch.empty_like(kk), "conn": 8 if k else 4})
            refs.append(("recon", oracle.fh(marker, mask, 8 if k else 4)))
        else:
            img, _ = synth.disks_binary(h, w, 4, 30, 0.3, seed=710 + k)
            b = on_device(img, 0)
            jobs.append({"op": "edt", "binary": b, "feature_nonzero": k == 3,
                         "sqdist": torch.empty((h, w), dtype=torch.int32, device=DEV),
                         "nearest": torch.empty((h, w), dtype=torch.int32, device=DEV)})
            refs.append(("edt", img, k == 3))
    tickets = [cuda_ctx.submit(j) for j in jobs]
    assert len(set(tickets)) == len(tickets) and min(tickets) > 0
    # poll the first until done, wait for the rest
    st = None
    for _ in range(200000):
        st = cuda_ctx.poll(tickets[0])
        if st is not None:
            break
    assert st == IWPP_OK
    for t in tickets[1:]:
        assert cuda_ctx.wait(t) == IWPP_OK
    for job, ref in zip(jobs, refs):
        if ref[0] == "recon":
            np.testing.assert_array_equal(job["out"].cpu().numpy(), ref[1])
        else:
            edt_parity(ref[1], job["sqdist"].cpu().numpy(), job["nearest"].cpu().numpy(), ref[2])
    # retired and unknown tickets are rejected; a bad job gives no ticket
    with pytest.raises(IWPPError):
        cuda_ctx.poll(tickets[0])
    with pytest.raises(IWPPError):
        cuda_ctx.wait(123456789)
    bad = dict(jobs[0])
    bad["conn"] = 5
    with pytest.raises(IWPPError):
        cuda_ctx.submit(bad)
    # many more tickets than the status ring holds, none retired until the end
    img, _ = synth.disks_binary(64, 80, 4, 10, 0.3, seed=720)
    b = on_device(img, 0)
    small = {"op": "edt", "binary": b, "sqdist": torch.empty((64, 80), dtype=torch.int32, device=DEV),
             "nearest": torch.empty((64, 80), dtype=torch.int32, device=DEV)}
    many = [cuda_ctx.submit(small) for _ in range(300)]
    assert all(cuda_ctx.wait(t) == IWPP_OK for t in many)
    edt_parity(img, small["sqdist"].cpu().numpy(), small["nearest"].cpu().numpy())
