"""Parity at the batched and served workloads' own sizes.

* The batched workload exactly as the benchmark times it: the 512-image pool
  (sides log-uniform in 256..2048, half reconstruction, half distance
  transform, about 385 Mpx and 100 k tiles in one launch per operation
  family), run as an autotuned plan replayed as a CUDA graph.  Every image is
  compared with the oracle: reconstruction bit-exact (Section 2.1), the
  distance transform by the departure-aware criterion (Section 2.2).
* The served workload's large end: requests of sides 4096 and 8192 mixed with
  small ones through the continuous-batching server, each compared with the
  oracle and with the result of the same request served alone.

The oracle checks run in a thread pool (the C oracle and numpy release the
GIL), so the tests take a minute or two.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from parity import edt_parity
from paper_1209_3314_gb300 import synth
from paper_1209_3314_gb300.binding import Server

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = torch.device("cuda:0")


def pool_map(fn, items):
    z = np.zeros((2, 2), dtype=np.uint8)
    oracle.fh(z, z, 8)  # builds and loads the C oracle once, before the threads
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(fn, items))


def test_batched_512_images_as_benchmarked(cuda_ctx):
    wls = synth.batched_from_pool(512, seed=3000)
    jobs = []
    for wl in wls:
        if wl.op == "recon":
            wp = (wl.w + 15) // 16 * 16  # TMA-aligned pitch, as in the benchmark
            buf = torch.zeros((3, wl.h, wp), dtype=torch.uint8, device=DEV)
            buf[0, :, :wl.w] = torch.from_numpy(wl.marker).to(DEV)
            buf[1, :, :wl.w] = torch.from_numpy(wl.mask).to(DEV)
            jobs.append({"op": "recon", "marker": buf[0, :, :wl.w], "mask": buf[1, :, :wl.w],
                         "out": buf[2, :, :wl.w], "conn": 8})
        else:
            b = torch.from_numpy(wl.binary).to(DEV)
            jobs.append({"op": "edt", "binary": b,
                         "sqdist": torch.empty(b.shape, dtype=torch.int32, device=DEV),
                         "nearest": torch.empty(b.shape, dtype=torch.int32, device=DEV)})
    assert sum(w.pixels for w in wls) > 300e6
    plan = cuda_ctx.plan(jobs)
    try:
        plan.autotune(reps=1)
        for j in jobs:  # results must come from the replay below
            if j["op"] == "recon":
                j["out"].fill_(0)
            else:
                j["sqdist"].fill_(-1)
                j["nearest"].fill_(-1)
        plan.launch(graph=True)
        plan.launch(graph=True)
        cuda_ctx.sync()
    finally:
        plan.close()
    got = [(j["out"].cpu().numpy(),) if j["op"] == "recon" else
           (j["sqdist"].cpu().numpy(), j["nearest"].cpu().numpy()) for j in jobs]

    def check(k):
        wl = wls[k]
        if wl.op == "recon":
            return bool(np.array_equal(got[k][0], oracle.fh(wl.marker, wl.mask, 8)))
        edt_parity(wl.binary, got[k][0], got[k][1])
        return True

    ok = pool_map(check, range(len(wls)))
    assert all(ok), [k for k, v in enumerate(ok) if not v][:10]


def test_served_large_requests_alone_and_in_a_mix():
    marker8k, mask8k, bin8k = synth.served_pool(8192, seed=4000)
    rng = np.random.default_rng(4200)

    def window(side):
        y, x = (int(v) for v in rng.integers(0, 8192 - side + 1, 2))
        return slice(y, y + side), slice(x, x + side)

    reqs = []
    for k, side in enumerate((8192, 4096, 600, 8192, 4096, 1000, 777, 512)):
        ys, xs = window(side)
        if k % 2 == 0:
            reqs.append({"op": "recon", "marker": np.ascontiguousarray(marker8k[ys, xs]),
                         "mask": np.ascontiguousarray(mask8k[ys, xs])})
        else:
            reqs.append({"op": "edt", "binary": np.ascontiguousarray(bin8k[ys, xs])})

    def host_bufs(r):
        if r["op"] == "recon":
            return {"marker": torch.from_numpy(r["marker"]).pin_memory(),
                    "mask": torch.from_numpy(r["mask"]).pin_memory(),
                    "out": torch.empty(r["mask"].shape, dtype=torch.uint8).pin_memory()}
        return {"binary": torch.from_numpy(r["binary"]).pin_memory(),
                "sqdist": torch.empty(r["binary"].shape, dtype=torch.int32).pin_memory(),
                "nearest": torch.empty(r["binary"].shape, dtype=torch.int32).pin_memory()}

    def submit(srv, r, hb):
        if r["op"] == "recon":
            return srv.submit_recon(hb["marker"], hb["mask"], hb["out"], 8)
        return srv.submit_edt(hb["binary"], hb["sqdist"], hb["nearest"])

    # alone: one request at a time
    alone = []
    srv = Server(0, hbm_budget=120 << 30, streams=3, max_batch=32)
    try:
        for r in reqs:
            hb = host_bufs(r)
            st, _ = srv.wait(submit(srv, r, hb))
            assert st == 0
            alone.append(hb)
        # in a mix: all submitted back to back, so they batch and overlap
        mixed = [host_bufs(r) for r in reqs]
        tickets = [submit(srv, r, hb) for r, hb in zip(reqs, mixed)]
        assert all(srv.wait(t)[0] == 0 for t in tickets)
    finally:
        srv.close()

    def check(k):
        r, a, m = reqs[k], alone[k], mixed[k]
        if r["op"] == "recon":
            ref = oracle.fh(r["marker"], r["mask"], 8)
            return bool(np.array_equal(a["out"].numpy(), ref) and np.array_equal(m["out"].numpy(), ref))
        b = r["binary"]
        ex = oracle.edt_exact(b)
        sq_o, _ = oracle.edt(b)
        edt_parity(b, a["sqdist"].numpy(), a["nearest"].numpy(), sq_o=sq_o, exact=ex)
        edt_parity(b, m["sqdist"].numpy(), m["nearest"].numpy(), sq_o=sq_o, exact=ex)
        diff = a["sqdist"].numpy() != m["sqdist"].numpy()
        # alone and in the mix differ only at departure pixels
        return not bool((diff & (a["sqdist"].numpy() == ex) & (m["sqdist"].numpy() == ex)).any())

    ok = pool_map(check, range(len(reqs)))
    assert all(ok), ok
