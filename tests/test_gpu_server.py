"""The continuous-batching server (served mode): every result matches the
oracle, each request gives the same result alone and inside a mix (bit-exact
for reconstruction, departure-aware for the distance transform), and the
HBM budget bounds the memory in flight."""
import numpy as np
import pytest
import torch

import oracle
from parity import edt_parity
from paper_1209_3314_gb300 import synth
from paper_1209_3314_gb300.binding import Server

pytestmark = pytest.mark.gpu


def host(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def make_requests(seed, n):
    wls = synth.batched_workloads(n=n, seed=seed, smin=48, smax=600)
    reqs = []
    for k, wl in enumerate(wls):
        if wl.op == "recon":
            reqs.append({"op": "recon", "marker": host(wl.marker), "mask": host(wl.mask),
                         "out": torch.empty((wl.h, wl.w), dtype=torch.uint8).pin_memory(),
                         "conn": 8 if k % 3 else 4})
        else:
            reqs.append({"op": "edt", "binary": host(wl.binary), "fnz": k % 4 == 1,
                         "sqdist": torch.empty((wl.h, wl.w), dtype=torch.int32).pin_memory(),
                         "nearest": torch.empty((wl.h, wl.w), dtype=torch.int32).pin_memory()})
    return reqs


def submit(srv, r):
    if r["op"] == "recon":
        return srv.submit_recon(r["marker"], r["mask"], r["out"], r["conn"])
    return srv.submit_edt(r["binary"], r["sqdist"], r["nearest"], r["fnz"])


def snapshot(r):
    return r["out"].clone() if r["op"] == "recon" else (r["sqdist"].clone(), r["nearest"].clone())


def check(r):
    if r["op"] == "recon":
        np.testing.assert_array_equal(r["out"].numpy(), oracle.fh(r["marker"].numpy(), r["mask"].numpy(), r["conn"]))
    else:
        edt_parity(r["binary"].numpy(), r["sqdist"].numpy(), r["nearest"].numpy(), r["fnz"])


def test_server_results_match_oracle():
    reqs = make_requests(21, 24)
    srv = Server(0, hbm_budget=1 << 30, streams=3, max_batch=8)
    try:
        tickets = [submit(srv, r) for r in reqs]
        lats = []
        for t in tickets:
            st, lat = srv.wait(t)
            assert st == 0
            lats.append(lat)
        assert min(lats) > 0
        for r in reqs:
            check(r)
        s = srv.stats()
        assert s["completed"] == len(reqs) and s["batches"] >= 3
    finally:
        srv.close()


def test_alone_equals_in_mix():
    probes = make_requests(22, 4)
    others = make_requests(23, 20)
    srv = Server(0, hbm_budget=1 << 30, streams=3, max_batch=6)
    try:
        alone = []
        for r in probes:
            st, _ = srv.wait(submit(srv, r))
            assert st == 0
            alone.append(snapshot(r))
        tickets = []
        for k, r in enumerate(others):
            tickets.append(submit(srv, r))
            if k % 5 == 2:
                tickets.append(submit(srv, probes[k // 5]))
        for t in tickets:
            assert srv.wait(t)[0] == 0
        for r, a in zip(probes, alone):
            if r["op"] == "recon":
                assert torch.equal(r["out"], a)
            else:
                b = r["binary"].numpy()
                ex = oracle.edt_exact(b, r["fnz"])
                sq_mix, sq_alone = r["sqdist"].numpy(), a[0].numpy()
                edt_parity(b, sq_mix, r["nearest"].numpy(), r["fnz"], exact=ex)
                edt_parity(b, sq_alone, a[1].numpy(), r["fnz"], exact=ex)
                diff = sq_mix != sq_alone
                assert not (diff & (sq_mix == ex) & (sq_alone == ex)).any()
        for r in others:
            check(r)
    finally:
        srv.close()


def req_bytes(r):
    """The device bytes the server counts for a request: three buffers, each
    rounded up to 2 MiB."""
    mb2 = 2 << 20
    rnd = lambda n: -(-n // mb2) * mb2  # noqa: E731
    if r["op"] == "recon":
        return 3 * rnd(r["marker"].numel())
    return rnd(r["binary"].numel()) + 2 * rnd(4 * r["binary"].numel())


def test_budget_admission_counts_the_workspace_and_real_memory():
    """The budget bounds the device memory the server really holds: the
    memory pool's high-water mark of request images plus the resident
    workspace of the streams' contexts.  The budget leaves room for the
    workspace and 1.5 requests; were the workspace left out of admission,
    all ten requests would be admitted at once and the pool's high-water
    mark alone would break the bound."""
    reqs = make_requests(24, 10)
    # the workspace the contexts grow to on this mix (run twice, so that it
    # has settled); one request at a time needs no more than that
    probe = Server(0, hbm_budget=8 << 30, streams=3, max_batch=8)
    try:
        for _ in range(2):
            for t in [submit(probe, r) for r in reqs]:
                assert probe.wait(t)[0] == 0
        ws = probe.stats()["workspace_bytes"]
    finally:
        probe.close()
    biggest = max(req_bytes(r) for r in reqs)
    assert sum(req_bytes(r) for r in reqs) > 2 * biggest
    budget = ws + int(biggest * 1.5)
    srv = Server(0, hbm_budget=budget, streams=3, max_batch=8)
    try:
        tickets = [submit(srv, r) for r in reqs]
        for t in tickets:
            assert srv.wait(t)[0] == 0
        st = srv.stats()
        assert st["workspace_bytes"] <= ws
        assert st["peak_bytes_in_use"] <= budget
        assert st["pool_used_high"] + st["workspace_bytes"] <= budget
        assert st["records"] == 0  # every result was handed out and dropped
        for r in reqs:
            check(r)
        # a handed-out ticket is retired
        with pytest.raises(Exception):
            srv.wait(tickets[0])
        big = torch.zeros((2048, 2048), dtype=torch.uint8).pin_memory()  # 12 MiB > 1.5 requests
        out = torch.empty_like(big)
        st, _ = srv.wait(srv.submit_recon(big, big, out))
        assert st == -2  # cannot fit next to the workspace, even alone
    finally:
        srv.close()
