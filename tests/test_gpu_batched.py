"""Batched execution (mixed reconstruction and distance-transform jobs of
uneven sizes in one persistent launch): through iwpp_run_jobs, through a
plan, and through a plan replayed as a CUDA graph; each job's result must
match the oracle (reconstruction bit-exact, distance transform by the
departure-aware criterion), also after the inputs change between graph
replays and after autotuning."""
import numpy as np
import pytest
import torch

import oracle
from parity import edt_parity
from paper_1209_3314_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def make_jobs(seed, n=14):
    """Device jobs of mixed kinds and sizes; every fourth recon image has a
    TMA-aligned pitch (wider buffer), the others a packed odd width."""
    wls = synth.batched_workloads(n=n, seed=seed, smin=40, smax=700)
    jobs, refs = [], []
    for k, wl in enumerate(wls):
        if wl.op == "recon":
            if k % 4 == 0:
                marker, mask = wl.marker.astype(np.int32) - 77, wl.mask.astype(np.int32) - 77
            else:
                marker, mask = wl.marker, wl.mask
            def dev(a, pad=(k % 3 == 0)):
                if not pad:
                    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
                h, w = a.shape
                wp = (w + 15) // 16 * 16 + 16
                t = torch.zeros((h, wp), dtype=torch.from_numpy(a).dtype, device=DEV)
                t[:, :w] = torch.from_numpy(a).to(DEV)
                return t[:, :w]
            job = {"op": "recon", "marker": dev(marker), "mask": dev(mask), "conn": 8 if k % 5 else 4}
            job["out"] = torch.empty_like(job["mask"])
            jobs.append(job)
            refs.append(("recon", marker, mask, job["conn"]))
        else:
            b = torch.from_numpy(wl.binary).to(DEV)
            fnz = k % 3 == 1
            jobs.append({"op": "edt", "binary": b, "feature_nonzero": fnz,
                         "sqdist": torch.empty(b.shape, dtype=torch.int32, device=DEV),
                         "nearest": torch.empty(b.shape, dtype=torch.int32, device=DEV)})
            refs.append(("edt", wl.binary, fnz))
    return jobs, refs


def check(jobs, refs):
    for job, ref in zip(jobs, refs):
        if ref[0] == "recon":
            _, marker, mask, conn = ref
            np.testing.assert_array_equal(job["out"].cpu().numpy(), oracle.fh(marker, mask, conn))
        else:
            _, b, fnz = ref
            edt_parity(b, job["sqdist"].cpu().numpy(), job["nearest"].cpu().numpy(), fnz)


def test_run_jobs_mixed_batch(cuda_ctx):
    jobs, refs = make_jobs(11)
    cuda_ctx.run_jobs(jobs)
    torch.cuda.synchronize()
    check(jobs, refs)


def test_run_jobs_split_by_family(cuda_ctx):
    """batch_split: one persistent launch per operation family (uint8 and
    int32 reconstruction, distance transform) back to back; same results."""
    jobs, refs = make_jobs(16)
    old = cuda_ctx.options()
    cuda_ctx.set_options(batch_split=1)
    try:
        cuda_ctx.run_jobs(jobs)
        torch.cuda.synchronize()
    finally:
        cuda_ctx.set_options(**old)
    check(jobs, refs)


@pytest.mark.parametrize("split", [0, 1])
def test_plan_launch_and_graph_replay(cuda_ctx, split):
    jobs, refs = make_jobs(12)
    old = cuda_ctx.options()
    cuda_ctx.set_options(batch_split=split)
    try:
        plan = cuda_ctx.plan(jobs)
    finally:
        cuda_ctx.set_options(**old)
    try:
        plan.launch()
        cuda_ctx.sync()
        check(jobs, refs)
        # replay the captured graph twice with new contents in the same buffers
        for rep in range(2):
            g = torch.Generator(device=DEV).manual_seed(100 + rep)
            for j in jobs:
                if j["op"] == "recon":
                    drop = torch.randint(0, 90, j["mask"].shape, generator=g, device=DEV)
                    lo = 0 if j["mask"].dtype == torch.uint8 else -10**6
                    j["marker"].copy_(torch.clamp(j["mask"].to(torch.int64) - drop, min=lo).to(j["mask"].dtype))
                else:
                    flip = torch.rand(j["binary"].shape, generator=g, device=DEV) < 0.02
                    j["binary"].copy_(torch.where(flip, 1 - j["binary"], j["binary"]))
            plan.launch(graph=True)
            cuda_ctx.sync()
            refs_now = []
            for j, r in zip(jobs, refs):
                if r[0] == "recon":
                    refs_now.append(("recon", j["marker"].cpu().numpy(), j["mask"].cpu().numpy(), r[3]))
                else:
                    refs_now.append(("edt", j["binary"].cpu().numpy(), r[2]))
            check(jobs, refs_now)
    finally:
        plan.close()


def test_autotune_keeps_results(cuda_ctx):
    jobs, refs = make_jobs(15, n=10)
    plan = cuda_ctx.plan(jobs)
    try:
        best = plan.autotune(reps=2)
        assert 2 <= best["sweeps"] <= 4 and 1 <= best["edt_sweeps"] <= 3
        assert best["queue_factor"] in (8, 16, 32) and best["spill_cap"] in (1024, 8192)
        for j in jobs:
            if j["op"] == "recon":
                j["out"].fill_(0)
            else:
                j["sqdist"].fill_(-7)
        plan.launch(graph=True)
        cuda_ctx.sync()
        check(jobs, refs)
    finally:
        plan.close()
