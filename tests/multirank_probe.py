"""Run under torchrun by tests/test_bench_multirank.py (not a test module):
exercises bench.py's rank helpers on two gloo ranks."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

ws, rank, local = bench.dist_setup()
assert ws == 2 and dist.get_backend() == "gloo", (ws, dist.get_backend())
bench.barrier(ws)
got = bench.allreduce_max(10.0 * (rank + 1), ws)
assert got == 20.0, got
print(f"rank {rank}: max over ranks {got}", flush=True)
dist.destroy_process_group()
