"""bench.py's multi-rank launch on CPU: torchrun with two gloo ranks, as the
N>1 bench is launched (one process per GPU there; replicas, no data-path
collective).  The max-over-ranks timing helper must give every rank the
largest value; the reference arm (the CPU oracle) runs on rank 0 alone and
prints exactly one JSON line, while rank 1 exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=600):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_port()}"] + args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_max_over_ranks_and_barrier():
    r = _torchrun([os.path.join("tests", "multirank_probe.py")])
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.count("max over ranks 20.0") == 2


def test_reference_arm_on_two_ranks():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--side", "512",
                   "--reference-sample", "128", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]
