"""bench.py with two ranks under torchrun on one GPU: the N > 1 path end to
end (the weak-scaling job of two sets of the workload's k-points, whole
k-points per rank from flapw_partition, the timing reduction over a gloo
process group).  The two ranks' kernels never wait on each other, so they
may share the GPU; the rate they print says nothing about scaling."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_bench_two_ranks_share_one_gpu():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--gpus", "2", "--dist-backend", "gloo", "--config", "1", "--steps", "3", "--warmup", "3",
           "--fp64-steps", "0", "--no-cpu-baseline", "--e2e-steps", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak"
    assert d["config"]["job_kpoints"] == 2 and d["config"]["n_k"] == 1
    assert d["value"] > 0 and d["e2e"]["value"] > 0
    assert d["config"]["flops_per_step"] > 0
