"""The multi-rank logic on CPU: the max-over-ranks timing reduction with two
gloo ranks; the library's split of a job over independent parts
(flapw_partition, host only), which every rank must compute identically and
which must give every k-point to exactly one part with a bounded load, or
share all k-points by tiles; the bench's weak-scaling job (N sets of the
workload's k-points, whole k-points per rank); and the reference arm under
torchrun with two ranks (rank 0 alone runs the oracle and prints one line,
both exit 0).  They cover the host paths of N > 1 ranks without any GPU."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = bench.max_over_ranks(1.5 + rank)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 2.5, 1: 2.5}


# plane-wave counts of the synthetic workloads: 1 k-point (config 2), the
# 32 uneven k-points of config 4, and uneven sets that do not balance
PARTITION_CASES = [[3990], list(range(2540, 5869, 104)), [5868, 2540, 2600], [4000] * 5,
                   [6000, 500, 500, 500], list(range(100, 4100, 250))]


def _partition_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_1712_07206_gb300 as fl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for ng in PARTITION_CASES:
        own = fl.partition(ng, world)
        got = [torch.zeros(len(ng), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(got, torch.from_numpy(own.astype(np.int32)))
        res.append([g.tolist() for g in got])
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_partition_gloo_two_ranks():
    import numpy as np
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for case, ng in enumerate(PARTITION_CASES):
        a, b = out[0][case], out[1][case]
        assert a == b and a[0] == a[1]                 # both ranks: one identical split
        own = np.array(a[0])
        if own[0] < 0:                                 # shared by tiles: every k-point
            assert np.all(own == -1)
            continue
        assert set(own.tolist()) <= {0, 1} and len(own) >= 2
        w = np.asarray(ng, float) ** 2
        load = [w[own == r].sum() for r in (0, 1)]
        assert max(load) <= 1.1 * w.sum() / 2         # the balance the split promises
    # one k-point, or loads that cannot be balanced: tiles
    assert out[0][0][0] == [-1]
    assert out[0][2][0] == [-1, -1, -1] or max(
        sum(x * x for x, o in zip([5868, 2540, 2600], out[0][2][0]) if o == r) for r in (0, 1)) <= \
        1.1 * sum(x * x for x in [5868, 2540, 2600]) / 2


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-cols", "2",
           "--config", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["value"] > 0


def _job_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_1712_07206_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for cfg in (2, 4):
        mine, job, ng_job, owner = bench.job_split(inputs.CONFIGS[cfg](), world, rank)
        got = [torch.zeros(len(owner), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(got, torch.from_numpy(owner.astype(np.int32)))
        res[cfg] = {"owners": [g.tolist() for g in got], "ng": ng_job, "n_k": mine.n_k,
                    "k_frac": mine.k_frac.tolist(), "job_k": job.k_frac.tolist(),
                    "same_T": bool(np.array_equal(mine.T, job.T))}
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_bench_weak_scaling_job_gloo_two_ranks():
    # the bench's job for N ranks: N sets of the workload's k-points, every
    # k-point on exactly one rank, the same split on every rank, loads within
    # the partition's bound, and each rank's problem holds exactly its k-points
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_1712_07206_gb300 import inputs
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_job_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for cfg, n_k in ((2, 1), (4, 32)):
        a, b = out[0][cfg], out[1][cfg]
        assert a["owners"][0] == a["owners"][1] == b["owners"][0]
        own = np.array(a["owners"][0])
        assert len(own) == 2 * n_k and set(own.tolist()) == {0, 1}
        assert a["job_k"] == b["job_k"] and a["ng"] == b["ng"]
        w = np.asarray(a["ng"], float) ** 2
        assert max(w[own == 0].sum(), w[own == 1].sum()) <= 1.1 * w.sum() / 2
        for r, d in ((0, a), (1, b)):
            ks = np.flatnonzero(own == r)
            assert d["n_k"] == len(ks) and d["same_T"]
            assert np.allclose(d["k_frac"], np.asarray(a["job_k"])[ks])
        # the first set is the workload's own k-points
        assert np.allclose(np.asarray(a["job_k"])[:n_k], inputs.CONFIGS[cfg]().k_frac)
