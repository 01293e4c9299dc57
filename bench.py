"""Benchmark of the muffin-tin H/S build on GB300.

One step = one pass of the whole hot path over the workload's k-points:
plane waves (set up once per handle), A/B generation (flapw_build_AB), T
factorisation, operand formation, slicing and the lower-triangle contraction
(flapw_build_HS).  Metric: H+S build TFLOP/s at the Hermitian rank-K count
16 N_A N_L N_G^2 per k-point (H and S), and ms per k-point; the emulated
(FP16-slice) path is the headline, the plain FP64 path is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config 2] [--operands factored|from_ab]

Under torchrun with N > 1 the job is N sets of the workload's k-points (the
workload's own and seeded k-points of the same crystal); flapw_partition gives
every rank whole k-points, each rank builds H and S of its own on its GPU (no
exchange between ranks), and rank 0 prints one JSON line with the whole job's
rate over the slowest rank's time (weak scaling: the work per GPU stays that
of the workload).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# options.h_method values of include/flapw.h
H_METHODS = {"factored": 0, "alg3": 1, "spherical": 2, "alg1": 3}

METRIC = "H+S build TFLOP/s & ms/k-point, emulated vs FP64 path, at ≤1e-12 rel err"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """Largest value over the ranks of the default process group (x itself
    when there is none); NCCL reduces on the GPU, gloo on the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    if dist.get_backend() == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    else:
        dev = torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# DRAM bytes (read + write) per herk_emu_kernel launch, mean of the S and the
# H launch of one step, from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum; profiles/herk_emu_*), keyed by workload, slices, S
# method, H method, tile cover, tile order and load pipeline, with the hash of
# the kernel sources it was taken on (kernel_source_hash).  A capture of other
# sources, or of another shape or configuration, reports null.
MEASURED_TRAFFIC = {
    ("c2_ortho_16at_l8_ng4000", 7, "contraction", "factored", 1, 0, 1):
        {"bytes": 2.1783e9, "kernel_sha": "f7ebd60ead70bd98"},
    ("c2_ortho_16at_l8_ng4000", 7, "contraction", "factored", 1, 5, 1):
        {"bytes": 2.1770e9, "kernel_sha": "f7ebd60ead70bd98"},
}

KERNEL_SOURCES = ("herk_emu.cu", "tc_common.cuh", "tiles.cuh", "fixed64.cuh")


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the emulated contraction's sources
    (the kernel, its device helpers and the tile cover that orders its work)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1712_07206_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, slices, s_method, h_method, cover, order, pipeline):
    rec = MEASURED_TRAFFIC.get((workload, slices, s_method, h_method, cover, order, pipeline))
    if rec and rec["kernel_sha"] == kernel_source_hash():
        return rec["bytes"]
    return None


def fp64_peak_tflops():
    """Measured FP64 peak of this GPU: best of 5 cuBLAS DGEMMs (torch.matmul,
    float64, 4096^3, 2 N^3 flops each), CUDA events on the current stream."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = torch.empty_like(a)
    torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def columns_from_lower(x, ng, layout, cols):
    """Full columns cols[c] of a Hermitian matrix given as the library's lower
    triangle (full layout, ld = ng, or LAPACK packed), as [len(cols)][ng]."""
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    packed = layout == 1
    out = np.zeros((len(cols), ng), complex)
    i = np.arange(ng)
    for c, g in enumerate(cols):
        lo = i >= g
        hi = i[~lo]
        if packed:
            out[c, lo] = x[g * ng - g * (g - 1) // 2 + (i[lo] - g)]
            out[c, ~lo] = np.conj(x[hi * ng - hi * (hi - 1) // 2 + (g - hi)])
        else:
            out[c, lo] = x[g * ng + i[lo]]
            out[c, ~lo] = np.conj(x[hi * ng + g])
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), \
            float(d["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 1700.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.out, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.out):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                pass
        os.unlink(self.out)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


def workload(cfg):
    from paper_1712_07206_gb300 import inputs
    return inputs.CONFIGS[cfg]()


def job_split(p, ws, rank):
    """Weak scaling over ws ranks: the job is ws sets of the workload's
    k-points (inputs.with_kpoints), split by whole k-points with
    flapw_partition; returns (this rank's problem, the job, the job's N_G per
    k-point, the owner of each).  Every rank computes the same split."""
    import paper_1712_07206_gb300 as fl
    from paper_1712_07206_gb300 import inputs
    job = inputs.with_kpoints(p, ws)
    ng_job = [len(fl.enumerate_g(job.lattice, job.k_frac[k], job.kmax[k])) for k in range(job.n_k)]
    owner = fl.partition(ng_job, ws)
    if (owner < 0).any():
        raise RuntimeError("the job's k-points must go to the ranks whole")
    return inputs.subset_kpoints(job, [k for k in range(job.n_k) if owner[k] == rank]), job, ng_job, owner


def hs_flops(p, ngs, per=16.0):
    """per N_A N_L N_G^2 per k-point: 16 in the rank-K (HERK) count of the metric,
    20 in the count of the paper's Alg. 3 operation sequence."""
    return per * p.n_atoms * p.n_L * float(np.sum(np.asarray(ngs, dtype=np.float64) ** 2))


def run_ours(args):
    import torch
    import paper_1712_07206_gb300 as fl

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        # one GPU per rank (more ranks than GPUs share them round-robin, which
        # only the host-side gloo backend allows: no rank's kernels wait on
        # another's)
        dev_i = local % torch.cuda.device_count()
        torch.cuda.set_device(dev_i)
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", dev_i))
        else:
            dist.init_process_group("gloo")
    else:
        torch.cuda.set_device(0)
    fl.build()
    p = workload(args.config)
    job_flops = None
    n_job = p.n_k
    if ws > 1:
        p, job, ng_job, _ = job_split(p, ws, rank)
        job_flops = hs_flops(job, ng_job)
        n_job = job.n_k
    t_sph = None
    if args.h_method == "spherical":
        # the workload with T replaced by its spherical part (per slot and l the
        # means over m of the l-diagonal entries): H then comes from the
        # addition theorem alone, with no H contraction
        p.T, t_sph = spherical_part(p.T, p.lmax)
    operands = fl.OPERANDS_FACTORED if args.operands == "factored" else fl.OPERANDS_FROM_AB
    layout = fl.LAYOUT_LOWER_PACKED if p.layout == "packed" else fl.LAYOUT_LOWER_FULL
    opt = fl.default_options(precision=fl.PREC_EMU, layout=layout, operands=operands, n_slices=args.slices,
                             tile_order=args.tile_order, pipeline=args.pipeline, tile_cover=args.cover,
                             autotune=1 if args.autotune else 0, use_graph=1 if args.graph else 0,
                             s_method=fl.S_LEGENDRE if args.s_method == "legendre" else fl.S_CONTRACTION,
                             h_method=H_METHODS[args.h_method])
    h = fl.from_problem(p, opt)
    if t_sph is not None:
        h.set_spherical_T(t_sph)
    ngs = [h.num_g(k) for k in range(p.n_k)]
    flops = hs_flops(p, ngs)          # this rank's k-points
    if job_flops is None:
        job_flops = flops
    dev = torch.device("cuda")
    nab = h.ab_offset(p.n_k)
    A = torch.empty(nab, dtype=torch.complex128, device=dev)
    B = torch.empty_like(A)

    def outsz(ng):
        return ng * (ng + 1) // 2 if layout == fl.LAYOUT_LOWER_PACKED else ng * ng

    H = [torch.zeros(outsz(ng), dtype=torch.complex128, device=dev) for ng in ngs]
    S = [torch.zeros(outsz(ng), dtype=torch.complex128, device=dev) for ng in ngs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        h.build_AB(p.radial, A, B, stream)
        h.build_HS(p.T, p.atom_slot, p.U, A, B, H, S, stream)

    def timed(n_steps, collect_kernel=False):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        kms, abms = [], []
        for i in range(n_steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            if collect_kernel:
                h.sync()
                st_ = h.stats()
                # the tensor-core contraction alone (with Legendre S only the H half,
                # with H by the addition theorem only the S half)
                if args.h_method == "spherical":
                    kms.append(st_["ms_s"])
                else:
                    kms.append(st_["ms_contract"] - (st_["ms_s"] if args.s_method == "legendre" else 0.0))
                abms.append(st_["ms_ab_assemble"])
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], (kms, abms)

    for _ in range(args.warmup):
        step()
    h.sync()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall = time.time()
    step_ms, _ = timed(args.steps)
    t_wall = time.time() - t_wall
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean(step_ms)))
    # contraction kernel duration, from the library's own events on the launching stream
    _, (kms, abms) = timed(3, collect_kernel=True)
    st = h.stats()
    k_ms = float(np.mean(kms))
    bf16_burst, bf16_sus, hbm, src = peaks()
    # a contraction of a second or more runs under the power cap: sustained peak
    peak, peak_kind = (bf16_sus, "sustained") if k_ms >= 1000.0 else (bf16_burst, "burst")
    achieved = st["flops_tensor"] / (k_ms * 1e-3) / 1e12
    n_pairs = args.slices * (args.slices + 1) // 2
    # slice-pair products of the timed launches: H (K = k_total) and, unless S
    # comes from the addition theorem, S (K = 2 N_A N_L)
    k_s = 0 if args.s_method == "legendre" else 2 * p.n_atoms * p.n_L
    k_h = 0 if args.h_method == "spherical" else st["k_total"]
    alg_tensor = n_pairs * 4.0 * (k_h + k_s) * float(np.sum(np.asarray(ngs, float) ** 2))
    achieved_alg = alg_tensor / (k_ms * 1e-3) / 1e12
    stage = {k: round(st[k], 4) for k in ("ms_ab", "ms_factor", "ms_operands", "ms_slice", "ms_contract",
                                          "ms_hs_total")}
    # the measured FP64 peak (DGEMM), the bound of the FP64 path and of the A/B assembly
    fp64_peak = fp64_peak_tflops()
    ab_instr = 8.0 * p.n_atoms * p.n_L * sum(ngs)
    # the plain FP64 path on the same workload (fewer steps: ~0.3 s each)
    f64_ms = None
    H64 = S64 = None
    if args.fp64_steps > 0:
        # the FP64 leg writes its own outputs, so both paths can be checked
        H64 = [None if x is None else torch.zeros_like(x) for x in H]
        S64 = [None if x is None else torch.zeros_like(x) for x in S]
        h.set_options(fl.default_options(precision=fl.PREC_FP64, layout=layout, operands=operands,
                                         use_graph=1 if args.graph else 0, s_method=opt.s_method,
                                         h_method=opt.h_method))
        f_ms, f_kms = [], []
        for i in range(args.fp64_steps + 1):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.build_AB(p.radial, A, B, stream)
            h.build_HS(p.T, p.atom_slot, p.U, A, B, H64, S64, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                f_ms.append(e0.elapsed_time(e1))
                h.sync()
                f_kms.append(h.stats()["ms_contract"])
        f64_ms = float(np.mean(f_ms))
        f64_kms = float(np.mean(f_kms))
        h.set_options(opt)
    # end-to-end through the C ABI: the step's inputs (radial data, T, U, slots)
    # from host memory and its results H and S into pinned host buffers, copies
    # inside the timed region; A and B, an intermediate of the step, stay in
    # device memory
    e2e = None
    if args.e2e:
        Hh = [torch.empty(outsz(ng), dtype=torch.complex128).pin_memory() for ng in ngs]
        Sh = [torch.empty(outsz(ng), dtype=torch.complex128).pin_memory() for ng in ngs]

        def step_host():
            h.build_AB(p.radial, A, B, stream)
            h.build_HS(p.T, p.atom_slot, p.U, A, B, Hh, Sh, stream)
            h.sync()

        step_host()
        torch.cuda.synchronize()
        e_steps, e_enq, e_lib = [], [], []
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            h.build_AB(p.radial, A, B, stream)
            h.build_HS(p.T, p.atom_slot, p.U, A, B, Hh, Sh, stream)
            t2 = time.perf_counter()
            h.sync()
            t3 = time.perf_counter()
            e_steps.append((t3 - t1) * 1e3)
            e_enq.append((t2 - t1) * 1e3)
            e_lib.append(h.stats()["ms_hs_total"])
        e_ms = max_over_ranks(float(np.mean(e_steps)))
        h2d = p.T.nbytes + p.U.nbytes + p.radial.nbytes + p.atom_slot.nbytes
        # the library's own count of the bytes its copies to host memory move
        # (the lower triangles, plus the small triangles above the diagonal
        # inside the column blocks of the full layout)
        st_e = h.stats()
        d2h = st_e["bytes_d2h"]
        e2e = {"value": round(job_flops / (e_ms * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
               "ms_per_step": round(e_ms, 4), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "d2h_copies_per_step": int(st_e["copy_ops"]),
               "steps_ms": [round(x, 3) for x in e_steps],
               # per step: host time until build_HS returned, and the library's
               # own device time of build_HS (its events, copies included)
               "enqueue_ms": [round(x, 3) for x in e_enq], "hs_device_ms": [round(x, 3) for x in e_lib]}
    # the whole job's flops over the slowest rank's time (each rank computes its k-points)
    value = job_flops / (ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "ms_per_kpoint": round(ms / p.n_k, 4),
        "value_alg3_count": round(job_flops * 20.0 / 16.0 / (ms * 1e-3) / 1e12, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 via fp16 slices (int64 accumulation)", "data": "synthetic",
        "config": {"workload": p.name, "n_atoms": p.n_atoms, "n_types": p.n_types, "lmax": p.lmax,
                   "n_L": p.n_L, "n_k": p.n_k, "n_g": ngs if len(ngs) <= 4 else [min(ngs), max(ngs)],
                   "K": int(st["k_total"]), "slices": args.slices, "operands": args.operands,
                   "layout": p.layout, "l2": "256 MB L2 flush between steps; A/B 166 MB and operands exceed L2",
                   "job_kpoints": n_job, "flops_per_step": job_flops, "graph_replay": bool(args.graph),
                   "s_method": args.s_method,
                   "h_method": args.h_method,
                   # the contraction's tile cover (1 cyclic, 2 aligned), tile order and
                   # load pipeline (1: 3 stages of two K chunks, 2: 5 of one) in use,
                   # chosen by the library's autotuner unless forced
                   "autotune": bool(args.autotune), "tile_cover": st["tile_cover"],
                   "tile_order": st["tile_order"], "pipeline": st["pipeline"],
                   "parallelism": ("one GPU" if ws == 1 else
                                   f"{ws} ranks, each the whole k-points flapw_partition gives it "
                                   f"({n_job} in the job: {ws} sets of the workload's), no exchange")},
        "fp64_path": None if f64_ms is None else {
            "value": round(job_flops / (max_over_ranks(f64_ms) * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
            "ms_per_step": round(f64_ms, 3), "steps": args.fp64_steps,
            # the FP64 contraction kernel (DMMA) against the GPU's measured FP64
            # peak: cuBLAS DGEMM on the same device, in the same run
            "roofline": {"bound": "fp64", "kernel": "herk_f64_kernel (S and H launches)",
                         "kernel_ms": round(f64_kms, 3),
                         "achieved": round(flops / (f64_kms * 1e-3) / 1e12, 4),
                         "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                         "frac": round(flops / (f64_kms * 1e-3) / 1e12 / fp64_peak, 4),
                         "peak_source": "measured in this run: best of 5 cuBLAS DGEMM 4096^3 "
                                        "(torch.matmul float64)"}},
        "speedup_emu_vs_fp64": None if f64_ms is None else round(f64_ms / ms, 2),
        "stages_ms": stage,
        # achieved: the slice-product work the method needs (s(s+1)/2 pairs x
        # 4 K N_G^2 per matrix, no tile or K padding) per kernel second;
        # achieved_executed counts the MMAs the kernel issues
        "roofline": {"bound": "tensor", "achieved": round(achieved_alg, 2), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(achieved_alg / peak, 4),
                     "achieved_executed": round(achieved, 2),
                     "frac_executed": round(achieved / peak, 4),
                     "traffic": args.traffic if args.traffic is not None else
                     measured_traffic(p.name, args.slices, args.s_method, args.h_method,
                                      st["tile_cover"], st["tile_order"], st["pipeline"]),
                     "kernel_source_hash": kernel_source_hash(),
                     "kernel": "herk_emu_kernel (" + ("H launch; S by the addition theorem"
                                                      if args.s_method == "legendre" else
                                                      "S launch; H by the addition theorem"
                                                      if args.h_method == "spherical" else "S and H launches")
                               + ("; H as Alg. 3's L^H R" if args.h_method == "alg3" else
                                  "; H as Alg. 1's L^H R" if args.h_method == "alg1" else "") + ")",
                     "kernel_ms": round(k_ms, 4),
                     "peak_source": f"{src} bf16 {peak_kind} x 1.0 (fp16 = bf16 nominal rate)"},
        # the A/B assembly (HBM store-bound): 32 bytes stored per (atom, L, G)
        "roofline_ab": {"bound": "hbm", "kernel": "ab_assemble_kernel",
                        "bytes": int(32 * p.n_atoms * p.n_L * sum(ngs)),
                        "kernel_ms": round(float(np.mean(abms)), 4),
                        "achieved": round(32 * p.n_atoms * p.n_L * sum(ngs) / (float(np.mean(abms)) * 1e-3) / 1e9, 1),
                        "peak": hbm, "unit": "GB/s",
                        "frac": round(32 * p.n_atoms * p.n_L * sum(ngs) / (float(np.mean(abms)) * 1e-3) / 1e9 / hbm, 4),
                        # what bounds it: 8 FP64 instructions per (atom, L, G) (the
                        # complex phase x Y product, 2 DMUL + 2 DFMA, then 4 DMUL by
                        # a_l and b_l) against the FP64 issue rate of the measured DGEMM
                        # (one DFMA per 2 flops)
                        "fp64_issue": {"instr_per_elem": 8,
                                       "achieved_ginstr_s": round(ab_instr / (float(np.mean(abms)) * 1e-3) / 1e9, 1),
                                       "peak_ginstr_s": round(fp64_peak * 1e3 / 2, 1),
                                       "frac": round(ab_instr / (float(np.mean(abms)) * 1e-3) / 1e9
                                                     / (fp64_peak * 1e3 / 2), 4)}},
        "e2e": e2e,
        "gpu_launches": launches_per_step(args) * args.steps,
        "clocks": clk,
        "timed_wall_s": round(t_wall, 3),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, h, H, S, layout, ngs, args, H64, S64)
        line["refined_cpu"] = refined_cpu(p, args)
    if args.eigh and rank == 0 and H[0] is not None:
        line["eigh"] = eigh_leg(h, H[0], S[0], ngs[0], layout, args)
    h.destroy()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def eigh_leg(h, H, S, ng, layout, args):
    """The generalised eigensolve H c = lambda S c (flapw_eigh, cuSOLVER zhegvd
    in FP64) on k-point 0's H and S as built, outside the step: its time,
    the extreme eigenvalues, and the residual and S-orthonormality of the
    lowest and highest 8 eigenvectors against the matrices as built."""
    import torch
    import paper_1712_07206_gb300 as fl
    if layout != fl.LAYOUT_LOWER_FULL:
        return {"unavailable": "the eigensolve takes the full layout"}
    Hf = torch.tril(H.view(ng, ng).T)
    Hf = Hf + torch.tril(Hf, -1).conj().T
    Sf = torch.tril(S.view(ng, ng).T)
    Sf = Sf + torch.tril(Sf, -1).conj().T
    Hw, Sw = H.clone(), S.clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    try:
        w = h.eigh(ng, Hw, ng, Sw, ng)
    except fl.FlapwError as e:
        return {"n": ng, "error": str(e)}
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    C = Hw.view(ng, ng).T                     # column j: eigenvector j
    cols = list(range(8)) + list(range(ng - 8, ng))
    Cs = C[:, cols]
    ws_ = torch.tensor(w[cols], dtype=torch.float64, device=Cs.device)
    R = Hf @ Cs - (Sf @ Cs) * ws_[None, :]
    res = float(torch.linalg.norm(R) / (torch.linalg.norm(Hf) * torch.linalg.norm(Cs)
                                        + torch.linalg.norm(Sf) * torch.linalg.norm(Cs) * float(np.abs(w).max())))
    orth = float((Cs.conj().T @ Sf @ Cs - torch.eye(len(cols), dtype=Cs.dtype, device=Cs.device)).abs().max())
    # nominal complex FP64 operation count of the solve: Cholesky (4/3 n^3),
    # reduction to standard form (4 n^3), tridiagonalisation (16/3 n^3),
    # back-transformations of the eigenvectors (8 n^3 + 4 n^3)
    nominal = 22.7 * float(ng) ** 3
    # the CPU beside it: scipy's generalised Hermitian solver (LAPACK zhegvd) on
    # the leading n_s x n_s blocks of the same H and S on the host cores (a
    # leading block of a positive definite S is positive definite), scaled
    # to n by the n^3 cost
    import scipy.linalg as sl
    n_s = min(ng, 2048)
    Hc = Hf[:n_s, :n_s].cpu().numpy()
    Sc = Sf[:n_s, :n_s].cpu().numpy()
    t0 = time.perf_counter()
    sl.eigh(Hc, Sc)
    t_cpu = time.perf_counter() - t0
    return {"n": ng, "ms": round(ms, 1), "solver": "cuSOLVER zhegvd, FP64 (flapw_eigh)",
            "lambda_min": float(w[0]), "lambda_max": float(w[-1]),
            "residual_16_vectors": res, "s_orthonormality_16_vectors": orth,
            "nominal_tflops": round(nominal / (ms * 1e-3) / 1e12, 3),
            "cpu": {"solver": "scipy.linalg.eigh (LAPACK zhegvd)", "n_sample": n_s,
                    "s": round(t_cpu, 2), "cores": os.cpu_count(),
                    "scaled_to_n_s": round(t_cpu * (ng / n_s) ** 3, 1)}}


def spherical_part(T, lmax):
    """The l-diagonal part of T per slot: t[slot][l] = (t^AA_l, t^BB_l, Re t^BA_l,
    Im t^BA_l), the means over m of the diagonal entries of each block, and the
    matrix it makes (T^XY_{(lm),(lm)} = t^XY_l, zero elsewhere)."""
    ns, n = T.shape[0], T.shape[1]
    nl = n // 2
    t = np.zeros((ns, lmax + 1, 4))
    Ts = np.zeros_like(T)
    for s_ in range(ns):
        for l in range(lmax + 1):
            L = np.arange(l * l, (l + 1) * (l + 1))
            taa = float(np.mean(T[s_, L, L].real))
            tbb = float(np.mean(T[s_, nl + L, nl + L].real))
            tba = complex(np.mean(T[s_, nl + L, L]))
            t[s_, l] = (taa, tbb, tba.real, tba.imag)
            Ts[s_, L, L] = taa
            Ts[s_, nl + L, nl + L] = tbb
            Ts[s_, nl + L, L] = tba
            Ts[s_, L, nl + L] = np.conj(tba)
    return Ts, t


def launches_per_step(args):
    """Kernels one timed step launches: ab_prep and ab_assemble; the S half
    (opform_S, slicer, contraction; or the addition theorem's split and
    double-float kernels); the H contraction and the H operands:
      factored operands: tfactor, layout, W and conj(C^H) formed and sliced
        (4 kernels), their tensor-core product, and one kernel that applies
        the atom phases and slices the rows;
      A/B operands: tfactor, layout, opform_H and the slicer;
      Alg. 3 and Alg. 1: no tfactor and layout but the kernel that forms the
        operand matrix (with Alg. 1 the Cholesky factors of T^AA); factored,
        the same four factor kernels, the product, the phase kernel, the copy
        of A and B and the slicer; from A/B, the FP64 product and copy kernels
        and the slicer."""
    n = 2
    n += 2 if args.s_method == "legendre" else 3
    if args.h_method == "spherical":
        # T is its spherical part: the W factor formed and sliced, and the
        # addition-theorem kernel; no factorisation, H operands or H contraction
        return n + 3
    n += 1
    if args.h_method in ("alg3", "alg1"):
        n += 9 if args.operands == "factored" else 4
    else:
        n += 8 if args.operands == "factored" else 4
    return n


def refined_cpu(p, args):
    """The paper's refined CPU code path (Alg. 3: zherk, zher2k, zherkx on host
    BLAS) for a block of columns of k-point 0, numpy complex128 on all host
    cores, A/B from the oracle: a comparator in the manner of the paper's
    refined CPU baseline, in the metric's flop count."""
    import os
    import oracle

    oracle.build()
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    A, B = oracle.build_ab(p, 0, n3)
    ng, nl = len(n3), p.n_L
    m = min(ng, args.refined_cols)
    ls = np.concatenate([[l] * (2 * l + 1) for l in range(p.lmax + 1)])
    Ast = np.vstack(list(A))
    Bst = np.vstack(list(B))
    t0 = time.perf_counter()
    X = np.vstack([p.U[p.atom_type[a], ls][:, None] * B[a] for a in range(p.n_atoms)])
    S = Ast.conj().T @ Ast[:, :m] + X.conj().T @ X[:, :m]
    Z = np.vstack([p.T[p.atom_slot[a]][nl:, :nl] @ A[a] + 0.5 * p.T[p.atom_slot[a]][nl:, nl:] @ B[a]
                   for a in range(p.n_atoms)])
    H = Z.conj().T @ Bst[:, :m] + Bst.conj().T @ Z[:, :m]
    Y = np.vstack([p.T[p.atom_slot[a]][:nl, :nl] @ A[a] for a in range(p.n_atoms)])
    H += Ast.conj().T @ Y[:, :m]
    dt = time.perf_counter() - t0
    per_col = 16.0 * p.n_atoms * p.n_L * ng
    return {"value": round(m * per_col / dt / 1e12, 6), "unit": "TFLOP/s",
            "cores": len(os.sched_getaffinity(0)), "kind": "numpy BLAS, Alg. 3 sequence",
            "sample": f"{m} of {ng} columns of H and S at k-point 0 (operand products for all rows), {dt:.2f} s"}


def cpu_baseline(p, h, H, S, layout, ngs, args, H64=None, S64=None):
    """The oracle on sampled columns of the same workload, timed on the host
    cores; the same columns check the GPU results of both paths (relative
    Frobenius error over the sampled full columns)."""
    import oracle

    oracle.build()
    n3 = h.gvectors(0)
    ng = ngs[0]
    rng = np.random.default_rng(0)
    n_cols = args.cpu_cols
    if n_cols <= 0:
        # a bounded sample of about --cpu-seconds of oracle work, sized on 32
        # columns after a warm-up call (thread start-up)
        oracle.hs_columns(p, 0, n3, np.arange(min(4, ng)))
        t0 = time.perf_counter()
        oracle.hs_columns(p, 0, n3, np.arange(min(32, ng)))
        per_col = (time.perf_counter() - t0) / min(32, ng)
        n_cols = int(min(ng, max(16, args.cpu_seconds / max(per_col, 1e-9))))
    cols = np.unique(np.concatenate([[0, ng - 1], rng.integers(0, ng, size=max(0, n_cols - 2))]))
    t0 = time.perf_counter()
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    dt = time.perf_counter() - t0
    per_col = 16.0 * p.n_atoms * p.n_L * ng
    def err(Hx, Sx):
        Hg = columns_from_lower(Hx[0], ng, layout, cols)
        Sg = columns_from_lower(Sx[0], ng, layout, cols)
        return {"H": float(np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho)),
                "S": float(np.linalg.norm(Sg - So) / np.linalg.norm(So))}

    out = {"value": round(len(cols) * per_col / dt / 1e12, 6), "unit": "TFLOP/s",
           "cores": oracle.max_threads(), "kind": "oracle",
           "sample": f"{len(cols)} of {ng} columns of H and S at k-point 0 (A/B recomputed for every row), {dt:.1f} s",
           "parity_rel_err": err(H, S)}
    if H64 is not None:
        out["parity_rel_err_fp64_path"] = err(H64, S64)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1712_07206_gb300 import inputs

    oracle.build()
    p = inputs.CONFIGS[args.config]()
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    ng = len(n3)
    per_col = 16.0 * p.n_atoms * p.n_L * ng
    rng = np.random.default_rng(1)

    def step():
        cols = rng.integers(0, ng, size=args.ref_cols)
        oracle.hs_columns(p, 0, n3, cols)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = args.ref_cols * per_col / dt / 1e12
    sample = f"{args.ref_cols} random columns of H and S per step (of {ng}), workload {p.name}"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": p.name, "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def inputs_configs():
    """Workload number -> what it is (the input generator's description)."""
    from paper_1712_07206_gb300 import inputs
    return {c: (f.__doc__ or "").strip().rstrip(".") for c, f in inputs.CONFIGS.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2, choices=sorted(inputs_configs()),
                    help="workload: " + "; ".join(f"{c}: {d}" for c, d in sorted(inputs_configs().items())))
    ap.add_argument("--operands", choices=["factored", "from_ab"], default="factored")
    ap.add_argument("--slices", type=int, default=7)
    ap.add_argument("--tile-order", type=int, default=0,
                    help="0: library default; k+1 forces emulated tile order k")
    ap.add_argument("--cover", type=int, default=0, choices=[0, 1, 2],
                    help="contraction tile cover: 0 by size, 1 cyclic, 2 aligned 256-row blocks")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="fixed tile cover, order and pipeline (by size or as forced) instead of the "
                         "library's autotuner")
    ap.add_argument("--pipeline", type=int, default=0, choices=[0, 1, 2],
                    help="contraction load pipeline: 0 by size, 1 three stages of two K chunks, "
                         "2 five stages of one")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cols", type=int, default=0,
                    help="oracle columns of the CPU baseline (0: as many as --cpu-seconds allow)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--refined-cols", type=int, default=1024,
                    help="columns of the host-BLAS Alg. 3 comparator")
    ap.add_argument("--h-method", choices=list(H_METHODS), default="factored",
                    help="H as one Hermitian rank-K update after factorising T (default), by the "
                         "paper's Alg. 3 sequence (zher2k + zherkx as one L^H R contraction), or "
                         "(spherical) by the addition theorem on the workload with T replaced by "
                         "its spherical part")
    ap.add_argument("--s-method", choices=["contraction", "legendre"], default="contraction",
                    help="S by the slice contraction (default) or by the addition theorem")
    ap.add_argument("--dist-backend", choices=["nccl", "gloo"], default="nccl",
                    help="process group of N > 1 ranks (the timing reduction and barriers only)")
    ap.add_argument("--eigh", action="store_true",
                    help="also solve H c = lambda S c for k-point 0 (flapw_eigh; S must be positive "
                         "definite: 2 N_A N_L >= N_G, e.g. config 3)")
    ap.add_argument("--graph", action="store_true",
                    help="replay the captured build_HS sequence (the stage timers then read -1)")
    ap.add_argument("--ref-cols", type=int, default=32)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per contraction launch from an ncu capture")
    args = ap.parse_args()
    if args.tile_order or args.pipeline or args.cover:
        args.autotune = False  # a forced choice is measured as given
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
