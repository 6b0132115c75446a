#!/usr/bin/env python
"""Benchmark of the GB300 multigrid Poisson path; prints ONE JSON line on rank 0.

Default workload (dirichlet256): 256^3 homogeneous-Dirichlet FP64 Poisson problem split into
64 boxes of 64^3, rhs = seeded N(0,1) smoothed by one damped-Jacobi pass, V(2,2) red-black
Gauss-Seidel cycles to ||rhs - A phi||_inf <= 1e-10 ||rhs||_inf.  One step = one complete
solve (phi reset to 0, then mg_solve) with rhs already resident in HBM.  `value` is solves/s
over all ranks (each rank solves its own replica: this solve is not sharded across GPUs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload dirichlet256|periodic64|mixed512|batched512|serving|fill]
                    [--kernels-only] [--no-cpu-baseline]

Other workloads: mixed512 (512^3, FP32 inner / FP64 outer, against the FP64 solve),
batched512 (512 independent solves packed into shared launches), serving (5000 Poisson
arrivals through mg_submit/mg_poll, with latency percentiles and capacity, against a
one-solve-at-a-time FP64 server), fill (the ghost-fill microbench, fused against one launch
per copy tag).

`--impl reference` times the CPU oracle (the plain FP64 restatement under oracle/) on this
machine's host cores on the same workload, one V-cycle per step, extrapolated to a solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

WORKLOADS = {
    "dirichlet256": dict(n=256, box=64, periodic=(0, 0, 0), precision="f64",
                         desc="256^3 homogeneous Dirichlet, 64 boxes of 64^3 (phi 2 ghosts, rhs 1), "
                              "rhs = N(0,1) seed 2 smoothed by one damped-Jacobi pass, V(2,2) "
                              "red-black GS, coarsened to 2^3, tol 1e-10 relative max-norm residual"),
    "periodic64": dict(n=64, box=32, periodic=(1, 1, 1), precision="f64",
                       desc="64^3 periodic, 8 boxes of 32^3, rhs = -12 pi^2 prod sin(2 pi x) + "
                            "U(-1e-3,1e-3) seed 1, mean removed, V(2,2), tol 1e-10"),
    "mixed512": dict(n=512, box=128, periodic=(0, 0, 0), precision="mixed",
                     desc="512^3 homogeneous Dirichlet, 64 boxes of 128^3, 16 Gaussian blobs + "
                          "N(0,1e-3) seed 5, FP32 inner V(2,2) / FP64 outer residual, correction "
                          "and bottom, tol 1e-10"),
}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def make_rhs(wl):
    from paper_2403_12179_gb300 import inputs
    n = wl["n"]
    if wl is WORKLOADS["dirichlet256"]:
        return inputs.dirichlet_jacobi(n, seed=2)
    if wl is WORKLOADS["periodic64"]:
        return inputs.periodic_sine(n, seed=1)
    return inputs.gaussian_blobs(n, seed=5)


# ---- clocks ------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- distributed plumbing ----------------------------------------------------------------

def dist_init(args, backend=None):
    """One process per GPU (torchrun's RANK / WORLD_SIZE / LOCAL_RANK); NCCL on GPUs, gloo
    where there is none (the host-side tests)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, max_total_ms):
    """Units per second over all ranks: every rank processed `steps` units, and the slowest
    rank's timed region (max over ranks) took max_total_ms."""
    return world * steps / (max_total_ms / 1e3)


# ---- our arm --------------------------------------------------------------------------------

# Source files whose contents define each profiled kernel (its launch configuration included).
KERNEL_SOURCES = {
    "rbgs_half_f64": ["mg_kernels.cu", "mg_kernels.hpp"],
    "rbgs_fused_f32": ["mg_fused.cu", "mg_kernels.hpp", "mg_runtime.cu"],
    "copy_tags_f64": ["mg_kernels.cu", "mg_kernels.hpp", "mg_runtime.cu"],
}


def kernel_source_hash(kernel):
    import hashlib
    src = os.path.join(ROOT, "paper_2403_12179_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def roofline_traffic(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (the summary records the source hash); else None."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    traffic = src_hash = None
    for line in open(p):
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":")[1])
        if line.startswith("source_hash:"):
            src_hash = line.split(":")[1].strip()
    return traffic if src_hash == kernel_source_hash(kernel) else None


def run_ours(args, wl_name):
    import numpy as np
    import torch
    from paper_2403_12179_gb300 import mg

    wl = WORKLOADS[wl_name]
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    n, box = wl["n"], wl["box"]
    dom = (n - 1,) * 3
    cells = n ** 3
    h = 1.0 / n
    ctx = mg.mg_init(local)
    stream = torch.cuda.Stream()
    mg.mg_set_stream(ctx, stream)
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), dom, (box,) * 3)
    rhs_np = make_rhs(wl)
    fr = mg.mg_fab_alloc(ctx, ba, 1, 1)
    fp = mg.mg_fab_alloc(ctx, ba, 1, 2)
    rhs_host = torch.from_numpy(rhs_np).pin_memory()
    out_host = torch.empty_like(rhs_host).pin_memory()
    rhs_dev = rhs_host.cuda()
    mg.mg_fab_copy_from_dense(ctx, fr, rhs_dev.data_ptr(), False, stream)
    stream.synchronize()
    del rhs_dev
    bc = mg.make_bc(wl["periodic"])
    prec = mg.MG_PREC_MIXED if wl["precision"] == "mixed" else mg.MG_PREC_F64
    opt = mg.make_options(precision=prec)

    def step():
        mg.mg_fab_set_val(ctx, fp, 0.0, True, stream)
        return mg.mg_solve(ctx, fr, fp, bc, 1e-10, opt)

    for _ in range(args.warmup):
        res = step()
    if res.status != 0:
        raise RuntimeError(f"solve failed: {res.as_dict()}")

    # ---- timed region: K solves, inputs resident, events on the solve stream around each
    # solve; between solves (outside the events) a 256 MiB write flushes L2
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    mg.mg_sweep_timing(ctx, True)   # time the finest-level half-sweep inside the solves
    l0 = mg_launches()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    results = []
    torch.cuda.nvtx.range_push("timed")  # (lets a profiler keep the timed solves only)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev0[k].record(stream)
            results.append(step())
            ev1[k].record(stream)
    torch.cuda.nvtx.range_pop()
    stream.synchronize()
    torch.cuda.synchronize()
    launches = mg_launches() - l0      # the library's own kernels (the flush is torch's)
    sweep_ms, sweep_n = mg.mg_sweep_timing(ctx, False)
    clocks = clk.stop()
    barrier(world)
    per = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    total_ms = max_over_ranks(sum(per), world)
    del flush
    value = whole_job_rate(world, args.steps, total_ms)
    vcycles = results[-1].vcycles
    assert all(r.status == 0 and r.rel_resid <= 1e-10 for r in results)

    # ---- dominant kernels on the fine level, timed alone on the solve stream
    kt = kernel_timings(ctx, stream, ba, fp, fr, bc, h, cells, box)
    if sweep_n:
        kt["rbgs_half_f64_in_solve"] = sweep_ms / sweep_n / 1e3
    roof = roofline(kt, wl_name, prec == mg.MG_PREC_F64, clocks, sweep_n)

    # ---- end to end through the C ABI with host buffers
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mg.mg_fab_copy_from_dense(ctx, fr, rhs_host.data_ptr(), True, stream)
        mg.mg_fab_set_val(ctx, fp, 0.0, True, stream)
        r = mg.mg_solve(ctx, fr, fp, bc, 1e-10, opt)
        mg.mg_fab_copy_to_dense(ctx, fp, out_host.data_ptr(), True, stream)
        stream.synchronize()
        assert r.status == 0
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    nbytes = rhs_host.numel() * rhs_host.element_size()

    line = {
        "metric": f"solves/s to 1e-10 relative residual ({wl_name})",
        "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == mg.MG_PREC_F64 else "f32 inner / f64 outer",
        "data": "synthetic",
        "config": {"workload": wl_name, "description": wl["desc"], "cells": cells,
                   "boxes": (n // box) ** 3, "parallelism": f"replicas x{world}",
                   "l2": "flushed before every timed solve (256 MiB write outside the "
                         f"timed events); phi and rhs are FP64 fields of {round(cells * 8 / 2**20)} MiB each"},
        "latency_ms": {"p50": round(statistics.median(per), 3),
                       "p99": round(float(np.percentile(per, 99)), 3)},
        "vcycles": vcycles, "rel_resid": results[-1].rel_resid,
        "cell_updates_per_s": round(cells * vcycles * (2 * (opt.nu1 + opt.nu2)) / (total_ms / args.steps / 1e3), 1),
        "roofline": roof,
        "e2e": {"value": round(world * e2e_steps / t_e2e, 3), "unit": "solves/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if wl_name == "periodic64":
        # error against the continuous solution prod sin(2 pi x_d) (second order in h; the
        # rhs noise adds at most ~1e-3 / lambda_min)
        x = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n
        sx = torch.sin(2 * np.pi * x)
        u = sx[:, None, None] * sx[None, :, None] * sx[None, None, :]
        a = _fab_to_dense(ctx, fp, (n,) * 3, stream)
        line["error_vs_continuous"] = {"max_abs": float((a - u).abs().max()), "h": 1.0 / n}
        del a, u
    if prec == mg.MG_PREC_MIXED:
        # the plain FP64 path on the same problem: time and the difference of the answers
        # (P7: two answers that both meet tol differ by at most 2 * 0.06 * tol * ||rhs||)
        fp64 = mg.mg_fab_alloc(ctx, ba, 1, 2)
        opt64 = mg.make_options()
        mg.mg_solve(ctx, fr, fp64, bc, 1e-10, opt64)
        t64 = []
        for _ in range(2):
            mg.mg_fab_set_val(ctx, fp64, 0.0, True, stream)
            stream.synchronize()
            t = time.perf_counter()
            r64 = mg.mg_solve(ctx, fr, fp64, bc, 1e-10, opt64)
            t64.append(time.perf_counter() - t)
        a = _fab_to_dense(ctx, fp, (n,) * 3, stream)
        b = _fab_to_dense(ctx, fp64, (n,) * 3, stream)
        diff = float((a - b).abs().max())
        del a, b
        line["vs_f64"] = {"f64_ms_per_solve": round(min(t64) * 1e3, 3), "f64_vcycles": r64.vcycles,
                          "max_abs_diff": diff,
                          "p7_bound": 2 * 0.06 * 1e-10 * float(np.abs(rhs_np).max())}
        mg.mg_fab_free(ctx, fp64, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl_name, vcycles)
    mg.mg_finalize(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


FP64_LANES_PER_SM_CLK = 2      # GB300 FP64 pipe: lane-operations per SM per clock
N_SM = 152
FP64_INST_PER_UPDATE = 7       # 5 DADD (neighbour sum) + 1 DFMA + 1 DMUL
FP64_INST_PER_RESIDUAL = 7     # 5 DADD + 2 DFMA


def _time(stream, fn, reps):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn(0)
    stream.synchronize()
    a.record(stream)
    for k in range(reps):
        fn(k)
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / reps / 1e3


def kernel_timings(ctx, stream, ba, fp, fr, bc, h, cells, box, reps=40):
    """Average launch durations (s) of the fine-level kernels, each launched back to back
    on `stream` between two CUDA events: FP64 half-sweep, FP64 residual + norm, FP32 fused
    sweep (out of place), FP32 half-sweep."""
    from paper_2403_12179_gb300 import mg
    out = {}
    mg.mg_fill_boundary(ctx, fp, bc, stream)
    # the FP64 half-sweep as the solver runs it on regular box grids (neighbour boxes read
    # directly), and with ghost cells
    out["rbgs_half_f64"] = _time(stream, lambda k: mg.mg_smooth(
        ctx, fp, fr, bc, h, (k & 1) | mg.MG_SMOOTH_DIRECT_READS, stream), reps)
    out["rbgs_half_f64_ghosts"] = _time(stream, lambda k: mg.mg_smooth(ctx, fp, fr, bc, h, k & 1, stream), reps)
    out["residual_f64"] = _time(stream, lambda k: mg.mg_residual(ctx, fp, fr, 0, h, False, stream), reps)
    out["fill_f64_g2"] = _time(stream, lambda k: mg.mg_fill_boundary(ctx, fp, bc, stream), reps)
    # FP32 fields of the same layout (the mixed form's inner cycle)
    a32 = mg.mg_fab_alloc(ctx, ba, 1, 2, mg.MG_F32)
    b32 = mg.mg_fab_alloc(ctx, ba, 1, 2, mg.MG_F32)
    r32 = mg.mg_fab_alloc(ctx, ba, 1, 1, mg.MG_F32)
    mg.mg_fab_set_val(ctx, r32, 1.0, True, stream)
    mg.mg_fill_boundary(ctx, a32, bc, stream)
    mg.mg_fill_boundary(ctx, b32, bc, stream)
    pair = (a32, b32)
    out["rbgs_fused_f32"] = _time(stream, lambda k: mg.mg_smooth_fused(ctx, pair[k & 1], r32, pair[(k + 1) & 1], bc, h, stream), reps)
    out["rbgs_half_f32"] = _time(stream, lambda k: mg.mg_smooth(ctx, a32, r32, bc, h, k & 1, stream), reps)
    for f in (a32, b32, r32):
        mg.mg_fab_free(ctx, f, stream)
    stream.synchronize()
    return out


def roofline(kt, wl_name, f64, clocks, in_solve_launches=0):
    peaks, src = load_peaks()
    cells = WORKLOADS[wl_name]["n"] ** 3
    sm_mhz = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = FP64_LANES_PER_SM_CLK * N_SM * sm_mhz * 1e6 / 1e9      # G lane-ops/s
    hbm = peaks["hbm_gbs"]
    # the FP64 half-sweep's duration inside the timed solves when measured there, else the
    # separate timing loop
    t = kt.get("rbgs_half_f64_in_solve") or kt["rbgs_half_f64"]
    half_ops = FP64_INST_PER_UPDATE * cells / 2
    extra = {
        "rbgs_half_f64": {"launch_us": round(kt["rbgs_half_f64"] * 1e6, 2),
                          "hbm_frac": round(16 * cells / kt["rbgs_half_f64"] / 1e9 / hbm, 4),
                          "fp64_frac": round(half_ops / kt["rbgs_half_f64"] / 1e9 / fp64_peak, 4)},
        "rbgs_half_f64_ghosts": {"launch_us": round(kt["rbgs_half_f64_ghosts"] * 1e6, 2)},
        "residual_f64": {"launch_us": round(kt["residual_f64"] * 1e6, 2),
                         "fp64_frac": round(FP64_INST_PER_RESIDUAL * cells / kt["residual_f64"] / 1e9 / fp64_peak, 4),
                         "hbm_frac": round(16 * cells / kt["residual_f64"] / 1e9 / hbm, 4)},
        "fill_f64_g2": {"launch_us": round(kt["fill_f64_g2"] * 1e6, 2)},
        "rbgs_fused_f32": {"launch_us": round(kt["rbgs_fused_f32"] * 1e6, 2),
                           "hbm_frac": round(12 * cells / kt["rbgs_fused_f32"] / 1e9 / hbm, 4)},
        "rbgs_half_f32": {"launch_us": round(kt["rbgs_half_f32"] * 1e6, 2),
                          "hbm_frac": round(8 * cells / kt["rbgs_half_f32"] / 1e9 / hbm, 4)},
    }
    if f64:
        ach = half_ops / t / 1e9
        where = (f"average of {in_solve_launches} launches inside the timed solves (CUDA events "
                 "on the solve stream)" if in_solve_launches else "separate timing loop")
        return {"kernel": "k_rbgs_half<double> (one colour, finest level, neighbour boxes read directly)",
                "bound": "alu", "measured": where,
                "achieved": round(ach, 1), "peak": round(fp64_peak, 1),
                "unit": "G FP64 lane-ops/s", "frac": round(ach / fp64_peak, 4),
                "peak_source": f"derived: {FP64_LANES_PER_SM_CLK} FP64 lanes/clk/SM x {N_SM} SMs x {sm_mhz:.0f} MHz",
                "algorithmic_ops_per_launch": half_ops,
                "traffic": roofline_traffic("rbgs_half_f64", wl_name), "kernels": extra}
    t = kt["rbgs_fused_f32"]
    ach = 12 * cells / t / 1e9
    return {"kernel": "k_rbgs_fused<float> (full sweep, fine level)", "bound": "hbm",
            "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
            "peak_source": src, "algorithmic_bytes_per_launch": 12 * cells,
            "traffic": roofline_traffic("rbgs_fused_f32", wl_name), "kernels": extra}


def run_kernels_only(args, wl_name):
    """Set up the workload's fine level and run only the kernel timing loops (for ncu)."""
    import torch
    from paper_2403_12179_gb300 import mg
    wl = WORKLOADS[wl_name]
    n, box = wl["n"], wl["box"]
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    mg.mg_set_stream(ctx, stream)
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
    fr = mg.mg_fab_alloc(ctx, ba, 1, 1)
    fp = mg.mg_fab_alloc(ctx, ba, 1, 2)
    mg.mg_fab_set_val(ctx, fr, 1.0, True, stream)
    kt = kernel_timings(ctx, stream, ba, fp, fr, mg.make_bc(wl["periodic"]), 1.0 / n, n ** 3, box,
                        reps=args.steps)
    mg.mg_finalize(ctx)
    print(json.dumps({"kernels_only": wl_name, "launch_s": kt}))


# ---- other workloads: batched, serving, mixed vs FP64, ghost-fill microbench ----------------

def _dense_to_fab(ctx, ba, dense_dev, ng, stream=None):
    from paper_2403_12179_gb300 import mg
    fab = mg.mg_fab_alloc(ctx, ba, 1, ng)
    mg.mg_fab_copy_from_dense(ctx, fab, dense_dev.data_ptr(), False, stream)
    return fab


def _fab_to_dense(ctx, fab, shape, stream=None):
    import torch
    from paper_2403_12179_gb300 import mg
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    mg.mg_fab_copy_to_dense(ctx, fab, out.data_ptr(), False, stream)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    return out


def run_batched(args):
    """512 independent periodic problems (edges from {32,48,64,96,128}, 32^3 boxes): all
    packed into one launch per V-cycle stage, FP64 and mixed; against the same problems
    solved one at a time with mg_solve (FP64)."""
    import numpy as np
    import torch
    from paper_2403_12179_gb300 import inputs, mg
    probs = inputs.batched_periodic(args.count, seed=4)
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    mg.mg_set_stream(ctx, stream)
    fr, fp, shapes = [], [], []
    for pb in probs:
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (pb.n - 1,) * 3, (pb.box,) * 3)
        d = torch.from_numpy(pb.rhs()).cuda()
        fr.append(_dense_to_fab(ctx, ba, d, 1, stream))
        fp.append(mg.mg_fab_alloc(ctx, ba, 1, 2))
        shapes.append((pb.n,) * 3)
    stream.synchronize()
    bcs = [mg.make_bc((1, 1, 1))] * len(probs)
    cells = sum(pb.n ** 3 for pb in probs)

    def batch(prec):
        for f in fp:
            mg.mg_fab_set_val(ctx, f, 0.0, True, stream)
        t = time.perf_counter()
        res = mg.mg_solve_batch(ctx, fr, fp, bcs, 1e-10, mg.make_options(precision=prec))
        dt = time.perf_counter() - t
        assert all(r.status == 0 and r.rel_resid <= 1e-10 for r in res), "batched solve failed"
        return dt, res

    out, vcs = {}, {}
    for name, prec in (("mixed", mg.MG_PREC_MIXED), ("f64", mg.MG_PREC_F64)):
        for _ in range(max(1, args.warmup)):
            batch(prec)
        runs = [batch(prec) for _ in range(args.steps)]
        out[name] = statistics.median(r[0] for r in runs)
        vcs[name] = [r.vcycles for r in runs[-1][1]]
    phis64 = [_fab_to_dense(ctx, f, sh, stream) for f, sh in zip(fp, shapes)]
    batch(mg.MG_PREC_MIXED)
    diff = 0.0
    for f, sh, p64 in zip(fp, shapes, phis64):
        pm = _fab_to_dense(ctx, f, sh, stream)
        d = (pm - pm.mean()) - (p64 - p64.mean())
        diff = max(diff, float(d.abs().max()))
    # one solve at a time, FP64, same problems
    seq = []
    for f in fp:
        mg.mg_fab_set_val(ctx, f, 0.0, True, stream)
    for a, b in zip(fr, fp):                       # warm: hierarchies and graphs exist
        mg.mg_solve(ctx, a, b, bcs[0], 1e-10)
    for f in fp:
        mg.mg_fab_set_val(ctx, f, 0.0, True, stream)
    stream.synchronize()
    t = time.perf_counter()
    for a, b in zip(fr, fp):
        r = mg.mg_solve(ctx, a, b, bcs[0], 1e-10)
        seq.append(r.vcycles)
    t_seq = time.perf_counter() - t
    n = len(probs)
    line = {"metric": f"solves/s, {n} batched periodic problems to 1e-10 (mixed precision)",
            "value": round(n / out["mixed"], 2), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(out["mixed"] * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": "batched512", "problems": n, "cells": cells,
                       "edges": "32/48/64/96/128 (seed 4)", "box": 32},
            "f64_batched_solves_per_s": round(n / out["f64"], 2),
            "f64_one_at_a_time_solves_per_s": round(n / t_seq, 2),
            "cell_updates_per_s_mixed": round(sum(pb.n ** 3 * 4 * v for pb, v in
                                                  zip(probs, vcs["mixed"])) / out["mixed"], 1),
            "cell_updates": "finest level: 4 per cell per V-cycle (V(2,2)), each problem's own count",
            "max_abs_diff_mixed_vs_f64_mod_const": diff}
    mg.mg_finalize(ctx)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batched(probs)
    print(json.dumps(line), flush=True)


def cpu_baseline_batched(probs, budget_s=10.0):
    """The oracle's mixed-precision solve on the batch's problems in order, whole solves, for
    about budget_s seconds (a leading subset of the batch)."""
    import oracle
    oracle.build()
    count, t = 0, time.perf_counter()
    for pb in probs:
        dom = (pb.n - 1,) * 3
        boxes = oracle.chop((0, 0, 0), dom, (pb.box,) * 3)
        _, st, _, _ = oracle.solve((0, 0, 0), dom, (1, 1, 1), boxes, 1.0 / pb.n, pb.rhs(), mixed=True)
        if st != 0:
            raise RuntimeError("oracle solve failed")
        count += 1
        if time.perf_counter() - t >= budget_s:
            break
    el = time.perf_counter() - t
    return {"value": round(count / el, 6), "unit": "solves/s",
            "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
            "sample": f"the first {count} of the {len(probs)} problems, whole oracle mixed solves, "
                      f"in {el:.1f} s"}


def run_serving(args):
    """Poisson arrivals (200/s), edges {32,64,128,256} p={.4,.3,.2,.1}, periodic/Dirichlet,
    32^3 or 64^3 boxes: real-time replay through mg_submit/mg_poll (mixed precision,
    continuous batching), against a one-at-a-time FP64 server (mg_solve in arrival order,
    latencies from measured service times).  Both are warmed up with one request per shape.
    Capacity: the mixed server with every request queued at once; the FP64 server's is one
    over its mean service time."""
    import threading
    import numpy as np
    import torch
    from paper_2403_12179_gb300 import inputs, mg
    reqs = inputs.serving_requests(args.requests, seed=6)
    ctx = mg.mg_init(0)
    fabs = []
    gen = torch.Generator(device="cuda")
    for rq in reqs:
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (rq.n - 1,) * 3, (rq.box,) * 3)
        gen.manual_seed(rq.seed)
        d = torch.randn((rq.n,) * 3, dtype=torch.float64, device="cuda", generator=gen)
        if rq.periodic:
            d -= d.mean()
        fr = _dense_to_fab(ctx, ba, d, 1)
        fp = mg.mg_fab_alloc(ctx, ba, 1, 2)
        fabs.append((fr, fp, mg.make_bc((1, 1, 1) if rq.periodic else (0, 0, 0))))
    torch.cuda.synchronize()
    opt = mg.make_options(precision=mg.MG_PREC_MIXED)
    shapes = sorted({(rq.n, rq.box, rq.periodic) for rq in reqs})

    def warm_fabs(ctx, n, box, per):
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
        d = torch.randn((n,) * 3, dtype=torch.float64, device="cuda", generator=gen)
        if per:
            d -= d.mean()
        return _dense_to_fab(ctx, ba, d, 1), mg.mg_fab_alloc(ctx, ba, 1, 2), \
            mg.make_bc((1, 1, 1) if per else (0, 0, 0))

    # warm-up (untimed): one request of every shape, so that one-time work (fused-sweep
    # autotuning, first launches) is not part of the replay
    gen.manual_seed(7)
    warm = [warm_fabs(ctx, *sh) for sh in shapes]
    for t in [mg.mg_submit(ctx, fr, fp, bc, 1e-10, opt) for fr, fp, bc in warm]:
        mg.mg_poll(ctx, t, -1)
    for fr, fp, _ in warm:
        mg.mg_fab_free(ctx, fr)
        mg.mg_fab_free(ctx, fp)
    stats0 = mg.mg_server_stats_get(ctx)
    results = [None] * len(reqs)
    tickets = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def poller():
        for i in range(len(reqs)):
            ready.acquire()
            rc, r = mg.mg_poll(ctx, tickets[i], -1)
            results[i] = r

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for i, rq in enumerate(reqs):
        delay = t0 + rq.t_arrive - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        fr, fp, bc = fabs[i]
        tickets[i] = mg.mg_submit(ctx, fr, fp, bc, 1e-10, opt)
        ready.release()
    th.join()
    wall = max(r.t_end for r in results) - min(r.t_start for r in results)
    lat = np.array([r.seconds for r in results]) * 1e3
    ok = all(r.status == 0 and r.rel_resid <= 1e-10 for r in results)
    stats = mg.mg_server_stats_get(ctx)
    stats = {k: (v - stats0[k] if k != "max_active" else v) for k, v in stats.items()}
    # capacity: the same requests all queued at once (phi reset to the zero guess); the
    # scheduler admits them as the pool allows
    for _, fp, _ in fabs:
        mg.mg_fab_set_val(ctx, fp, 0.0, True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    tk = [mg.mg_submit(ctx, fr, fp, bc, 1e-10, opt) for fr, fp, bc in fabs]
    burst = [mg.mg_poll(ctx, x, -1)[1] for x in tk]
    cap = len(reqs) / (time.perf_counter() - t)
    ok = ok and all(r.status == 0 and r.rel_resid <= 1e-10 for r in burst)
    mg.mg_finalize(ctx)
    # one-at-a-time FP64 server on the same requests (warmed up the same way)
    ctx = mg.mg_init(0)
    gen.manual_seed(7)
    for sh in shapes:
        fr, fp, bc = warm_fabs(ctx, *sh)
        mg.mg_solve(ctx, fr, fp, bc, 1e-10)
        mg.mg_fab_free(ctx, fr)
        mg.mg_fab_free(ctx, fp)
    svc = []
    for i, rq in enumerate(reqs):
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (rq.n - 1,) * 3, (rq.box,) * 3)
        gen.manual_seed(rq.seed)
        d = torch.randn((rq.n,) * 3, dtype=torch.float64, device="cuda", generator=gen)
        if rq.periodic:
            d -= d.mean()
        fr = _dense_to_fab(ctx, ba, d, 1)
        fp = mg.mg_fab_alloc(ctx, ba, 1, 2)
        bc = mg.make_bc((1, 1, 1) if rq.periodic else (0, 0, 0))
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = mg.mg_solve(ctx, fr, fp, bc, 1e-10)
        svc.append(time.perf_counter() - t)
        ok = ok and r.status == 0
        mg.mg_fab_free(ctx, fr)
        mg.mg_fab_free(ctx, fp)
    mg.mg_finalize(ctx)
    end, lat64 = 0.0, []
    for rq, sv in zip(reqs, svc):
        start = max(rq.t_arrive, end)
        end = start + sv
        lat64.append((end - rq.t_arrive) * 1e3)
    lat64 = np.array(lat64)
    wall64 = end - reqs[0].t_arrive
    n = len(reqs)
    line = {"metric": f"served solves/s and latency, {n} Poisson-arrival requests at 200/s",
            "value": round(n / wall, 2), "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 outer", "data": "synthetic (torch Philox rhs per request seed)",
            "config": {"workload": "serving", "requests": n, "rate_per_s": 200,
                       "warmup": f"one untimed request per shape ({len(shapes)} shapes) before the replay",
                       "edges": "32/64/128/256 p=.4/.3/.2/.1", "bc": "periodic/Dirichlet 50/50",
                       "box": "32 or 64"},
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 2),
                           "p99": round(float(np.percentile(lat, 99)), 2)},
            "all_converged_to_1e-10": ok, "scheduler": stats,
            "capacity_solves_per_s": round(cap, 2),
            "f64_one_at_a_time": {"solves_per_s": round(n / wall64, 2),
                                  "capacity_solves_per_s": round(1.0 / float(np.mean(svc)), 2),
                                  "latency_ms": {"p50": round(float(np.percentile(lat64, 50)), 2),
                                                 "p99": round(float(np.percentile(lat64, 99)), 2)},
                                  "mean_service_ms": round(float(np.mean(svc)) * 1e3, 3)}}
    print(json.dumps(line), flush=True)


def run_fill(args):
    """FillBoundary microbench: 256^3 periodic, 64 boxes of 64^3, 4 FP64 components, 2 ghost
    layers; one fill kernel per call."""
    import torch
    from paper_2403_12179_gb300 import inputs, mg
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), (255,) * 3, (64,) * 3)
    fab = mg.mg_fab_alloc(ctx, ba, 4, 2)
    d = torch.from_numpy(inputs.fill_microbench(256, seed=3)).cuda()
    mg.mg_fab_copy_from_dense(ctx, fab, d.data_ptr(), False, stream)
    bc = mg.make_bc((1, 1, 1))
    for _ in range(args.warmup):
        mg.mg_fill_boundary(ctx, fab, bc, stream)
    t = _time(stream, lambda k: mg.mg_fill_boundary(ctx, fab, bc, stream), args.steps * 10)
    # the unfused form (one launch per copy tag), the paper's Sec. 3.2 comparison
    t_unfused = _time(stream, lambda k: mg.mg_fill_boundary_unfused(ctx, fab, bc, stream), args.steps)
    ntags = len(mg.mg_copy_tags(ctx, ba, bc, 2))
    ghost = 64 * (68 ** 3 - 64 ** 3)
    nbytes = ghost * 4 * 8 * 2
    peaks, src = load_peaks()
    ach = nbytes / t / 1e9
    line = {"metric": "FillBoundary time per fill (256^3, 64 boxes, 4 comps, 2 ghosts, periodic)",
            "value": round(t * 1e6, 2), "unit": "us", "n_gpus": 1, "steps": args.steps * 10,
            "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fill", "ghost_cells": ghost, "bytes_per_fill": nbytes},
            "unfused": {"us_per_fill": round(t_unfused * 1e6, 2), "launches_per_fill": ntags,
                        "fused_speedup": round(t_unfused / t, 2)},
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                         "peak_source": src, "traffic": roofline_traffic("copy_tags_f64", "fill")}}
    mg.mg_finalize(ctx)
    print(json.dumps(line), flush=True)


def mg_launches():
    import ctypes
    from paper_2403_12179_gb300 import mg
    n = ctypes.c_int64()
    mg.lib().mg_kernel_launches(ctypes.byref(n))
    return n.value


# ---- the oracle on the host cores ----------------------------------------------------------

def oracle_sample(wl_name, vcycles=None):
    """Time the oracle on the workload: setup + norm (0 V-cycles) and one V-cycle; solve time
    extrapolated as t0 + vcycles * (t1 - t0).  If vcycles is None it is taken from a full
    oracle solve (timed too)."""
    import oracle
    wl = WORKLOADS[wl_name]
    n, box = wl["n"], wl["box"]
    dom = (n - 1,) * 3
    rhs = make_rhs(wl)
    boxes = oracle.chop((0, 0, 0), dom, (box,) * 3)
    mixed = wl["precision"] == "mixed"
    oracle.build()
    t = time.perf_counter()
    oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs, fixed_vcycles=0, mixed=mixed)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs, fixed_vcycles=1, mixed=mixed)
    t1 = time.perf_counter() - t
    return t0, t1, max(t1 - t0, 1e-9)


def cpu_baseline(wl_name, vcycles, budget_s=10.0):
    """The oracle as it stands on the host cores, on about budget_s seconds of work: whole
    solves (the GPU's V-cycle count, fixed) repeated while they fit, else runs with one
    V-cycle repeated and extrapolated to the solve.  Beside it, the same oracle on one thread
    (one setup run and one one-V-cycle run, extrapolated the same way)."""
    out = _cpu_baseline_all_cores(wl_name, vcycles, budget_s)
    if 1.0 / out["value"] > 2.0:  # one thread would take too long for a default run
        return out
    import oracle
    oracle.set_threads(1)
    try:
        t0, t1, tv = oracle_sample(wl_name)
    finally:
        oracle.set_threads(int(os.environ["OMP_NUM_THREADS"]))
    est = t0 + vcycles * tv
    out["single_thread"] = {"value": round(1.0 / est, 6), "unit": "solves/s", "cores": 1,
                            "sample": f"{wl_name}: one run with 0 V-cycles ({t0:.2f} s) and one "
                                      f"with 1 ({t1:.2f} s) on one thread, extrapolated to "
                                      f"{vcycles} V-cycles ({est:.2f} s)"}
    return out


def _cpu_baseline_all_cores(wl_name, vcycles, budget_s):
    import oracle
    wl = WORKLOADS[wl_name]
    n, box = wl["n"], wl["box"]
    dom = (n - 1,) * 3
    rhs = make_rhs(wl)
    boxes = oracle.chop((0, 0, 0), dom, (box,) * 3)
    mixed = wl["precision"] == "mixed"
    t0, t1, tv = oracle_sample(wl_name)
    est = t0 + vcycles * tv
    cores = int(os.environ["OMP_NUM_THREADS"])
    run = lambda k: oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs,
                                 fixed_vcycles=k, mixed=mixed)
    count, t = 0, time.perf_counter()
    if est <= budget_s / 2:
        while count == 0 or time.perf_counter() - t < budget_s:
            run(vcycles)
            count += 1
        el = time.perf_counter() - t
        return {"value": round(count / el, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": f"{wl_name}: {count} whole oracle solves ({vcycles} V-cycles each) "
                          f"in {el:.1f} s"}
    while count == 0 or time.perf_counter() - t < budget_s:
        run(1)
        count += 1
    t1 = (time.perf_counter() - t) / count
    est = t0 + vcycles * max(t1 - t0, 1e-9)
    return {"value": round(1.0 / est, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{wl_name}: {count} oracle runs with 1 V-cycle (mean {t1:.2f} s) and one "
                      f"with 0 ({t0:.2f} s); solve time extrapolated to {vcycles} V-cycles "
                      f"({est:.2f} s)"}


def run_reference(args, wl_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[wl_name]
    n, box = wl["n"], wl["box"]
    dom = (n - 1,) * 3
    rhs = make_rhs(wl)
    boxes = oracle.chop((0, 0, 0), dom, (box,) * 3)
    mixed = wl["precision"] == "mixed"
    oracle.build()
    # V-cycle count of the oracle's own solve (from its convergence history on 1 cycle would
    # be a guess; the full solve is run once, untimed, when it fits in a few minutes)
    _, st, vcycles, _ = oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs, mixed=mixed)
    t = time.perf_counter()
    oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs, fixed_vcycles=0, mixed=mixed)
    t0 = time.perf_counter() - t
    for _ in range(args.warmup):
        oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs, fixed_vcycles=1, mixed=mixed)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.solve((0, 0, 0), dom, wl["periodic"], boxes, 1.0 / n, rhs, fixed_vcycles=1, mixed=mixed)
        times.append(time.perf_counter() - t)
    t1 = statistics.median(times)
    est = t0 + vcycles * max(t1 - t0, 1e-9)
    value = 1.0 / est
    cores = int(os.environ["OMP_NUM_THREADS"])
    line = {"impl": "reference", "metric": f"solves/s to 1e-10 relative residual ({wl_name})",
            "value": round(value, 6), "unit": "solves/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t1 * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl_name, "description": wl["desc"]},
            "vcycles": vcycles,
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"each step = oracle run with 1 V-cycle (median {t1:.2f} s); "
                                       f"setup + norm run {t0:.2f} s; solve time extrapolated to "
                                       f"the oracle's {vcycles} V-cycles"},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dirichlet256",
                    choices=sorted(WORKLOADS) + ["batched512", "serving", "fill"])
    ap.add_argument("--count", type=int, default=512, help="problems in batched512")
    ap.add_argument("--requests", type=int, default=5000, help="requests in serving")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time only the fine-level kernels (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.workload == "batched512":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "fill":
        run_fill(args)
    elif args.kernels_only:
        run_kernels_only(args, args.workload)
    elif args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
