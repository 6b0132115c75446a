#!/usr/bin/env python
"""Benchmark of the GB300 multigrid Poisson path; prints ONE JSON line on rank 0.

Headline (dirichlet256): 256^3 homogeneous-Dirichlet FP64 Poisson problem split into 64
boxes of 64^3, rhs = seeded N(0,1) smoothed by one damped-Jacobi pass, V(2,2) red-black
Gauss-Seidel cycles to ||rhs - A phi||_inf <= 1e-10 ||rhs||_inf.  One step = one complete
solve (phi reset to 0, then mg_solve) with rhs already resident in HBM.  `value` is solves/s
over all ranks (each rank solves its own replica: this solve is not sharded across GPUs).

On one GPU the same line also carries the other workloads as sub-objects, each with its own
clock record: mixed512 (512^3, FP32 inner / FP64 outer, against the FP64 solve), batched512
(512 independent solves packed into shared launches, mixed and FP64, against FP64 one at a
time), serving (5000 Poisson arrivals whose data lives in host memory, through
mg_submit_host, with latency percentiles and capacity, against a one-solve-at-a-time FP64
server), fill (the ghost-fill microbench, fused against one launch per copy tag), triad
(the STREAM triad of the paper's Sec. 3.1-3.2, per-box launches against one launch), amr (a
two-level composite solve, 128^3 coarse with the middle half refined) and the measured FP64
rate that the FP64 kernels' roofline uses.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload dirichlet256|periodic64|mixed256|mixed512|batched512|serving|fill|triad|amr]
                    [--headline-only] [--kernels-only] [--no-cpu-baseline]

`--workload X` prints X's line alone; `--headline-only` skips the sub-objects.
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
    "mixed256": dict(n=256, box=64, periodic=(0, 0, 0), precision="mixed",
                     desc="256^3 homogeneous Dirichlet, 64 boxes of 64^3, rhs = N(0,1) seed 2 "
                          "smoothed by one damped-Jacobi pass, FP32 inner V(2,2) (2 per outer "
                          "iteration) / FP64 outer residual, correction and bottom, tol 1e-10 (a "
                          "smaller mixed case, for profiling)"),
    "mixed512": dict(n=512, box=128, periodic=(0, 0, 0), precision="mixed",
                     desc="512^3 homogeneous Dirichlet, 64 boxes of 128^3, 16 Gaussian blobs + "
                          "N(0,1e-3) seed 5, FP32 inner V(2,2) (2 per outer iteration) / FP64 "
                          "outer residual, correction and bottom, tol 1e-10"),
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
    if wl is WORKLOADS["dirichlet256"] or wl is WORKLOADS["mixed256"]:
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
    fp64 = measure_fp64_peak(stream, local)
    roof = roofline(kt, wl_name, prec == mg.MG_PREC_F64, fp64, sweep_n)

    # ---- end to end through the C ABI with host buffers: every step copies its rhs in from
    # pinned host memory and its phi out to pinned host memory.  Two fab sets, the copies on a
    # stream of their own: step k+1's copy in and step k-1's copy out run while step k solves
    # (the first copy in and the last copy out are exposed).
    e2e_steps = max(2, min(args.steps, 6))
    cstream = torch.cuda.Stream()
    sets = [(fr, fp), (mg.mg_fab_alloc(ctx, ba, 1, 1), mg.mg_fab_alloc(ctx, ba, 1, 2))]
    outs = [out_host, torch.empty_like(rhs_host).pin_memory()]
    mg.mg_fab_copy_from_dense(ctx, sets[1][0], rhs_host.data_ptr(), True, stream)
    mg.mg_fab_set_val(ctx, sets[1][1], 0.0, True, stream)
    mg.mg_solve(ctx, sets[1][0], sets[1][1], bc, 1e-10, opt)  # its hierarchy and graph
    copied_in = [torch.cuda.Event() for _ in range(2)]
    solved = [torch.cuda.Event() for _ in range(2)]

    def copy_in(k):  # (cstream order puts it after the copy out of the set's previous step)
        a, b = sets[k % 2]
        mg.mg_fab_copy_from_dense(ctx, a, rhs_host.data_ptr(), True, cstream)
        mg.mg_fab_set_val(ctx, b, 0.0, True, cstream)
        copied_in[k % 2].record(cstream)

    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    copy_in(0)
    for k in range(e2e_steps):
        if k + 1 < e2e_steps:
            copy_in(k + 1)
        stream.wait_event(copied_in[k % 2])
        r = mg.mg_solve(ctx, sets[k % 2][0], sets[k % 2][1], bc, 1e-10, opt)
        assert r.status == 0
        solved[k % 2].record(stream)
        cstream.wait_event(solved[k % 2])
        mg.mg_fab_copy_to_dense(ctx, sets[k % 2][1], outs[k % 2].data_ptr(), True, cstream)
    cstream.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    assert torch.equal(outs[0], outs[1]), "pipelined end-to-end solves differ"
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
        "cell_updates_per_s": round(cells * vcycles * (opt.nu1 + opt.nu2) / (total_ms / args.steps / 1e3), 1),
        "cell_updates": "finest level only: nu1 + nu2 = 4 updates per cell per V-cycle",
        "roofline": roof,
        "e2e": {"value": round(world * e2e_steps / t_e2e, 3), "unit": "solves/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                "how": "mg_fab_copy_from_dense (pinned host rhs) + mg_solve + mg_fab_copy_to_dense "
                       "(pinned host phi) per step, host wall time; two fab sets, copies on their "
                       "own stream overlapping the neighbouring steps' solves"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "fp64_peak": fp64,
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
    del fr, fp
    torch.cuda.empty_cache()
    if wl_name == "dirichlet256" and world == 1 and not args.headline_only:
        # the other workloads on this GPU, each with its own clock record
        for key, fn in (("mixed512", sub_mixed512), ("batched512", sub_batched),
                        ("serving", sub_serving), ("amr", sub_amr), ("fill", sub_fill),
                        ("triad", sub_triad)):
            t = time.perf_counter()
            line[key] = fn(args)
            line[key]["wall_s"] = round(time.perf_counter() - t, 1)
            torch.cuda.empty_cache()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


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


def measure_fp64_peak(stream, device_index, target_ms=40.0):
    """The device's FP64 issue rate (G lane-ops/s): the library's FMA-chain probe, sized to
    run about target_ms, best of 5 timed launches (CUDA events on `stream`) after 3
    warm-ups, with the SM clock sampled meanwhile."""
    import torch
    from paper_2403_12179_gb300 import mg
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = 200
    a.record(stream)
    ops = mg.mg_calib_fp64(stream, iters)
    b.record(stream)
    stream.synchronize()
    iters = max(1, int(iters * target_ms / max(a.elapsed_time(b), 1e-3)))
    for _ in range(3):
        mg.mg_calib_fp64(stream, iters)
    stream.synchronize()
    clk = Clocks(device_index)
    best = 0.0
    for _ in range(5):
        a.record(stream)
        ops = mg.mg_calib_fp64(stream, iters)
        b.record(stream)
        stream.synchronize()
        best = max(best, ops / (a.elapsed_time(b) / 1e3) / 1e9)
    clocks = clk.stop()
    return {"value": round(best, 1), "unit": "G FP64 lane-ops/s",
            "how": f"mg_calib_fp64: {ops} DFMA lane-ops per launch (8 independent chains per "
                   "thread, 8 blocks of 256 threads per SM), best of 5 launches, CUDA events",
            "clocks": clocks}


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


def roofline(kt, wl_name, f64, fp64, in_solve_launches=0):
    peaks, src = load_peaks()
    cells = WORKLOADS[wl_name]["n"] ** 3
    fp64_peak = fp64["value"]                                          # G lane-ops/s, measured
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
                          "hbm_frac": round(8 * cells / kt["rbgs_half_f32"] / 1e9 / hbm, 4),
                          # the colours interleave within every 32-byte sector, so a half-sweep
                          # reads all of phi and rhs and writes back all of phi: 12 B/cell
                          "dram_min_frac": round(12 * cells / kt["rbgs_half_f32"] / 1e9 / hbm, 4)},
    }
    extra["note"] = ("the FP64 kernels (half-sweep, residual) are bound by GB300's FP64 issue "
                     "rate, measured by fp64_peak: at 100% of it a half-sweep moves about 42% of "
                     "the HBM copy peak, so the 70%-of-HBM target applies to the FP32 kernels "
                     "(rbgs_fused_f32, rbgs_half_f32) only")
    if f64:
        ach = half_ops / t / 1e9
        where = (f"average of {in_solve_launches} launches inside the timed solves (CUDA events "
                 "on the solve stream)" if in_solve_launches else "separate timing loop")
        return {"kernel": "k_rbgs_half<double> (one colour, finest level, neighbour boxes read directly)",
                "bound": "alu", "measured": where,
                "achieved": round(ach, 1), "peak": round(fp64_peak, 1),
                "unit": "G FP64 lane-ops/s", "frac": round(ach / fp64_peak, 4),
                "peak_source": "measured: mg_calib_fp64 (independent DFMA chains on every SM, "
                               "CUDA events; see fp64_peak)",
                "hbm": {"achieved_gbs": round(16 * cells / t / 1e9, 1), "peak": hbm,
                        "frac": round(16 * cells / t / 1e9 / hbm, 4),
                        "algorithmic_bytes_per_launch": 16 * cells},
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


def _events(n):
    import torch
    return ([torch.cuda.Event(enable_timing=True) for _ in range(n)],
            [torch.cuda.Event(enable_timing=True) for _ in range(n)])


def sub_mixed512(args, steps=5, warmup=2):
    """512^3 Dirichlet, 64 boxes of 128^3, Gaussian blobs: the mixed-precision solve (FP32
    inner V-cycle, FP64 outer residual / correction / bottom) against the plain FP64 solve of
    the same problem, both timed with CUDA events on the solve stream (L2 flushed before each
    solve, outside the events); the difference of the two answers against the bound two
    converged answers obey (P7); the FP32 smoother kernels at this size."""
    import numpy as np
    import torch
    from paper_2403_12179_gb300 import mg
    wl = WORKLOADS["mixed512"]
    n, box = wl["n"], wl["box"]
    cells = n ** 3
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    mg.mg_set_stream(ctx, stream)
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
    rhs_np = make_rhs(wl)
    rhs_max = float(np.abs(rhs_np).max())
    fr = mg.mg_fab_alloc(ctx, ba, 1, 1)
    d = torch.from_numpy(rhs_np).cuda()
    mg.mg_fab_copy_from_dense(ctx, fr, d.data_ptr(), False, stream)
    stream.synchronize()
    del d, rhs_np
    bc = mg.make_bc(wl["periodic"])
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    out = {"workload": wl["desc"], "cells": cells, "boxes": (n // box) ** 3}
    phis = {}
    for name, prec in (("mixed", mg.MG_PREC_MIXED), ("f64", mg.MG_PREC_F64)):
        fp = mg.mg_fab_alloc(ctx, ba, 1, 2)
        opt = mg.make_options(precision=prec)

        def solve():
            mg.mg_fab_set_val(ctx, fp, 0.0, True, stream)
            return mg.mg_solve(ctx, fr, fp, bc, 1e-10, opt)
        for _ in range(warmup):
            solve()
        k = steps if name == "mixed" else max(2, steps // 2)
        e0, e1 = _events(k)
        clk = Clocks(torch.cuda.current_device())
        res = []
        with torch.cuda.stream(stream):
            for i in range(k):
                flush.zero_()
                e0[i].record(stream)
                res.append(solve())
                e1[i].record(stream)
        stream.synchronize()
        clocks = clk.stop()
        ms = [e0[i].elapsed_time(e1[i]) for i in range(k)]
        assert all(r.status == 0 and r.rel_resid <= 1e-10 for r in res), f"{name} solve failed"
        out[name] = {"solves_per_s": round(1e3 / statistics.median(ms), 3),
                     "ms_per_solve": round(statistics.median(ms), 3), "steps": k,
                     "outer_iterations" if name == "mixed" else "vcycles": res[-1].vcycles,
                     "rel_resid": res[-1].rel_resid, "clocks": clocks}
        phis[name] = _fab_to_dense(ctx, fp, (n,) * 3, stream)
        mg.mg_fab_free(ctx, fp, stream)
    diff = float((phis["mixed"] - phis["f64"]).abs().max())
    del phis
    out["mixed_speedup_vs_f64"] = round(out["f64"]["ms_per_solve"] / out["mixed"]["ms_per_solve"], 3)
    out["max_abs_diff_vs_f64"] = diff
    out["p7_bound"] = 2 * 0.06 * 1e-10 * rhs_max
    # the FP32 smoother kernels on this level, back to back on the solve stream
    peaks, _ = load_peaks()
    hbm = peaks["hbm_gbs"]
    a32 = mg.mg_fab_alloc(ctx, ba, 1, 2, mg.MG_F32)
    b32 = mg.mg_fab_alloc(ctx, ba, 1, 2, mg.MG_F32)
    r32 = mg.mg_fab_alloc(ctx, ba, 1, 1, mg.MG_F32)
    mg.mg_fab_set_val(ctx, r32, 1.0, True, stream)
    mg.mg_fill_boundary(ctx, a32, bc, stream)
    mg.mg_fill_boundary(ctx, b32, bc, stream)
    pair = (a32, b32)
    h = 1.0 / n
    t_f = _time(stream, lambda k: mg.mg_smooth_fused(ctx, pair[k & 1], r32, pair[(k + 1) & 1], bc, h, stream), 20)
    t_h = _time(stream, lambda k: mg.mg_smooth(ctx, a32, r32, bc, h, (k & 1) | mg.MG_SMOOTH_DIRECT_READS, stream), 20)
    out["kernels"] = {
        "rbgs_fused_f32": {"launch_us": round(t_f * 1e6, 1), "gbs": round(12 * cells / t_f / 1e9, 1),
                           "hbm_frac": round(12 * cells / t_f / 1e9 / hbm, 4),
                           "algorithmic_bytes_per_cell": 12},
        "rbgs_half_f32": {"launch_us": round(t_h * 1e6, 1), "gbs": round(8 * cells / t_h / 1e9, 1),
                          "hbm_frac": round(8 * cells / t_h / 1e9 / hbm, 4),
                          "dram_min_frac": round(12 * cells / t_h / 1e9 / hbm, 4),
                          "algorithmic_bytes_per_cell": 8}}
    mg.mg_finalize(ctx)
    return out


def sub_batched(args, steps=3, warmup=1):
    """512 independent periodic problems (edges from {32,48,64,96,128}, 32^3 boxes): all
    packed into one launch per V-cycle stage, mixed and FP64; against the same problems solved
    one at a time with mg_solve (FP64).  Times are host wall times around the synchronous
    calls (inputs resident)."""
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
        stream.synchronize()
        t = time.perf_counter()
        res = mg.mg_solve_batch(ctx, fr, fp, bcs, 1e-10, mg.make_options(precision=prec))
        dt = time.perf_counter() - t
        assert all(r.status == 0 and r.rel_resid <= 1e-10 for r in res), "batched solve failed"
        return dt, res

    out, vcs, clocks = {}, {}, {}
    for name, prec in (("mixed", mg.MG_PREC_MIXED), ("f64", mg.MG_PREC_F64)):
        for _ in range(max(1, warmup)):
            batch(prec)
        clk = Clocks(torch.cuda.current_device())
        torch.cuda.nvtx.range_push(f"timed_{name}")  # (lets a profiler keep these runs only)
        runs = [batch(prec) for _ in range(steps)]
        torch.cuda.nvtx.range_pop()
        clocks[name] = clk.stop()
        out[name] = statistics.median(r[0] for r in runs)
        vcs[name] = [r.vcycles for r in runs[-1][1]]
    phis64 = [_fab_to_dense(ctx, f, sh, stream) for f, sh in zip(fp, shapes)]
    batch(mg.MG_PREC_MIXED)
    diff = 0.0
    for f, sh, p64 in zip(fp, shapes, phis64):
        pm = _fab_to_dense(ctx, f, sh, stream)
        dd = (pm - pm.mean()) - (p64 - p64.mean())
        diff = max(diff, float(dd.abs().max()))
    del phis64
    # one solve at a time, FP64, same problems (hierarchies and graphs built beforehand)
    for f in fp:
        mg.mg_fab_set_val(ctx, f, 0.0, True, stream)
    for a, b in zip(fr, fp):
        mg.mg_solve(ctx, a, b, bcs[0], 1e-10)
    for f in fp:
        mg.mg_fab_set_val(ctx, f, 0.0, True, stream)
    stream.synchronize()
    clk = Clocks(torch.cuda.current_device())
    t = time.perf_counter()
    for a, b in zip(fr, fp):
        r = mg.mg_solve(ctx, a, b, bcs[0], 1e-10)
        assert r.status == 0
    t_seq = time.perf_counter() - t
    clocks["f64_one_at_a_time"] = clk.stop()
    mg.mg_finalize(ctx)
    n = len(probs)
    line = {"problems": n, "cells": cells, "edges": "32/48/64/96/128 (seed 4)", "box": 32,
            "mixed_batched_solves_per_s": round(n / out["mixed"], 2),
            "f64_batched_solves_per_s": round(n / out["f64"], 2),
            "f64_one_at_a_time_solves_per_s": round(n / t_seq, 2),
            "mixed_batched_vs_f64_one_at_a_time": round(t_seq / out["mixed"], 3),
            "ms_per_batch": {"mixed": round(out["mixed"] * 1e3, 2), "f64": round(out["f64"] * 1e3, 2)},
            "cell_updates_per_s_mixed": round(sum(pb.n ** 3 * 4 * v for pb, v in
                                                  zip(probs, vcs["mixed"])) / out["mixed"], 1),
            "cell_updates": "finest level: 4 per cell per V-cycle (V(2,2)), each problem's own count",
            "max_abs_diff_mixed_vs_f64_mod_const": diff, "steps": steps, "clocks": clocks}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batched(probs, budget_s=6.0)
    return line


def run_batched(args):
    sub = sub_batched(args, steps=args.steps, warmup=args.warmup)
    n = sub["problems"]
    line = {"metric": f"solves/s, {n} batched periodic problems to 1e-10 (mixed precision)",
            "value": sub["mixed_batched_solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sub["ms_per_batch"]["mixed"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer",
            "data": "synthetic", "config": {"workload": "batched512"}}
    line.update(sub)
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


class HostInputs:
    """Draws the serving requests' right-hand sides into pinned host memory ahead of their
    arrival, in arrival order, on a pool of threads (NumPy releases the GIL while it draws),
    keeping at most `budget` bytes of drawn-but-unsubmitted data.  Buffers are recycled per
    size; `get(i)` waits for request i's rhs; `put(a)` returns a buffer to its pool."""

    def __init__(self, reqs, threads, budget, start=0, stop=None):
        import threading
        self.reqs = reqs
        self.stop_at = len(reqs) if stop is None else stop
        self.next = start
        self.budget = budget
        self.ahead = 0
        self.mu = threading.Lock()
        self.cv = threading.Condition(self.mu)
        self.ready = {}
        self.free = {}
        self.quit = False
        self.threads = [threading.Thread(target=self._work, daemon=True) for _ in range(threads)]
        for t in self.threads:
            t.start()

    def buffer(self, n):
        import torch
        with self.mu:
            lst = self.free.get(n)
            if lst:
                return lst.pop()
        return torch.empty((n, n, n), dtype=torch.float64, pin_memory=True)

    def put(self, a):
        with self.mu:
            self.free.setdefault(a.shape[0], []).append(a)

    def prewarm(self, n, count):
        """Adds `count` pinned (n, n, n) buffers to the pool, so that the replay itself does
        not wait for a pinned allocation (one of 128 MB takes tens of milliseconds)."""
        import torch
        bufs = [torch.empty((n, n, n), dtype=torch.float64, pin_memory=True) for _ in range(count)]
        with self.mu:
            self.free.setdefault(n, []).extend(bufs)

    def _work(self):
        while True:
            with self.cv:
                while not self.quit and self.next < self.stop_at and self.ahead >= self.budget:
                    self.cv.wait()
                if self.quit or self.next >= self.stop_at:
                    return
                i = self.next
                self.next += 1
                nb = self.reqs[i].n ** 3 * 8
                self.ahead += nb
            buf = self.buffer(self.reqs[i].n)
            self.reqs[i].rhs_into(buf.numpy())
            with self.cv:
                self.ready[i] = buf
                self.cv.notify_all()

    def get(self, i):
        with self.cv:
            while i not in self.ready:
                self.cv.wait()
            buf = self.ready.pop(i)
            self.ahead -= buf.numel() * 8
            self.cv.notify_all()
            return buf

    def wait_ahead(self, fraction=0.9):
        with self.cv:
            while self.ahead < fraction * self.budget and self.next < self.stop_at:
                self.cv.wait()

    def close(self):
        with self.cv:
            self.quit = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()


def sub_serving(args):
    """Serving: Poisson arrivals (200/s) of requests with edges {32,64,128,256}
    (p = .4/.3/.2/.1), periodic / Dirichlet, 32^3 or 64^3 boxes, rhs = PCG64 N(0,1) per request
    (inputs.serving_requests).  Each request's data lives in pinned host memory, drawn ahead
    of its arrival by a pool of host threads; at its arrival time it is submitted with
    mg_submit_host, so its latency (submit -> answer back in host memory) includes the copy
    in, the queueing, the shared V-cycle steps and the copy out, and the scheduler admits it
    only when the pool holds its whole hierarchy (fine level included).  Latencies are taken
    from the scheduled arrival.  Against it: one solve at a time in FP64 (mg_solve on fabs
    reused per shape, copy in / solve / copy out per request, service times measured
    back to back, latencies from the arrival times through a FIFO queue).  Capacity: a burst
    of the first requests queued at once (as many as fit in a pinned budget)."""
    import threading
    import numpy as np
    import torch
    from paper_2403_12179_gb300 import inputs, mg
    reqs = inputs.serving_requests(args.requests, seed=6)
    N = len(reqs)
    cores = os.cpu_count() or 4
    gen_threads = max(2, cores - 4)
    budget = 4 << 30
    opt = mg.make_options(precision=mg.MG_PREC_MIXED)
    shapes = sorted({(rq.n, rq.box, rq.periodic) for rq in reqs})
    bcs = {p: mg.make_bc((1, 1, 1) if p else (0, 0, 0)) for p in (True, False)}
    ctx = mg.mg_init(0)
    # warm-up (untimed): one request of every shape through the same path
    warm = []
    for k, (n, b, p) in enumerate(shapes):
        r = inputs.Request(0.0, n, p, b, 77 + k)
        ra = torch.from_numpy(r.rhs()).pin_memory()
        pa = torch.empty_like(ra).pin_memory()
        warm.append((ra, pa, mg.mg_submit_host(ctx, (0, 0, 0), (n - 1,) * 3, (b,) * 3, bcs[p],
                                               ra.data_ptr(), pa.data_ptr(), False, 1e-10, opt)))
    for _, _, t in warm:
        mg.mg_poll(ctx, t, -1)
    del warm
    stats0 = mg.mg_server_stats_get(ctx)
    gen = HostInputs(reqs, gen_threads, budget)
    gen.wait_ahead(0.9)
    # output buffers for the requests in flight, pinned before the replay starts
    for n, count in ((32, 48), (64, 48), (128, 32), (256, 16)):
        gen.prewarm(n, count)
    # a few sampled Dirichlet requests of edge <= 64 keep their answer for the oracle check
    sample = [i for i, rq in enumerate(reqs) if not rq.periodic and rq.n <= 64][:: max(1, N // 400)][:10]
    results = [None] * N
    tickets = [None] * N
    phis = [None] * N
    rhss = [None] * N
    lag = np.zeros(N)
    t_sub = np.zeros(N)
    kept = {}
    ready = threading.Semaphore(0)

    def poller():
        for i in range(N):
            ready.acquire()
            rc, r = mg.mg_poll(ctx, tickets[i], -1)
            results[i] = r
            if i in sample:
                kept[i] = phis[i].numpy().copy()
            gen.put(rhss[i])
            gen.put(phis[i])
            rhss[i] = phis[i] = None

    th = threading.Thread(target=poller)
    clk = Clocks(torch.cuda.current_device())
    import gc
    gc.disable()  # (no collector pauses in the submitting thread during the replay)
    th.start()
    t0 = time.perf_counter()
    for i, rq in enumerate(reqs):
        a = gen.get(i)
        ph = gen.buffer(rq.n)
        delay = t0 + rq.t_arrive - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        rhss[i], phis[i] = a, ph
        t_sub[i] = time.perf_counter()
        lag[i] = t_sub[i] - (t0 + rq.t_arrive)
        tickets[i] = mg.mg_submit_host(ctx, (0, 0, 0), (rq.n - 1,) * 3, (rq.box,) * 3,
                                       bcs[rq.periodic], a.data_ptr(), ph.data_ptr(), False,
                                       1e-10, opt)
        ready.release()
    th.join()
    gc.enable()
    clocks = clk.stop()
    gen.close()
    # latency from the scheduled arrival: the library's submit -> done, plus the submission lag
    lat = np.array([r.seconds for r in results]) + np.maximum(lag, 0.0)
    wall = max((t_sub[i] - t0) + results[i].seconds for i in range(N)) - reqs[0].t_arrive
    ok = all(r.status == 0 and r.rel_resid <= 1e-10 for r in results)
    stats = mg.mg_server_stats_get(ctx)
    stats = {k: (v - stats0[k] if k != "max_active" else v) for k, v in stats.items()}
    # capacity: a burst of the first M requests queued at once (rhs drawn beforehand; the
    # answer is written over the rhs buffer, which the scheduler has copied in by then)
    cap_budget = 6 << 30
    M, tot = 0, 0
    while M < N and tot + reqs[M].n ** 3 * 8 <= cap_budget:
        tot += reqs[M].n ** 3 * 8
        M += 1
    bufs = []
    for i in range(M):
        b = torch.empty((reqs[i].n,) * 3, dtype=torch.float64, pin_memory=True)
        reqs[i].rhs_into(b.numpy())
        bufs.append(b)
    t = time.perf_counter()
    tk = [mg.mg_submit_host(ctx, (0, 0, 0), (reqs[i].n - 1,) * 3, (reqs[i].box,) * 3,
                            bcs[reqs[i].periodic], bufs[i].data_ptr(), bufs[i].data_ptr(), False,
                            1e-10, opt) for i in range(M)]
    burst = [mg.mg_poll(ctx, x, -1)[1] for x in tk]
    cap = M / (time.perf_counter() - t)
    ok = ok and all(r.status == 0 and r.rel_resid <= 1e-10 for r in burst)
    del bufs
    mg.mg_finalize(ctx)
    # oracle check of the sampled answers (mixed oracle solve; P7 bound of two converged
    # answers on the Dirichlet unit cube)
    import oracle
    oracle.build()
    worst = 0.0
    for i in sample:
        rq = reqs[i]
        rhs = rq.rhs()
        dom = (rq.n - 1,) * 3
        o, st, _, _ = oracle.solve((0, 0, 0), dom, (0, 0, 0), oracle.chop((0, 0, 0), dom, (rq.box,) * 3),
                                   1.0 / rq.n, rhs, mixed=True)
        assert st == 0
        worst = max(worst, float(np.abs(kept[i] - o).max()) / (2 * 0.06 * 1e-10 * float(np.abs(rhs).max())))
    # one-at-a-time FP64 server on the same requests: fabs reused per shape, each request's
    # rhs copied in from pinned memory, solved, answer copied out
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    mg.mg_set_stream(ctx, stream)
    fabs = {}
    for (n, b, p) in shapes:
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (b,) * 3)
        fabs[(n, b, p)] = (mg.mg_fab_alloc(ctx, ba, 1, 1), mg.mg_fab_alloc(ctx, ba, 1, 2))
        r = inputs.Request(0.0, n, p, b, 77)
        ra = torch.from_numpy(r.rhs()).pin_memory()
        fr, fp = fabs[(n, b, p)]
        mg.mg_fab_copy_from_dense(ctx, fr, ra.data_ptr(), True, stream)
        mg.mg_solve(ctx, fr, fp, bcs[p], 1e-10)
    gen = HostInputs(reqs, gen_threads, budget)
    svc = np.zeros(N)
    clk = Clocks(torch.cuda.current_device())
    for i, rq in enumerate(reqs):
        a = gen.get(i)
        ph = gen.buffer(rq.n)
        fr, fp = fabs[(rq.n, rq.box, rq.periodic)]
        t = time.perf_counter()
        mg.mg_fab_copy_from_dense(ctx, fr, a.data_ptr(), True, stream)
        mg.mg_fab_set_val(ctx, fp, 0.0, True, stream)
        r = mg.mg_solve(ctx, fr, fp, bcs[rq.periodic], 1e-10)
        mg.mg_fab_copy_to_dense(ctx, fp, ph.data_ptr(), True, stream)
        stream.synchronize()
        svc[i] = time.perf_counter() - t
        ok = ok and r.status == 0
        gen.put(a)
        gen.put(ph)
    clocks64 = clk.stop()
    gen.close()
    mg.mg_finalize(ctx)
    end, lat64 = 0.0, []
    for rq, sv in zip(reqs, svc):
        start = max(rq.t_arrive, end)
        end = start + sv
        lat64.append((end - rq.t_arrive) * 1e3)
    lat64 = np.array(lat64)
    wall64 = end - reqs[0].t_arrive
    return {"requests": N, "rate_per_s": 200, "edges": "32/64/128/256 p=.4/.3/.2/.1",
            "bc": "periodic/Dirichlet 50/50", "box": "32 or 64", "precision": "mixed",
            "data": "PCG64 N(0,1) per request (inputs.serving_requests), drawn into pinned "
                    "host memory ahead of arrival; submitted with mg_submit_host",
            "solves_per_s": round(N / wall, 2),
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)) * 1e3, 2),
                           "p99": round(float(np.percentile(lat, 99)) * 1e3, 2),
                           "includes": "copy in from host, queueing, V-cycle steps, copy out; "
                                       "from the scheduled arrival"},
            "submit_lag_ms": {"p50": round(float(np.percentile(lag, 50)) * 1e3, 3),
                              "max": round(float(lag.max()) * 1e3, 3)},
            "all_converged_to_1e-10": bool(ok), "scheduler": stats,
            "capacity_solves_per_s": round(cap, 2), "capacity_burst_requests": M,
            "oracle_check": {"requests": len(sample), "kind": "mixed oracle solve, Dirichlet, edge <= 64",
                             "worst_diff_over_p7_bound": round(worst, 6), "pass": bool(worst <= 1.0)},
            "f64_one_at_a_time": {"solves_per_s": round(N / wall64, 2),
                                  "capacity_solves_per_s": round(1.0 / float(np.mean(svc)), 2),
                                  "latency_ms": {"p50": round(float(np.percentile(lat64, 50)), 2),
                                                 "p99": round(float(np.percentile(lat64, 99)), 2)},
                                  "mean_service_ms": round(float(np.mean(svc)) * 1e3, 3),
                                  "clocks": clocks64},
            "clocks": clocks}


def run_serving(args):
    sub = sub_serving(args)
    line = {"metric": f"served solves/s and latency, {sub['requests']} Poisson-arrival requests at 200/s",
            "value": sub["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": "serving"}}
    line.update(sub)
    print(json.dumps(line), flush=True)


def sub_fill(args, reps=200):
    """FillBoundary microbench: 256^3 periodic, 64 boxes of 64^3, 4 FP64 components, 2 ghost
    layers; one fill kernel per call, against one launch per copy tag."""
    import torch
    from paper_2403_12179_gb300 import inputs, mg
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), (255,) * 3, (64,) * 3)
    fab = mg.mg_fab_alloc(ctx, ba, 4, 2)
    d = torch.from_numpy(inputs.fill_microbench(256, seed=3)).cuda()
    mg.mg_fab_copy_from_dense(ctx, fab, d.data_ptr(), False, stream)
    stream.synchronize()
    del d
    bc = mg.make_bc((1, 1, 1))
    for _ in range(3):
        mg.mg_fill_boundary(ctx, fab, bc, stream)
    clk = Clocks(torch.cuda.current_device())
    t = _time(stream, lambda k: mg.mg_fill_boundary(ctx, fab, bc, stream), reps)
    t_unfused = _time(stream, lambda k: mg.mg_fill_boundary_unfused(ctx, fab, bc, stream), 5)
    clocks = clk.stop()
    ntags = len(mg.mg_copy_tags(ctx, ba, bc, 2))
    mg.mg_finalize(ctx)
    ghost = 64 * (68 ** 3 - 64 ** 3)
    nbytes = ghost * 4 * 8 * 2
    peaks, src = load_peaks()
    ach = nbytes / t / 1e9
    return {"us_per_fill": round(t * 1e6, 2), "ghost_cells": ghost, "bytes_per_fill": nbytes,
            "unfused": {"us_per_fill": round(t_unfused * 1e6, 2), "launches_per_fill": ntags,
                        "fused_speedup": round(t_unfused / t, 2)},
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                         "peak_source": src, "traffic": roofline_traffic("copy_tags_f64", "fill")},
            "clocks": clocks}


def run_fill(args):
    sub = sub_fill(args, reps=args.steps * 10)
    line = {"metric": "FillBoundary time per fill (256^3, 64 boxes, 4 comps, 2 ghosts, periodic)",
            "value": sub["us_per_fill"], "unit": "us", "n_gpus": 1, "steps": args.steps * 10,
            "warmup": 3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": "fill"}}
    line.update(sub)
    print(json.dumps(line), flush=True)


def sub_amr(args, n0=128, steps=5, warmup=2):
    """Two-level AMR composite solve: a 128^3 Dirichlet coarse level (32^3 boxes) with the
    middle half of the domain refined by 2 (a 128^3 fine region, 32^3 boxes); lap u = f with
    u = prod sin(pi x_d) sampled at both levels' cell centres; solved to 1e-10 with
    mg_amr2_solve (CUDA events on the solve stream).  Reported beside it: the error against u
    (second order: the same run at half the resolution gives about 4x the error) and the
    oracle's composite iteration on the host cores at 16^3 (its scheme step by step)."""
    import numpy as np
    import torch
    from paper_2403_12179_gb300 import inputs, mg
    out = {"workload": "coarse 128^3 Dirichlet (32^3 boxes), region [32, 96)^3 refined by 2 "
                       "(128^3 fine cells, 32^3 boxes), u = prod sin(pi x_d), tol 1e-10"}
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    mg.mg_set_stream(ctx, stream)

    errs = {}
    for n in (n0 // 2, n0):
        f0, f1, u0, u1 = inputs.amr_sine(n, (n // 4,) * 3, (3 * n // 4,) * 3)
        covered = np.zeros((n,) * 3, bool)
        covered[n // 4:3 * n // 4, n // 4:3 * n // 4, n // 4:3 * n // 4] = True
        ba0 = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (32,) * 3)
        ba1 = mg.mg_box_array_create(ctx, (n // 2,) * 3, (3 * n // 2 - 1,) * 3, (32,) * 3)
        fr0, fr1 = _dense_to_fab(ctx, ba0, torch.from_numpy(f0).cuda(), 0, stream), \
            _dense_to_fab(ctx, ba1, torch.from_numpy(f1).cuda(), 0, stream)
        fp0, fp1 = mg.mg_fab_alloc(ctx, ba0, 1, 1), mg.mg_fab_alloc(ctx, ba1, 1, 1)
        bc = mg.make_bc((0, 0, 0))

        def solve():
            mg.mg_fab_set_val(ctx, fp0, 0.0, True, stream)
            mg.mg_fab_set_val(ctx, fp1, 0.0, True, stream)
            return mg.mg_amr2_solve(ctx, fr0, fp0, fr1, fp1, bc, 1e-10)
        for _ in range(warmup):
            solve()
        if n == n0:
            e0, e1 = _events(steps)
            clk = Clocks(torch.cuda.current_device())
            res = []
            torch.cuda.nvtx.range_push("timed_amr")  # (lets a profiler keep these solves only)
            with torch.cuda.stream(stream):
                for i in range(steps):
                    e0[i].record(stream)
                    res.append(solve())
                    e1[i].record(stream)
            torch.cuda.nvtx.range_pop()
            stream.synchronize()
            clocks = clk.stop()
            ms = [e0[i].elapsed_time(e1[i]) for i in range(steps)]
            assert all(r.status == 0 and r.rel_resid <= 1e-10 for r in res)
            out.update({"solves_per_s": round(1e3 / statistics.median(ms), 3),
                        "ms_per_solve": round(statistics.median(ms), 3), "steps": steps,
                        "iterations": res[-1].vcycles, "rel_resid": res[-1].rel_resid,
                        "unknowns": n ** 3 - (n // 2) ** 3 + n ** 3, "clocks": clocks})
        else:
            r = solve()
            assert r.status == 0
        a0 = _fab_to_dense(ctx, fp0, u0.shape, stream).cpu().numpy()
        a1 = _fab_to_dense(ctx, fp1, u1.shape, stream).cpu().numpy()
        errs[n] = max(float(np.abs(a1 - u1).max()), float(np.abs((a0 - u0)[~covered]).max()))
        for f in (fr0, fr1, fp0, fp1):
            mg.mg_fab_free(ctx, f, stream)
    mg.mg_finalize(ctx)
    out["error_vs_u"] = {str(k): v for k, v in errs.items()}
    out["error_ratio_h_over_h2"] = round(errs[n0 // 2] / errs[n0], 3)
    if not args.no_cpu_baseline:
        import oracle
        from oracle import amr
        oracle.build()
        g = amr.Geometry((16,) * 3, (4,) * 3, (12,) * 3)
        f0, f1, _, _ = inputs.amr_sine(16, (4,) * 3, (12,) * 3)
        t = time.perf_counter()
        _, _, hist = amr.iterate(f0, f1, g, 9)
        el = time.perf_counter() - t
        out["cpu_baseline"] = {"value": round(1.0 / el, 4), "unit": "solves/s", "kind": "oracle",
                               "cores": int(os.environ["OMP_NUM_THREADS"]),
                               "sample": f"the oracle's composite iteration (numpy + the C++ "
                                         f"single-level oracle), 16^3 coarse with [4, 12)^3 "
                                         f"refined, 9 iterations to {hist[-1]:.1e}, {el:.2f} s"}
    return out


def run_amr(args):
    sub = sub_amr(args)
    line = {"metric": "two-level AMR composite solves/s to 1e-10 (128^3 coarse, middle half refined)",
            "value": sub["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": sub["steps"],
            "warmup": 2, "ms_per_step": sub["ms_per_solve"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "amr"}}
    line.update(sub)
    print(json.dumps(line), flush=True)


# The paper's own triad timings (Sec. 3.2, one MI250X GCD), for context only
PAPER_TRIAD = {"512x32^3": {"per_box_s": 1.16e-3, "fused_s": 3.67e-4},
               "1x256^3": {"per_box_s": 3.28e-4, "fused_s": 3.35e-4}}


def sub_triad(args, reps=50):
    """STREAM triad a = b + s c (FP64) over a 256^3 domain as 512 boxes of 32^3 and as one
    box of 256^3 (the paper's Sec. 3.2 cases): one launch per box against one launch over
    all boxes, CUDA events on the launching stream; 24 B per cell (fields > L2)."""
    import torch
    from paper_2403_12179_gb300 import mg
    peaks, src = load_peaks()
    hbm = peaks["hbm_gbs"]
    ctx = mg.mg_init(0)
    stream = torch.cuda.Stream()
    out = {}
    clk = Clocks(torch.cuda.current_device())
    for name, box in (("512x32^3", 32), ("1x256^3", 256)):
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (255,) * 3, (box,) * 3)
        a, b, c = (mg.mg_fab_alloc(ctx, ba, 1, 1) for _ in range(3))
        mg.mg_fab_set_val(ctx, b, 1.0, False, stream)
        mg.mg_fab_set_val(ctx, c, 2.0, False, stream)
        cells = 256 ** 3
        res = {}
        for form, per_box in (("fused", False), ("per_box", True)):
            for _ in range(3):
                mg.mg_triad(ctx, a, b, c, 0.5, per_box, stream)
            t = _time(stream, lambda k: mg.mg_triad(ctx, a, b, c, 0.5, per_box, stream),
                      reps if not per_box else max(5, reps // 5))
            res[form] = {"us": round(t * 1e6, 2), "gbs": round(24 * cells / t / 1e9, 1),
                         "hbm_frac": round(24 * cells / t / 1e9 / hbm, 4)}
        res["launches_per_box_form"] = (256 // box) ** 3
        res["fused_speedup"] = round(res["per_box"]["us"] / res["fused"]["us"], 3)
        res["paper_mi250x_context"] = PAPER_TRIAD[name]
        out[name] = res
        for f in (a, b, c):
            mg.mg_fab_free(ctx, f, stream)
    out["clocks"] = clk.stop()
    out["peak_source"] = src
    mg.mg_finalize(ctx)
    return out


def run_triad(args):
    sub = sub_triad(args)
    line = {"metric": "STREAM triad over 512 boxes of 32^3: one launch vs one launch per box",
            "value": sub["512x32^3"]["fused"]["us"], "unit": "us", "n_gpus": 1, "steps": 50,
            "warmup": 3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": "triad"}}
    line.update(sub)
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
                    choices=sorted(WORKLOADS) + ["batched512", "serving", "fill", "triad", "amr"])
    ap.add_argument("--headline-only", action="store_true",
                    help="the dirichlet256 line without the other workloads' sub-objects")
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
    elif args.workload == "triad":
        run_triad(args)
    elif args.workload == "amr":
        run_amr(args)
    elif args.kernels_only:
        run_kernels_only(args, args.workload)
    elif args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
