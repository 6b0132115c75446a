#!/usr/bin/env python
"""Benchmark of the GB300 multigrid Poisson path; prints ONE JSON line on rank 0.

Default workload (dirichlet256): 256^3 homogeneous-Dirichlet FP64 Poisson problem split into
64 boxes of 64^3, rhs = seeded N(0,1) smoothed by one damped-Jacobi pass, V(2,2) red-black
Gauss-Seidel cycles to ||rhs - A phi||_inf <= 1e-10 ||rhs||_inf.  One step = one complete
solve (phi reset to 0, then mg_solve) with rhs already resident in HBM.  `value` is solves/s
over all ranks (each rank solves its own replica: the solve does not shard).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload dirichlet256|periodic64|mixed512]

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
                                       "--format=csv,noheader,nounits", "-lms", "200"],
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

def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
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
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- our arm --------------------------------------------------------------------------------

def roofline_traffic(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (the summary records the source hash); else None."""
    import hashlib
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    src = os.path.join(ROOT, "paper_2403_12179_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        if f.endswith((".cu", ".hpp")):
            h.update(open(os.path.join(src, f), "rb").read())
    cur = h.hexdigest()[:16]
    traffic = src_hash = None
    for line in open(p):
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":")[1])
        if line.startswith("source_hash:"):
            src_hash = line.split(":")[1].strip()
    return traffic if src_hash == cur else None


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

    # ---- timed region: K solves, inputs resident, events on the solve stream
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    l0 = mg_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    results = []
    for k in range(args.steps):
        results.append(step())
        evs[k + 1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    launches = mg_launches() - l0
    clocks = clk.stop()
    barrier(world)
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = max_over_ranks(total_ms, world)
    value = world * args.steps / (total_ms / 1e3)
    vcycles = results[-1].vcycles
    assert all(r.status == 0 and r.rel_resid <= 1e-10 for r in results)

    # ---- dominant kernels on the fine level, timed alone on the solve stream
    kt = kernel_timings(ctx, stream, ba, fp, fr, bc, h, cells, box)
    roof = roofline(kt, wl_name, prec == mg.MG_PREC_F64, clocks)

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
                   "l2": "inputs larger than L2: two FP64 fields of "
                         f"{round(cells * 8 / 2**20)} MiB each are streamed every sweep"},
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
    out["rbgs_half_f64"] = _time(stream, lambda k: mg.mg_smooth(ctx, fp, fr, bc, h, k & 1, stream), reps)
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


def roofline(kt, wl_name, f64, clocks):
    peaks, src = load_peaks()
    cells = WORKLOADS[wl_name]["n"] ** 3
    sm_mhz = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = FP64_LANES_PER_SM_CLK * N_SM * sm_mhz * 1e6 / 1e9      # G lane-ops/s
    hbm = peaks["hbm_gbs"]
    t = kt["rbgs_half_f64"]
    half_ops = FP64_INST_PER_UPDATE * cells / 2
    fused_bytes = 24 * cells          # read phi, read rhs, write phi: one full sweep
    extra = {
        "rbgs_half_f64": {"launch_us": round(t * 1e6, 2),
                          "hbm_frac": round(16 * cells / t / 1e9 / hbm, 4),
                          "fp64_frac": round(half_ops / t / 1e9 / fp64_peak, 4)},
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
        return {"kernel": "k_rbgs_half<double> (one colour, fine level)", "bound": "alu",
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


def cpu_baseline(wl_name, vcycles):
    t0, t1, tv = oracle_sample(wl_name)
    est = t0 + vcycles * tv
    return {"value": round(1.0 / est, 6), "unit": "solves/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{wl_name}: oracle run with 0 and with 1 V-cycle ({t0:.2f} s, {t1:.2f} s); "
                      f"solve time extrapolated to the {vcycles} V-cycles of the solve "
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dirichlet256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time only the fine-level kernels (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.kernels_only:
        run_kernels_only(args, args.workload)
    elif args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
