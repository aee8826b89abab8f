#!/usr/bin/env python3
"""Benchmark: cell-steps/s of the lid-driven-cavity fractional step on GB300.

Workload (default): the FP64 cavity of Sec. 3 / 3.1 of arXiv 2504.03697 at
64^3 cells, lid 1.0, nu 1e-3, dt 1e-2, pressure by unpreconditioned CG to
rtol 1e-8 (true FP64 residual), velocity initialised to the seeded
uniform[-1e-3, 1e-3] perturbation (seed 2 + rank).  One bench "step" is one
time step: applyForces, advection, implicit diffusion (3 CG solves),
divergence, pressure CG, correction.  Inputs are synthetic and resident in
HBM when the timed region starts; L2 is flushed (256 MiB write) between
timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: one independent cavity per rank (weak scaling,
no data-path collective); the timed region is bracketed by a barrier and a
synchronize and its maximum over ranks is reported.  ``--impl reference``
times the FP64 CPU oracle on the host cores instead (rank 0 only).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "cavity64": dict(n=64, nu=1e-3, dt=1e-2, lid_u=1.0, seed=2, amp=1e-3,
                     desc="lid-driven cavity 64^3 cells, FP64, lid 1.0, nu 1e-3, dt 1e-2, "
                          "pressure CG to rtol 1e-8, seeded 1e-3 perturbation"),
    "cavity384": dict(n=384, nu=1e-3, dt=1e-2, lid_u=1.0, seed=5, amp=1e-3,
                      desc="lid-driven cavity 384^3 cells, FP64, lid 1.0, nu 1e-3, dt 1e-2, "
                           "pressure solve to rtol 1e-8, seeded 1e-3 perturbation"),
    "cavity16": dict(n=16, nu=1e-2, dt=1e-2, lid_u=1.0, seed=1, amp=1e-3,
                     desc="lid-driven cavity 16^3 cells, FP64, lid 1.0, nu 1e-2, dt 1e-2, "
                          "pressure CG to rtol 1e-8, seeded 1e-3 perturbation"),
}

# Algorithmic work of one pressure-CG iteration per cell (FP64, matrix-free):
# p = z + beta p (2), q = A p (5 adds + 6 x_c - sum: 7), p.q (2), x += a p (2),
# r -= a q (2), r.r (2)  -> 17 flops; bytes: read r, p_old, write p, q (32) +
# read x, p, r, q, write x, r (48) -> 80 B.  Setup + true residual + gauge per
# solve: ~14 flops and ~72 B per cell.
CG_FLOPS_PER_CELL_ITER = 17
CG_BYTES_PER_CELL_ITER = 80
CG_FLOPS_PER_CELL_SOLVE = 14
CG_BYTES_PER_CELL_SOLVE = 72
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of
# cg1_fp64_kernel<8> on the 64^3 cavity in its automatic shape (128 blocks,
# tile depth 8), from one ncu capture of the pressure solve of the first timed
# step: the 26 MB working set is L2-resident, so DRAM sees almost nothing
CG1_CAVITY64_DRAM_BYTES = 2342400 + 84992
CG1_CAVITY64_SHAPE = {"blocks": 128, "tile_depth": 8, "register_path": True}
IR_BYTES_PER_CELL_ITER = 40
IR_GRAPH_BYTES_PER_CELL_ITER = 32


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cavity64")
    ap.add_argument("--solver", default="cg")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--poisson", type=int, default=0,
                    help="standalone Neumann-Poisson solves on an N^3 grid instead of the cavity "
                         "(one bench step = one solve of a seeded Gaussian right-hand side)")
    ap.add_argument("--max-iters", type=int, default=0, help="CG iteration cap per solve (0: 20 N)")
    ap.add_argument("--no-precision-study", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="benchmark N batched uneven cavities (edges from {32,48,64,96}) instead of one cavity")
    ap.add_argument("--no-batch-study", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the automatic solver shape")
    ap.add_argument("--cg-variant", choices=["single", "two"], default="single",
                    help="FP64 CG form: one grid reduction per iteration (default) or the textbook two")
    ap.add_argument("--spmv", type=int, default=0,
                    help="time the pressure operator on an N^3 grid: matrix-free stencil vs the assembled CSR matrix")
    ap.add_argument("--ir-form", choices=["tuned", "auto", "persistent", "graph"], default="tuned",
                    help="execution of the mixed-precision solve in --poisson mode (default: the autotuner's choice)")
    ap.add_argument("--blas", type=int, default=0,
                    help="time the stand-alone building blocks on an N^3 grid: FP32 operator, FP64 / FP32 CG update")
    ap.add_argument("--concurrent-diffusion", choices=["on", "off"], default="on",
                    help="run the u, v, w diffusion solves of a step at once (grids up to 2^21 cells; "
                         "the library's default there)")
    ap.add_argument("--advect-order", type=int, default=1, choices=[1, 2],
                    help="backtrace of the cavity workload: 1 explicit Euler (default), 2 explicit midpoint")
    ap.add_argument("--unet", type=int, default=0,
                    help="time the learned preconditioner's U-Net application on an N^3 grid (N % 4 == 0) "
                         "instead of the cavity")
    ap.add_argument("--unet-weights", default="", help="FP32 parameter file for --unet (default: seeded init)")
    ap.add_argument("--unet-conv-mode", choices=["registers", "bulk", "two_stage"], default="bulk",
                    help="staging of the tiled convolutions (comparison)")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--max-seconds", type=float, default=150.0, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed plumbing (measurement only: barrier + max of the timed region)
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init_dist(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def reduce_max(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(cells_per_rank, steps, world, max_seconds):
    """Whole-job throughput: all ranks' cell-steps over the slowest rank's time."""
    return cells_per_rank * steps * world / max_seconds


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def physical_gpu(local):
    """nvidia-smi index (or UUID) of this process's CUDA device."""
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    if cvd:
        parts = [p.strip() for p in cvd.split(",") if p.strip()]
        if local < len(parts):
            return parts[local]
    return local


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm): runs in a child process
# ---------------------------------------------------------------------------
def oracle_sample_main(args):
    """Child process: time the FP64 oracle on the workload for a bounded
    number of steps; print one JSON object."""
    from oracle import fractional_step as fs
    from oracle.mac import Cavity
    from paper_2504_03697_gb300.synthetic import cavity_perturbation

    wl = WORKLOADS[args.workload]
    n = wl["n"]
    cav = Cavity(n, n, n, dt=wl["dt"], nu=wl["nu"], lid_u=wl["lid_u"])
    st = fs.initial_state(cav, cavity_perturbation(n, n, n, wl["seed"], wl["amp"]))
    for _ in range(args.warmup):
        st, _ = fs.step(cav, st)
    t0 = time.perf_counter()
    done = 0
    per_step = []
    while done < args.steps:
        a = time.perf_counter()
        st, _ = fs.step(cav, st)
        per_step.append(time.perf_counter() - a)
        done += 1
        if time.perf_counter() - t0 > args.max_seconds:
            break
    el = time.perf_counter() - t0
    print(json.dumps({"steps": done, "seconds": el, "cells": n ** 3, "per_step_s": per_step}))


def run_oracle_child(workload, steps, warmup, max_seconds):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "LOCAL_WORLD_SIZE", "GROUP_RANK", "ROLE_RANK"):
        env.pop(k, None)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", workload,
           "--steps", str(steps), "--warmup", str(warmup), "--max-seconds", str(max_seconds)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------------------
# reference arm
# ---------------------------------------------------------------------------
def main_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    res = run_oracle_child(args.workload, args.steps, min(args.warmup, 1), args.max_seconds)
    value = res["cells"] * res["steps"] / res["seconds"]
    sample = (f"{res['steps']} time steps of the {wl['n']}^3 cavity (of {args.steps} requested; capped at "
              f"{args.max_seconds:.0f} s), FP64 numpy/scipy oracle, single thread, after "
              f"{min(args.warmup, 1)} warm-up step")
    line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": res["steps"], "warmup": min(args.warmup, 1),
            "ms_per_step": 1e3 * res["seconds"] / max(res["steps"], 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": wl["n"], "parallelism": "host oracle, rank 0 only"},
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model(), "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = init_dist("nccl")

    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd
    from paper_2504_03697_gb300.synthetic import cavity_perturbation

    wl = WORKLOADS[args.workload]
    n = wl["n"]
    cells = n ** 3
    prm = cfd.make_params(n, n, n, dt=wl["dt"], nu=wl["nu"], lid_u=wl["lid_u"], solver=args.solver,
                          advect_order=args.advect_order)
    stream = torch.cuda.current_stream(device)
    cav = cfd.Cavity(prm, device=device)
    init = cavity_perturbation(n, n, n, wl["seed"] + rank, wl["amp"])
    for name, f in zip("uvw", init):
        cav.set_field(name, f)
    cav.set_cg_variant(args.cg_variant)
    if args.concurrent_diffusion == "off":
        cav.set_concurrent_diffusion(False)
    # solver shape for this grid (blocks per SM x tile depth), picked by
    # timing fixed-length solves; outside the timed region, state untouched
    tune = None if args.no_autotune else cav.autotune(iters=50)

    # warm-up
    if args.warmup > 0:
        rc, _ = cav.step(args.warmup, stats=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    cav.phase_times()  # reset
    cav.enable_timing(True)
    launches0 = cav.launch_count()
    sampler = ClockSampler(physical_gpu(local)) if rank == 0 else None
    barrier(dist, device)
    torch.cuda.synchronize(device)
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()  # L2 flush, outside the timed events
        starts[s].record(stream)
        cav.step(1, stats=False)
        ends[s].record(stream)
    torch.cuda.synchronize(device)
    wall = time.perf_counter() - wall0
    barrier(dist, device)
    clocks = sampler.stop() if sampler else None
    launches = cav.launch_count() - launches0
    cav.enable_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    t_local = sum(step_ms) / 1e3
    t_max = reduce_max(dist, t_local, device)
    phases = cav.phase_times()
    rc, stats = cav.recent_stats(args.steps)
    iters = [s["iters"] for s in stats]
    worst_resid = max(s["rel_resid"] for s in stats)
    ok = rc == cfd.CFD_OK and worst_resid <= 1e-8 * 1.0000001

    value = aggregate(cells, args.steps, world, t_max)
    pcg_ms, pcg_calls = phases["pcg"]
    pcg_avg_s = pcg_ms / max(pcg_calls, 1) / 1e3
    mean_iters = float(np.mean(iters))
    flops_per_launch = cells * (CG_FLOPS_PER_CELL_ITER * mean_iters + CG_FLOPS_PER_CELL_SOLVE)
    bytes_per_launch = cells * (CG_BYTES_PER_CELL_ITER * mean_iters + CG_BYTES_PER_CELL_SOLVE)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp64_peak_tflops = 1.20  # FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (measured with DFMA chains)
    achieved_tflops = flops_per_launch / pcg_avg_s / 1e12
    variant = tune["cg_variant"] if tune is not None else (0 if args.cg_variant == "single" else 1)
    # the launch the captured counters belong to: 128 blocks, register path, tile depth 8
    pressure_shape = cav.solver_shape(0)
    roofline = {"bound": "alu",
                "kernel": ("cg1_fp64_kernel (pressure CG, single reduction per iteration, persistent)" if variant == 0
                           else "cg_fp64_kernel (pressure CG, two reductions per iteration, persistent)"),
                "achieved": achieved_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / fp64_peak_tflops,
                "traffic": (CG1_CAVITY64_DRAM_BYTES if (args.workload == "cavity64" and variant == 0
                                                         and args.solver == "cg"
                                                         and pressure_shape == CG1_CAVITY64_SHAPE) else None),
                "launch_shape": pressure_shape,
                "peak_source": "FP64 FMA rate from the recipe's unit counts and clocks (1.2-1.25 TFLOP/s)",
                "hbm_achieved_gbs": bytes_per_launch / pcg_avg_s / 1e9,
                "hbm_peak_gbs": hbm_peak, "hbm_frac_of_measured": bytes_per_launch / pcg_avg_s / 1e9 / hbm_peak,
                "launch_ms": pcg_avg_s * 1e3, "flops_per_launch": flops_per_launch,
                "bytes_per_launch": bytes_per_launch}
    if args.solver == "ir":
        # bytes per cell and FP32 iteration: persistent form 40 (direction:
        # read r32, p_old, write p, q; update: read p, q, x32, r32, write x32,
        # r32); graph form 32 (q is formed again in the update, never stored);
        # the FP64 refinements add a few residual passes, left out of the count
        form = tune["ir_form"] if tune is not None else 0
        graph = form == 2 or (form == 0 and n % 4 == 0 and cells >= 1 << 21)
        ir_bytes = cells * (IR_GRAPH_BYTES_PER_CELL_ITER if graph else IR_BYTES_PER_CELL_ITER) * mean_iters
        ir_gbs = ir_bytes / pcg_avg_s / 1e9
        roofline = {"bound": "hbm",
                    "kernel": ("g_dir + g_upd (FP32 CG iteration, graph form)" if graph
                               else "ir_kernel (FP32 CG + FP64 refinement, persistent)"),
                    "achieved": ir_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": ir_gbs / hbm_peak,
                    "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                    "launch_ms": pcg_avg_s * 1e3, "bytes_per_launch": ir_bytes}
    phase_ms_per_step = {k: v[0] / max(args.steps, 1) for k, v in phases.items()}

    # end-to-end through the C-ABI with host buffers (state round-trips per step)
    e2e = None
    if args.e2e_steps > 0:
        host = {f: torch.empty(cav.shape(f), dtype=torch.float64).pin_memory() for f in "uvwp"}
        for f in "uvwp":
            cav.read_field(f, out=host[f])
        bytes_io = sum(host[f].numel() * 8 for f in "uvwp")
        barrier(dist, device)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for f in "uvwp":
                cav.lib.cfd_set_field(cav.h, cfd.FIELD[f], host[f].data_ptr(), 0)
            cav.step(1, stats=False)
            for f in "uvwp":
                cav.read_field(f, out=host[f])
        torch.cuda.synchronize(device)
        te = reduce_max(dist, time.perf_counter() - t0, device)
        e2e = {"value": aggregate(cells, args.e2e_steps, world, te), "unit": "cell-steps/s",
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": args.e2e_steps,
               "how": "per step: cfd_set_field(u,v,w,p) from pinned host, cfd_step(1), cfd_read_field(u,v,w,p) "
                      "to pinned host; wall clock"}

    # precision study on the standalone 256^3 Neumann-Poisson system: FP64 CG
    # vs FP32 CG with FP64 refinement, both to a true FP64 rtol of 1e-8
    precision = None
    if rank == 0 and world == 1 and not args.no_precision_study:
        cav.close()
        del cav
        torch.cuda.empty_cache()
        study = {}
        for solver in ("cg", "ir"):
            res = time_solves(cfd, 256, solver, [0, 1], 1, 0, device)
            study[solver] = {"ms_per_solve": [round(r["ms"], 3) for r in res], "iters": [r["iters"] for r in res],
                             "refinements": [r["refinements"] for r in res],
                             "rel_resid": [r["rel_resid"] for r in res]}
        cg_ms = statistics.mean(study["cg"]["ms_per_solve"])
        ir_ms = statistics.mean(study["ir"]["ms_per_solve"])
        precision = {"workload": "Neumann-Poisson 256^3, N(0,1) right-hand sides seeds 0-1, rtol 1e-8 (true FP64)",
                     "fp64_cg": study["cg"], "fp32_cg_fp64_refined": study["ir"],
                     "speedup_ir_over_fp64_cg": cg_ms / ir_ms}

    # batched uneven cavities: FP64 CG vs mixed precision, graph-replayed
    batch = None
    if rank == 0 and world == 1 and not args.no_batch_study:
        batch = {s: time_batch(cfd, 64, s, 3, 1, device) for s in ("cg", "ir")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = run_oracle_child(args.workload, 10 ** 6, 0, args.cpu_seconds)
        cpu = {"value": res["cells"] * res["steps"] / res["seconds"], "unit": "cell-steps/s", "cores": 1,
               "kind": "oracle",
               "sample": f"first {res['steps']} time steps of the same {n}^3 cavity ({res['seconds']:.1f} s), "
                         f"FP64 numpy/scipy oracle, single thread",
               "cpu": cpu_model(), "host_cores": os.cpu_count()}

    if rank == 0:
        line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": wl["desc"], "n": n, "cells": cells, "solver": args.solver,
                           "steps_per_rank": args.steps, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                           "solver_shape": tune if tune is not None else "automatic",
                           "cg_variant": args.cg_variant, "advect_order": args.advect_order,
                           "concurrent_diffusion": args.concurrent_diffusion},
                "solve": {"pcg_iters_mean": mean_iters, "pcg_iters_min": min(iters), "pcg_iters_max": max(iters),
                          "time_to_rtol_ms_mean": pcg_avg_s * 1e3, "rel_resid_max": worst_resid,
                          "all_converged": bool(ok)},
                "phase_ms_per_step": phase_ms_per_step,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "precision_study": precision, "batch_study": batch,
                "clocks": clocks, "wall_s_timed": wall}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0 if ok else 1


def time_solves(cfd, n, solver, seeds, warmup, max_iters=0, device=None, autotune=True, ir_form=None):
    """Standalone FP64-judged pressure solves of Gaussian right-hand sides:
    per-solve device time of the solve kernel (CUDA events inside the
    library), iterations and the true relative residual.  The solver shape
    is autotuned for the grid first (outside the timed solves)."""
    import torch
    from paper_2504_03697_gb300.synthetic import gaussian_rhs

    cav = cfd.Cavity(cfd.make_params(n, n, n, solver=solver, max_iters=max_iters), device=device)
    if autotune:
        cav.autotune(iters=30)
    if ir_form is not None and solver == "ir":
        cav.set_ir_form(ir_form)
    bs = [torch.tensor(gaussian_rhs(n, n, n, seed=s), device=device) for s in seeds]
    x = torch.zeros_like(bs[0])
    for i in range(warmup):
        cav.solve_pressure(bs[i % len(bs)], x)
    out = []
    for b in bs:
        cav.phase_times()
        cav.enable_timing(True)
        rc, st = cav.solve_pressure(b, x)
        cav.enable_timing(False)
        ms, calls = cav.phase_times()["pcg"]
        out.append({"ms": ms / max(calls, 1), "iters": st["iters"], "refinements": st["outer_iters"],
                    "rel_resid": st["rel_resid"], "rc": rc})
    del cav
    return out


def time_batch(cfd, n_cav, solver, steps, warmup, device, graph=True, seed=5):
    """Batched uneven cavities (edges from {32, 48, 64, 96}, seed 5), lid 1.0,
    nu 1e-3, dt 1e-2; per-step device time with L2 flushed between steps."""
    import torch
    from paper_2504_03697_gb300.synthetic import batch_edges, cavity_perturbation

    edges = batch_edges(n_cav, seed)
    prms = [cfd.make_params(e, e, e, dt=1e-2, nu=1e-3, lid_u=1.0, solver=solver) for e in edges]
    b = cfd.Batch(prms, device=device)
    for i, e in enumerate(edges):
        for name, f in zip("uvw", cavity_perturbation(e, e, e, 100 + i, 1e-3)):
            b.cavity(i).set_field(name, f)
    if graph:
        b.use_graph(True)
    if warmup:
        b.step(warmup, stats=False)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = b.launch_count()
    torch.cuda.synchronize(device)
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        b.step(1, stats=False)
        ev[s][1].record(stream)
    torch.cuda.synchronize(device)
    ms = [a.elapsed_time(z) for a, z in ev]
    rc, st = b.step(1, stats=True)  # one more step to read converged statistics
    cells = sum(e ** 3 for e in edges)
    out = {"cavities": n_cav, "edges_hist": {str(k): edges.count(k) for k in (32, 48, 64, 96)}, "cells": cells,
           "solver": solver, "graph": b.graph_active(), "steps": steps, "ms_per_step": sum(ms) / steps,
           "cell_steps_per_s": cells * steps / (sum(ms) / 1e3), "launches_per_step": (b.launch_count() - l0) / steps,
           "pressure_blocks": b.blocks(4 if solver == "ir" else 3),
           "all_converged": rc == cfd.CFD_OK and all(x["rel_resid"] <= 1e-8 for x in st),
           "pressure_iters_max": max(x["iters"] for x in st)}
    b.close()
    return out


def main_poisson(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd

    n = args.poisson
    form = None if args.ir_form == "tuned" else args.ir_form
    res = time_solves(cfd, n, args.solver, list(range(args.steps)), args.warmup, args.max_iters, device,
                      autotune=not args.no_autotune, ir_form=form)
    ms = sorted(r["ms"] for r in res)
    line = {"metric": "time-to-rtol-1e-8 per solve", "value": statistics.median(ms), "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "f32+f64" if args.solver == "ir" else "f64", "data": "synthetic",
            "config": {"workload": f"Neumann-Poisson {n}^3, N(0,1) right-hand sides (seeds 0..{args.steps - 1}), "
                                   f"solver {args.solver}, rtol 1e-8", "max_iters": args.max_iters,
                       "ir_form": args.ir_form if args.solver == "ir" else None},
            "solves": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.oracle_sample:
        oracle_sample_main(args)
        return 0
    if args.impl == "reference":
        return main_reference(args)
    if args.poisson > 0:
        return main_poisson(args)
    if args.batch > 0:
        return main_batch(args)
    if args.unet > 0:
        return main_unet(args)
    if args.spmv > 0:
        return main_spmv(args)
    if args.blas > 0:
        return main_blas(args)
    return main_ours(args)


def main_batch(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd

    res = time_batch(cfd, args.batch, args.solver, args.steps, args.warmup, device)
    line = {"metric": "cell-steps/s", "value": res["cell_steps_per_s"], "unit": "cell-steps/s",
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"], "dtype": "f32+f64" if args.solver == "ir" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.batch} batched uneven cavities (edges from {{32,48,64,96}}, seed 5), "
                                   f"nu 1e-3, lid 1.0, dt 1e-2, solver {args.solver}, graph-replayed steps"},
            "batch": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0



# U-Net layers (level, c_in, c_out, taps) in application order; MACs per
# fine-grid voxel = sum over layers of taps * c_in * c_out / 8^level
UNET_LAYERS = [(0, 1, 16, 27), (0, 16, 16, 27), (1, 16, 32, 27), (1, 32, 32, 27), (2, 32, 64, 27), (2, 64, 64, 27),
               (1, 96, 32, 27), (0, 48, 16, 27), (0, 16, 1, 1)]
UNET_TC_LAYERS = [1, 2, 3, 4, 5, 6, 7]  # the ones on the tensor cores


def main_unet(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd

    n = args.unet
    net = cfd.UNet(n, n, n, seed=0)
    net.set_conv_mode(args.unet_conv_mode)
    if args.unet_weights:
        net.set_params(torch.from_numpy(np.fromfile(args.unet_weights, dtype="<f4")))
    V = n ** 3
    from paper_2504_03697_gb300.synthetic import gaussian_rhs
    r = torch.from_numpy(gaussian_rhs(n, n, n, 0).reshape(-1)).to(device)
    z = torch.empty_like(r)
    for _ in range(args.warmup):
        net.apply(r, z)
    torch.cuda.synchronize()
    l0 = net.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream = torch.cuda.current_stream()
    ev[0].record(stream)
    for _ in range(args.steps):
        net.apply(r, z)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / max(args.steps, 1)
    macs = sum(t * ci * co / 8 ** lv for lv, ci, co, t in UNET_LAYERS) * V
    tc_macs = sum(UNET_LAYERS[i][3] * UNET_LAYERS[i][1] * UNET_LAYERS[i][2] / 8 ** UNET_LAYERS[i][0]
                  for i in UNET_TC_LAYERS) * V
    line = {"metric": "U-Net application time", "value": ms, "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic",
            "config": {"workload": f"3-level linear U-Net (16/32/64 channels) applied to an N(0,1) field on {n}^3 "
                                   f"cells, {'trained weights' if args.unet_weights else 'seeded init'}",
                       "convolution": args.unet_conv_mode},
            "flops_per_apply": 2 * macs, "tensor_core_flops_per_apply": 2 * tc_macs,
            "achieved_tflops": 2 * macs / (ms * 1e-3) / 1e12,
            "gpu_launches": (net.launch_count() - l0)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main_spmv(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd
    from paper_2504_03697_gb300.synthetic import uniform_field

    n = args.spmv
    cells = n ** 3
    cav = cfd.Cavity(cfd.make_params(n, n, n), device=device)
    M = cfd.CsrMatrix(n, n, n, device=device)
    x = torch.tensor(uniform_field((n, n, n), seed=1), device=device)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(args.steps):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / args.steps

    ms_free = timed(lambda: cav.apply_poisson(x, y))
    ms_csr = timed(lambda: M.spmv(x, y))
    bytes_free = 16 * cells                                   # read x, write y (halo re-reads from cache)
    bytes_csr = 16 * cells + 4 * (cells + 1) + 12 * M.nnz     # + row_ptr, col, val
    hbm = 6800.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = json.load(f).get("hbm_gbs", hbm)
    except (OSError, ValueError):
        pass
    line = {"metric": "pressure operator application time", "value": ms_free, "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"y = A x for the Neumann pressure matrix on {n}^3 cells (x uniform in [-1, 1])"},
            "matrix_free": {"ms": ms_free, "algorithmic_bytes": bytes_free,
                            "gbs": bytes_free / ms_free / 1e6, "frac_of_measured_hbm": bytes_free / ms_free / 1e6 / hbm},
            "csr": {"ms": ms_csr, "nnz": M.nnz, "algorithmic_bytes": bytes_csr, "gbs": bytes_csr / ms_csr / 1e6,
                    "frac_of_measured_hbm": bytes_csr / ms_csr / 1e6 / hbm},
            "speedup_matrix_free": ms_csr / ms_free}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def measured_hbm_gbs(default=6800.0):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("hbm_gbs", default))
    except (OSError, ValueError):
        return default


def main_blas(args):
    """Stand-alone operator and CG update kernels.  When the FP32 operand
    alone is larger than L2 (129 MB: N >= 320) the launches run back to back
    between two CUDA events; below that each launch is timed alone after an
    L2 flush (a 256 MB write), which adds the launch latency (about 6 us) to
    every sample."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd
    from paper_2504_03697_gb300.synthetic import uniform_field

    n = args.blas
    cells = n ** 3
    kk = cfd.KrylovKernels(device=device)
    x32 = torch.tensor(uniform_field((n, n, n), seed=1), device=device).float()
    y32 = torch.empty_like(x32)
    gen = torch.Generator(device="cpu").manual_seed(5)
    vec64 = [torch.rand(cells, generator=gen, dtype=torch.float64).to(device) * 2 - 1 for _ in range(4)]
    vec32 = [v.float() for v in vec64]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()

    back_to_back = 4 * cells > 129e6

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        if back_to_back:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(args.steps):
                fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / args.steps
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            ev[1].synchronize()
            total += ev[0].elapsed_time(ev[1])
        return total / args.steps

    hbm = measured_hbm_gbs()
    res = {}
    for name, fn, nbytes in (
            ("apply_poisson_f32", lambda: kk.apply_poisson_f32(x32, y32), 8 * cells),
            ("cg_update_f64", lambda: kk.cg_update(1e-3, *vec64), 48 * cells),
            ("cg_update_f32", lambda: kk.cg_update(1e-3, *vec32), 24 * cells)):
        ms = timed(fn)
        gbs = nbytes / ms / 1e6
        res[name] = {"ms": ms, "algorithmic_bytes": nbytes, "gbs": gbs, "frac_of_measured_hbm": gbs / hbm}
    a = res["apply_poisson_f32"]
    line = {"metric": "FP32 pressure operator application time", "value": a["ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"stand-alone Krylov kernels on {n}^3 cells (uniform [-1, 1] inputs)",
                       "l2": "inputs larger than L2, launches back to back" if back_to_back
                       else "flushed before every timed launch"},
            "roofline": {"bound": "hbm", "achieved": a["gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": a["frac_of_measured_hbm"], "traffic": None},
            "kernels": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
