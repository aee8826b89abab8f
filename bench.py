#!/usr/bin/env python3
"""Benchmark: cell-steps/s of the lid-driven-cavity fractional step on GB300,
and time to rtol 1e-8 per pressure solve: learned preconditioner vs plain CG.

Default workload: the 384^3 cavity (56.6 M cells) of Sec. 3 / 3.1 of arXiv
2504.03697 with lid 1.0, nu 1e-3, dt 1e-2, the seeded uniform[-1e-3, 1e-3]
perturbation (seed 5 + rank), every solve to the FP64 true-residual rtol
1e-8, on the learned + mixed-precision path (``--solver``: the pressure solve
as FP32 CG with FP64 refinement started from the previous step's pressure
corrected by the U-Net, the diffusion solves in the same mixed precision).  One bench "step" is one time
step: applyForces, advection, implicit diffusion (3 solves), divergence,
pressure solve, correction.  Inputs are synthetic and resident in HBM when
the timed region starts; at this size they are larger than L2 (no flush).

The same line carries: the same cavity with FP64 CG and with plain IR, both
warm-started too (samples of steps); time to rtol per solve of FP64 CG, IR, learned flexible
CG and IR from the learned guess on held-out 128^3 and 256^3 systems; the
64^3 FP64 cavity; the 256^3 precision study; the 64-cavity batch study; the
oracle on the host cores (single thread and all cores, a sampled step
scaled to the workload).

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
    "cavity384": dict(n=384, nu=1e-3, dt=1e-2, lid_u=1.0, seed=5, amp=1e-3, steps_total=50, warm_start=True,
                      desc="lid-driven cavity 384^3 cells (56.6 M), lid 1.0, nu 1e-3, dt 1e-2, "
                           "solves to rtol 1e-8 (FP64 true residual), pressure solves warm-started from the "
                           "previous step's p, seeded 1e-3 perturbation"),
    "cavity64": dict(n=64, nu=1e-3, dt=1e-2, lid_u=1.0, seed=2, amp=1e-3, steps_total=100,
                     desc="lid-driven cavity 64^3 cells, lid 1.0, nu 1e-3, dt 1e-2, "
                          "solves to rtol 1e-8 (FP64 true residual), seeded 1e-3 perturbation"),
    "cavity16": dict(n=16, nu=1e-2, dt=1e-2, lid_u=1.0, seed=1, amp=1e-3, steps_total=20,
                     desc="lid-driven cavity 16^3 cells, lid 1.0, nu 1e-2, dt 1e-2, "
                          "solves to rtol 1e-8 (FP64 true residual), seeded 1e-3 perturbation"),
}
SOLVER_DESC = {
    "cg": "FP64 CG (plain method)",
    "ir": "FP32 CG + FP64 refinement (mixed precision)",
    "fpcg": "flexible CG with the learned U-Net preconditioner, FP32 + FP64 refinement (graph form)",
    "guess": "learned U-Net initial guess (with a warm start: the network's correction of the previous p), then "
             "FP32 CG + FP64 refinement (mixed precision)",
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
# dram__bytes_read.sum + dram__bytes_write.sum and the L2 throughput of one
# launch of the 64^3 cavity's pressure CG in its automatic shape (the
# tile-resident single-reduction kernel cgt_fp64_kernel: 128 blocks of 256
# threads, one 32 x 8 x 8 tile each), from one ncu capture of the pressure
# solve of the timed step (the 26 MB working set is L2-resident;
# profiles/cgt_fp64_cavity64_full.md)
CGT_CAVITY64_DRAM_BYTES = 2347520 + 113408
CGT_CAVITY64_LTS_PCT = 5.2
CGT_CAVITY64_SHAPE = {"blocks": 128, "tile_depth": 8, "register_path": True, "tile_resident": True}
IR_BYTES_PER_CELL_ITER = 40
# graph form: g_dir 12 B; g_upd 20 B every other iteration (x32 read and
# written) and 12 B in between (x32 term deferred): 28 B on average
IR_GRAPH_BYTES_PER_CELL_ITER = 28
# DRAM bytes per cell and FP32 iteration of the graph-form solve, from the
# ncu capture of a 256^3 solve (whole-graph dram__bytes read + write,
# 655.6 GB, over 16.78 M cells x 1,388 iterations, refinements included;
# profiles/ir_graph_poisson256.md); the traffic of a larger solve is this
# times its cells and iterations (the solve's traffic grows in proportion)
IR_GRAPH_DRAM_BYTES_PER_CELL_ITER = 655.6e9 / (256 ** 3 * 1388)
# FP64 FMA rate of the GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz from
# the recipe's unit counts and clocks; bench.py --fp64-peak measures it
FP64_PEAK_TFLOPS = 1.26
FP64_PEAK_SOURCE = "FP64 FMA rate from the recipe's unit counts and clocks (152 x 2 x 2 x 2.07 GHz)"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cavity384")
    ap.add_argument("--solver", default="guess",
                    help="cg | ir | fpcg | guess (the cavity's solve path; --poisson/--batch: cg | ir | dic)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--warm-start", choices=["auto", "on", "off"], default="auto",
                    help="pressure solves start from the previous step's p (with --solver guess: the network "
                         "corrects that start); auto: the workload's setting")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-studies", action="store_true",
                    help="only the headline cavity (no comparison, time-to-rtol, 64^3, precision and batch blocks)")
    ap.add_argument("--sample-n", type=int, default=96, help=argparse.SUPPRESS)
    ap.add_argument("--sample-iters", type=int, default=30, help=argparse.SUPPRESS)
    ap.add_argument("--full-iters", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--poisson", type=int, default=0,
                    help="standalone Neumann-Poisson solves on an N^3 grid instead of the cavity "
                         "(one bench step = one solve of a seeded Gaussian right-hand side)")
    ap.add_argument("--max-iters", type=int, default=0, help="CG iteration cap per solve (0: 20 N)")
    ap.add_argument("--batch", type=int, default=0,
                    help="benchmark N batched uneven cavities (edges from {32,48,64,96}) instead of one cavity")
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
    ap.add_argument("--unet-conv-mode", choices=["registers", "bulk", "two_stage", "persistent"], default="bulk",
                    help="staging of the tiled convolutions (comparison)")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="measure the FP64 FMA rate (cfd_probe_fp64_fma) instead of the cavity")
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
# oracle timing (CPU baseline / reference arm): runs in child processes
# ---------------------------------------------------------------------------
# CG iterations per pressure solve of the 384^3 cavity (nu 1e-3, dt 1e-2, the
# seeded perturbation), cold and warm-started, measured on the GPU with the
# stopping rule of the oracle's CG (cold: FP64 CG; warm: the FP32/FP64 solve,
# which takes CG's iterates): used to scale the oracle's sampled cost per CG
# iteration to a whole step when no measurement of this run is at hand
CG_ITERS_PER_STEP = {(384, False): 1914, (384, True): 1716}


def oracle_sample_main(args):
    """Child process: time the FP64 oracle on a bounded sample of the
    workload and print one JSON object.

    Workloads of at most 64^3 cells run whole time steps.  Larger ones run
    one step of the same-parameter cavity at args.sample_n^3 with the
    pressure CG cut to args.sample_iters iterations (replayed with the
    oracle's fixed-iteration mode) after its CSR assembly; the sweeps
    (forces, advection, diffusion, divergence, correction, gauge) and the
    assembly are scaled to the workload by the cell count, the CG by cells x
    the workload's CG iterations per solve (args.full_iters)."""
    from oracle import fractional_step as fs
    from oracle.krylov import pcg
    from oracle.mac import Cavity
    from oracle.operators import poisson_csr
    from paper_2504_03697_gb300.synthetic import cavity_perturbation

    wl = WORKLOADS[args.workload]
    n = wl["n"]
    if n <= 64:
        cav = Cavity(n, n, n, dt=wl["dt"], nu=wl["nu"], lid_u=wl["lid_u"])
        st = fs.initial_state(cav, cavity_perturbation(n, n, n, wl["seed"], wl["amp"]))
        for _ in range(args.warmup):
            st, _ = fs.step(cav, st)
        t0 = time.perf_counter()
        per_step = []
        while len(per_step) < args.steps:
            a = time.perf_counter()
            st, _ = fs.step(cav, st)
            per_step.append(time.perf_counter() - a)
            if time.perf_counter() - t0 > args.max_seconds:
                break
        el = sum(per_step)
        print(json.dumps({"steps": len(per_step), "seconds": el, "cells": n ** 3, "per_step_s": per_step,
                          "value": n ** 3 * len(per_step) / el,
                          "sample": f"{len(per_step)} whole time steps of the {n}^3 cavity"}))
        return
    ns, k = args.sample_n, args.sample_iters
    cav = Cavity(ns, ns, ns, dt=wl["dt"], nu=wl["nu"], lid_u=wl["lid_u"])
    st = fs.initial_state(cav, cavity_perturbation(ns, ns, ns, wl["seed"], wl["amp"]))
    scale = (n / ns) ** 3
    full = args.full_iters
    estimates = []
    for rep in range(args.warmup + args.steps):
        u, v, w, _ = st
        t0 = time.perf_counter()
        u, v, w = fs.apply_forces(cav, u, v, w)
        u, v, w = fs.advect(cav, u, v, w)
        (u, v, w), _ = fs.diffuse(cav, (u, v, w))
        b = fs.pressure_rhs(cav, u, v, w)
        A = poisson_csr(ns, ns, ns)
        t1 = time.perf_counter()
        x, _ = pcg(A, b.ravel(), rtol=cav.rtol, max_iters=k, fixed_iters=k)
        t2 = time.perf_counter()
        x = x.reshape(cav.cell_shape)
        u, v, w = fs.correct(cav, u, v, w, x)
        st = (u, v, w, fs.gauge(x))
        t3 = time.perf_counter()
        sweeps = (t1 - t0) + (t3 - t2)
        per_iter = (t2 - t1) / k
        est = scale * (sweeps + per_iter * full)
        if rep >= args.warmup:
            estimates.append({"sweeps_s": sweeps, "cg_s_per_iter": per_iter, "est_step_s": est,
                              "wall_s": t3 - t0})
    wall = sum(e["wall_s"] for e in estimates)
    est_total = sum(e["est_step_s"] for e in estimates)
    print(json.dumps({"steps": len(estimates), "seconds": wall, "est_seconds": est_total, "cells": n ** 3,
                      "value": n ** 3 * len(estimates) / est_total, "per_step": estimates,
                      "sample": f"{len(estimates)} time step(s) of the same-parameter {ns}^3 cavity with the "
                                f"pressure CG cut to {k} iterations (after its CSR assembly); sweeps and "
                                f"assembly scaled by the cell ratio {scale:.0f}, CG by the cell ratio x "
                                f"{full} FP64 CG iterations per solve"}))


def run_oracle_child(workload, steps, warmup, max_seconds, sample_n=96, sample_iters=30, full_iters=0, threads=1):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "LOCAL_WORLD_SIZE", "GROUP_RANK", "ROLE_RANK"):
        env.pop(k, None)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", workload,
           "--steps", str(steps), "--warmup", str(warmup), "--max-seconds", str(max_seconds),
           "--sample-n", str(sample_n), "--sample-iters", str(sample_iters), "--full-iters", str(full_iters)]
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)


def collect_oracle(proc):
    out, err = proc.communicate()
    if proc.returncode != 0:
        raise RuntimeError("oracle sample failed: " + err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def oracle_baseline(workload, full_iters, max_seconds=60.0):
    """The oracle on the host cores: one single-thread sample, then one
    sample per host core at once (independent cavities, weak scaling)."""
    one = collect_oracle(run_oracle_child(workload, 1, 0, max_seconds, full_iters=full_iters))
    cores = os.cpu_count() or 1
    procs = [run_oracle_child(workload, 1, 0, max_seconds, full_iters=full_iters) for _ in range(cores)]
    many = [collect_oracle(p) for p in procs]
    return {"value": one["value"], "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": one["sample"] + " (FP64 numpy/scipy oracle, one thread)",
            "all_cores": {"value": sum(m["value"] for m in many), "cores": cores,
                          "sample": f"{cores} concurrent single-thread oracle processes, each the sample above"},
            "cpu": cpu_model(), "host_cores": cores}


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
    full = CG_ITERS_PER_STEP.get((wl["n"], wl.get("warm_start", False)), 0)
    res = collect_oracle(run_oracle_child(args.workload, args.steps, args.warmup, args.max_seconds, sample_n=64,
                                          sample_iters=40, full_iters=full))
    value = res["value"]
    sample = res["sample"] + f" per timed step, after {args.warmup} warm-up sample(s); FP64 numpy/scipy oracle, " \
                             f"single thread"
    line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": res["steps"], "warmup": args.warmup,
            "ms_per_step": 1e3 * wl["n"] ** 3 / value, "higher_is_better": True,
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
def weights_path():
    return os.path.join(ROOT, "paper_2504_03697_gb300", "weights", "unet_cavity128.f32")


def make_cavity(cfd, n, wl, solver, device, params=None, advect_order=1, warm_start=False):
    """A cavity of the workload with one of the solver paths: 'cg' (FP64 CG),
    'ir' (FP32 CG + FP64 refinement), 'fpcg' (flexible CG with the learned
    U-Net, mixed precision, graph form), 'guess' (IR from the learned initial
    guess).  Returns (cavity, network or None)."""
    kw = dict(dt=wl["dt"], nu=wl["nu"], lid_u=wl["lid_u"], advect_order=advect_order, warm_start=warm_start)
    if solver == "guess":
        prm = cfd.make_params(n, n, n, solver="ir", learned_guess=True, **kw)
    else:
        prm = cfd.make_params(n, n, n, solver=solver, **kw)
    cav = cfd.Cavity(prm, device=device)
    net = None
    if solver in ("fpcg", "guess"):
        net = cfd.UNet(n, n, n, seed=0, device=device)
        net.set_params(params)
        cav.attach_preconditioner(net)
    return cav, net


def init_fields(cav, n, wl, seed_offset=0):
    from paper_2504_03697_gb300.synthetic import cavity_perturbation
    for name, f in zip("uvw", cavity_perturbation(n, n, n, wl["seed"] + seed_offset, wl["amp"])):
        cav.set_field(name, f)


def timed_steps(cav, steps, stream, device, flush=None):
    """Per-step device time (CUDA events on the cavity's stream), L2 flushed
    before each step when a flush buffer is given."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize(device)
    for s in range(steps):
        if flush is not None:
            flush.zero_()
        ev[s][0].record(stream)
        cav.step(1, stats=False)
        ev[s][1].record(stream)
    torch.cuda.synchronize(device)
    return [a.elapsed_time(b) for a, b in ev]


def cavity_sample(cfd, n, wl, solver, steps, warmup, device, params=None, warm_start=False):
    """Cell-steps/s of the workload's cavity with another solver path, on a
    sample of steps (warm-up steps first); returns a summary dict."""
    import torch
    cav, net = make_cavity(cfd, n, wl, solver, device, params, warm_start=warm_start)
    init_fields(cav, n, wl)
    if solver in ("cg", "ir"):
        cav.autotune(iters=30)
    if warmup:
        cav.step(warmup, stats=False)
    cav.phase_times()
    cav.enable_timing(True)
    ms = timed_steps(cav, steps, torch.cuda.current_stream(device), device)
    cav.enable_timing(False)
    ph = cav.phase_times()
    rc, st = cav.recent_stats(steps)
    shape0 = cav.solver_shape(0)
    out = {"solver": solver, "warm_start": warm_start, "steps_timed": steps, "warmup": warmup,
           "ms_per_step": sum(ms) / steps, "step_ms": [round(m, 3) for m in ms],
           "cell_steps_per_s": n ** 3 * steps / (sum(ms) / 1e3),
           "pressure_ms_per_step": ph["pcg"][0] / steps, "diffuse_ms_per_step": ph["diffuse"][0] / steps,
           "pressure_iters": [s["iters"] for s in st], "refinements": [s["outer_iters"] for s in st],
           "pressure_shape": shape0,
           "all_converged": rc == cfd.CFD_OK and all(s["rel_resid"] <= 1e-8 * 1.0000001 for s in st)}
    del cav, net
    torch.cuda.empty_cache()
    return out


def time_to_rtol(cfd, params, device, sizes=(128, 256), fpcg_systems=None):
    """Time to the FP64 true-residual rtol 1e-8 per solve of FP64 CG, IR,
    learned FPCG (mixed precision, graph form) and IR from the learned guess,
    on held-out cavity pressure systems (seeds 200..203, step 10) and a
    Gaussian right-hand side.  Flexible CG applies the network in every
    iteration; at 256^3 it is timed on fpcg_systems[256] system(s) only."""
    import torch
    from paper_2504_03697_gb300 import learned
    fpcg_systems = fpcg_systems or {256: 1}
    out = {}
    for n in sizes:
        systems = learned.eval_systems(n)
        res = {}
        for label in learned.SOLVERS:
            use = systems[:fpcg_systems[n]] if (label == "fpcg" and n in fpcg_systems) else systems
            r = learned.evaluate(n, params, use, solvers=(label,), log=lambda *a: None)
            res[label] = dict(r["summary"][label], systems=len(use),
                              converged=all(e["status"] == 0 and e["rel_resid"] <= 1e-8 * 1.0000001
                                            for row in r["rows"].values() for e in row),
                              plain_iters=[e["plain_iters"] for row in r["rows"].values() for e in row])
        cg = res["cg"]["median_ms"]
        out[str(n)] = {"systems": [nm for nm, _ in systems], "solvers": res,
                       "speedup_vs_fp64_cg": {k: cg / v["median_ms"] for k, v in res.items()}}
        del systems
        torch.cuda.empty_cache()
    return out


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

    wl = WORKLOADS[args.workload]
    n = wl["n"]
    cells = n ** 3
    solver = args.solver
    warm = wl.get("warm_start", False) if args.warm_start == "auto" else args.warm_start == "on"
    params = None
    if solver in ("fpcg", "guess"):
        from paper_2504_03697_gb300 import learned
        path = args.unet_weights or weights_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: the learned solvers need the trained U-Net parameters")
        params = learned.load_params(path)
    stream = torch.cuda.current_stream(device)
    cav, net = make_cavity(cfd, n, wl, solver, device, params, args.advect_order, warm)
    init_fields(cav, n, wl, rank)
    cav.set_cg_variant(args.cg_variant) if solver == "cg" else None
    if args.concurrent_diffusion == "off" and solver in ("cg", "jacobi"):
        cav.set_concurrent_diffusion(False)
    # solver shape for this grid (blocks per SM x tile depth), picked by
    # timing fixed-length solves; outside the timed region, state untouched
    tune = None if (args.no_autotune or solver not in ("cg", "ir")) else cav.autotune(iters=50)

    # the clock sampler (nvidia-smi) starts before the warm-up steps, so that
    # its start-up is over before the timed region, which it samples
    sampler = ClockSampler(physical_gpu(local)) if rank == 0 else None
    if args.warmup > 0:
        cav.step(args.warmup, stats=True)
    # inputs larger than L2 (129 MB) need no flush: the 384^3 state is ~7 GB
    big = cells * 8 * 4 > 512 * 1024 * 1024
    flush = None if big else torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)

    cav.phase_times()  # reset
    cav.enable_timing(True)
    launches0 = cav.launch_count()
    barrier(dist, device)
    torch.cuda.synchronize(device)
    wall0 = time.perf_counter()
    step_ms = timed_steps(cav, args.steps, stream, device, flush)
    wall = time.perf_counter() - wall0
    barrier(dist, device)
    clocks = sampler.stop() if sampler else None
    launches = cav.launch_count() - launches0
    cav.enable_timing(False)
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
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    if solver == "cg":
        flops = cells * (CG_FLOPS_PER_CELL_ITER * mean_iters + CG_FLOPS_PER_CELL_SOLVE)
        bytes_ = cells * (CG_BYTES_PER_CELL_ITER * mean_iters + CG_BYTES_PER_CELL_SOLVE)
        achieved = flops / pcg_avg_s / 1e12
        shape0 = cav.solver_shape(0)
        roofline = {"bound": "alu", "kernel": "cgt_fp64_kernel (pressure CG, tile-resident single-reduction form)"
                    if shape0["tile_resident"] else "cg1_fp64_kernel / cg_fp64_kernel (pressure CG, persistent)",
                    "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": CGT_CAVITY64_DRAM_BYTES if (args.workload == "cavity64"
                                                           and shape0 == CGT_CAVITY64_SHAPE) else None,
                    "peak_source": FP64_PEAK_SOURCE, "launch_ms": pcg_avg_s * 1e3,
                    "hbm_achieved_gbs": bytes_ / pcg_avg_s / 1e9, "hbm_frac_of_measured": bytes_ / pcg_avg_s / 1e9 / hbm_peak}
    else:
        # the FP32 iteration of the graph form moves 28 B per cell on average
        # (g_dir reads r32, p_old and writes p; g_upd reads p, r32 and writes
        # r32, and reads and writes x32 every other iteration);
        # the FP64 refinements and the learned guess are inside the timed
        # solve but left out of the algorithmic bytes (a lower bound on frac)
        ir_bytes = cells * IR_GRAPH_BYTES_PER_CELL_ITER * mean_iters
        gbs = ir_bytes / pcg_avg_s / 1e9
        roofline = {"bound": "hbm", "kernel": "g_dir + g_upd (FP32 CG iteration, graph form; whole pressure solve timed)",
                    "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "traffic": IR_GRAPH_DRAM_BYTES_PER_CELL_ITER * cells * mean_iters
                    if IR_GRAPH_DRAM_BYTES_PER_CELL_ITER else None,
                    "peak_source": peak_src, "launch_ms": pcg_avg_s * 1e3, "bytes_per_launch": ir_bytes}
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
        del host
    del cav, net
    torch.cuda.empty_cache()

    extra = {}
    if rank == 0 and world == 1 and not args.no_studies:
        # the same cavity with the other solver paths (samples of steps)
        extra["same_cavity"] = {}
        # the same warm-up steps as the headline, so that the timed steps
        # start at the same point of the flow
        for other, k_steps, warm_steps in (("cg", 2, args.warmup), ("ir", 4, args.warmup)):
            if other != solver:
                extra["same_cavity"][other] = cavity_sample(cfd, n, wl, other, k_steps, warm_steps, device, params,
                                                            warm_start=warm)
        extra["same_cavity"]["note"] = (f"samples of {wl['steps_total']} steps: FP64 CG 2 timed steps, IR 4, both after "
                                        f"the headline's {args.warmup} warm-up steps (compare with the headline's "
                                        f"first steps in step_ms); flexible CG with the network in every iteration is timed on "
                                        f"standalone systems only (time_to_rtol), since one application of the "
                                        f"network costs tens of FP32 iterations at this size")
        if params is not None:
            extra["time_to_rtol"] = time_to_rtol(cfd, params, device)
        # the 64^3 FP64 cavity (plain method on the GPU)
        c2 = cavity_sample(cfd, 64, WORKLOADS["cavity64"], "cg", 20, 3, device)
        # its pressure CG against the rooflines that bound it at this size:
        # the FP64 pipe (the kernel is FP64-ALU-bound) and L2 (the 26 MB
        # working set is L2-resident; DRAM sees ~2.4 MB per solve)
        cells64 = 64 ** 3
        its = sum(c2["pressure_iters"]) / len(c2["pressure_iters"])
        t_s = c2["pressure_ms_per_step"] / 1e3
        flops = (CG_FLOPS_PER_CELL_ITER * its + CG_FLOPS_PER_CELL_SOLVE) * cells64
        l2_bytes = (CG_BYTES_PER_CELL_ITER * its + CG_BYTES_PER_CELL_SOLVE) * cells64
        c2["roofline"] = {
            "bound": "alu", "kernel": "cgt_fp64_kernel (pressure CG, tile-resident single-reduction form)"
            if c2.get("pressure_shape", {}).get("tile_resident") else "cg1_fp64_kernel (pressure CG, single-reduction form)",
            "achieved": flops / t_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": flops / t_s / 1e12 / FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_SOURCE,
            "l2": {"algorithmic_bytes_per_solve": l2_bytes, "achieved_GBs": l2_bytes / t_s / 1e9,
                   # the ncu figures belong to the captured launch shape only
                   "ncu_lts_throughput_pct": CGT_CAVITY64_LTS_PCT if c2.get("pressure_shape") == CGT_CAVITY64_SHAPE
                   else None,
                   "dram_bytes_per_solve": CGT_CAVITY64_DRAM_BYTES if c2.get("pressure_shape") == CGT_CAVITY64_SHAPE
                   else None,
                   "source": "profiles/cgt_fp64_cavity64_full.md (lts__throughput.avg.pct_of_peak_sustained_"
                             "elapsed and dram bytes of one launch)"}}
        extra["cavity64_fp64_cg"] = c2
        # standalone 256^3 Poisson, FP64 CG vs FP32/FP64-IR (2 of 32 RHS)
        study = {}
        for sv in ("cg", "ir"):
            res = time_solves(cfd, 256, sv, [0, 1], 1, 0, device)
            study[sv] = {"ms_per_solve": [round(r["ms"], 3) for r in res], "iters": [r["iters"] for r in res],
                         "refinements": [r["refinements"] for r in res], "rel_resid": [r["rel_resid"] for r in res]}
        extra["precision_study"] = {
            "workload": "Neumann-Poisson 256^3, N(0,1) right-hand sides, rtol 1e-8 (true FP64); sample: seeds 0-1 "
                        "of the 32", "fp64_cg": study["cg"], "fp32_cg_fp64_refined": study["ir"],
            "speedup_ir_over_fp64_cg": statistics.mean(study["cg"]["ms_per_solve"]) /
            statistics.mean(study["ir"]["ms_per_solve"])}
        extra["batch_study"] = {sv: time_batch(cfd, 64, sv, 3, 1, device) for sv in ("cg", "ir")}
        extra["batch_study"]["note"] = "sample: 3 timed steps of the 50 (after 1 warm-up step), graph-replayed"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        full = CG_ITERS_PER_STEP.get((n, warm), 0)
        cgs = extra.get("same_cavity", {}).get("cg")
        if cgs:
            full = int(round(float(np.mean(cgs["pressure_iters"]))))
        cpu = oracle_baseline(args.workload, full)

    if rank == 0:
        line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"cg": "f64", "ir": "f32+f64", "fpcg": "bf16+f32+f64", "guess": "bf16+f32+f64"}[solver],
                "data": "synthetic",
                "config": {"workload": wl["desc"] + f"; solver {SOLVER_DESC[solver]}", "n": n, "cells": cells,
                           "solver": solver, "steps_per_rank": args.steps,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": ("inputs larger than L2 (state ~%.1f GB), no flush" % (cells * 8 * 13 / 1e9)) if big
                           else "flushed between timed steps (256 MiB write outside the timed events)",
                           "solver_shape": tune if tune is not None else "automatic",
                           "weights": os.path.relpath(args.unet_weights or weights_path(), ROOT) if params is not None
                           else None, "advect_order": args.advect_order, "warm_start": warm},
                "solve": {"pcg_iters_mean": mean_iters, "pcg_iters_min": min(iters), "pcg_iters_max": max(iters),
                          "time_to_rtol_ms_mean": pcg_avg_s * 1e3, "rel_resid_max": worst_resid,
                          "all_converged": bool(ok), "refinements": [s["outer_iters"] for s in stats]},
                "step_ms": [round(m, 3) for m in step_ms],
                "phase_ms_per_step": phase_ms_per_step,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "wall_s_timed": wall}
        line.update(extra)
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
    if args.fp64_peak:
        return main_fp64_peak(args)
    return main_ours(args)


def main_fp64_peak(args):
    """FP64 FMA rate of the device: a resident wave of DFMA-chain blocks
    (8 blocks of 256 threads per SM), best of `steps` timed launches after
    `warmup` (CUDA events on the launching stream)."""
    import ctypes

    import torch
    torch.cuda.set_device(0)
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd
    lib = cfd.load_library()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, iters = sms * 8, 20000
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flops = 2.0 * 8 * iters * 256 * blocks
    times = []
    for i in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = lib.cfd_probe_fp64_fma(blocks, iters, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        b.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(lib.cfd_last_error(None).decode())
        if i >= args.warmup:
            times.append(a.elapsed_time(b) / 1e3)
    best = min(times)
    line = {"metric": "FP64 FMA rate", "value": flops / best / 1e12, "unit": "TFLOP/s", "higher_is_better": True,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{blocks} blocks x 256 threads x 8 DFMA chains x {iters} (best of {args.steps})",
                       "sms": sms, "flop_per_launch": flops},
            "ms_per_launch": [t * 1e3 for t in times]}
    print(json.dumps(line), flush=True)
    return 0


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
    # one training step (one pair: forward, loss, backward with input and
    # weight gradients, Adam) with the weight gradients on the tensor cores
    # and on the CUDA cores; a training step does about 3x the forward flops
    e = torch.from_numpy(gaussian_rhs(n, n, n, 1).reshape(-1)).to(device)
    train = {}
    for mode in ("tensor", "cuda_cores"):
        net.set_wgrad_mode(mode)
        net.train_step(r, e, lr=0.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            net.train_step(r, e, lr=0.0)
        b.record(stream)
        torch.cuda.synchronize()
        train[mode] = a.elapsed_time(b) / reps
    line["train_step_ms_one_pair"] = train
    line["train_step_tflops"] = {k: 3 * 2 * macs / (v * 1e-3) / 1e12 for k, v in train.items()}
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
