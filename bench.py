"""Benchmark: FP64 cell-updates per second per RK stage of the GB300 Euler solver.

Workload (the metric's configuration): 2D Euler, Kelvin-Helmholtz shear layer
on a periodic 4096 x 4096 grid, FP64, MUSCL-minmod + Roe flux + SSP-RK3 with
CFL 0.5.  One bench step is one SSP-RK3 time step (CFL time-step reduction +
three fused stage kernels), replayed from a CUDA graph by fv_run; the state
keeps evolving across steps as in the 200-step run.
  value = cells * 3 stages * steps / device time (CUDA events, max over ranks)
  e2e   = the same through fv_run with a pinned HOST state: every step copies
          the state in, advances it and copies it back.
The state (537 MB) is larger than L2 (129 MB), so no flush is needed.

At one GPU the default run adds two objects to the line:
  tuned     -- the autotuner (FCNN surrogate, Sec. 3.3-3.6) on KH 4096^2 with a
               bounded sample, then the naive default launch (32x8 threads,
               one cell per thread, a grid covering the domain), the library's
               default launch, the search's pick and the exhaustive best of the
               reduced space, timed interleaved (median of >= 5 replays each);
  workloads -- short timed runs of the other forward configurations (3D
               Taylor-Green 384^3, the 96-grid batched Sod set) and of the
               adjoint gradient (1024^2 vortex, 400 steps), each with its own
               clocks and CPU-oracle baseline.
--launch TILE:THREADS[:march] times one explicit launch (all three RK stages)
instead of the default.

--impl reference times the CPU oracle (the only reference this paper has; it
ships no code) on the host cores, on a bounded band of the same workload.
Multi-GPU: the method does not shard here; N ranks run N independent replicas
(weak scaling), value = all ranks' cell-stages / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS_SIDE = 4096
METRIC = "FP64 cell-updates/s per RK stage (2D Euler KH 4096^2, MUSCL-minmod + Roe + SSP-RK3)"
UNIT = "cell-stage/s"
# Algorithmic FP64 work per cell and RK stage, counted on the CPU oracle with an
# operation-counting scalar (python -m oracle.count_flops; 2D value at n = 4096,
# 3D at n = 384): every +, -, *, /, sqrt of the plain method counts one FLOP.
FLOP_PER_CELL_STAGE_2D = 496.44
FLOP_PER_CELL_STAGE_3D = 959.62
# Algorithmic HBM bytes per cell-stage: stage 1 reads U^n and writes U^1 (nvar
# + nvar doubles), stages 2 and 3 read U^s and U^n and write (3 nvar doubles):
# 8 nvar doubles per cell and step over 3 stages.
BYTES_PER_CELL_STAGE_2D = 256.0 / 3.0
BYTES_PER_CELL_STAGE_3D = 320.0 / 3.0
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz
# (a DFMA loop measured 1.18 TFLOP/s on this part).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM traffic of one stage-kernel launch from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, full 4096^2 launches, mean of the three stages of one
# step), valid for the kernel sources whose hash and the launch shape recorded
# with it; null otherwise.
STAGE_TRAFFIC = {"bytes": 1.3891e9, "source_hash": "b015986973ece0c2", "tile": [64, 16, 1], "threads": 192}
# FP64 instructions the fused stage kernels execute per cell and stage (ncu
# sm__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on, mean of the three
# stages at 2048^2 / 192^3), for the kernel sources with this hash; and the
# FP64 products evaluated on the integer pipe instead: 29 per face in 2D and 32
# in 3D (the Roe flux's products), times the faces per cell of the default
# tiles (2.078 for 64x16, 3.375 for 8x8x8).
STAGE_FP64_INST = {"2d": 114.3, "3d": 231.2, "source_hash": "b015986973ece0c2"}
INT_PIPE_PRODUCTS = {"2d": 60.3, "3d": 108.0}


# The naive default launch of the tuning comparison: 32x8 threads, one cell
# per thread, one CTA per 32x8 tile covering the domain (the analogue of a
# directive compiler's default launch).
NAIVE_TILE_2D, NAIVE_THREADS_2D = (32, 8, 1), 256


def parse_launch(text: str, dim: int):
    """'32x32:160' -> ((32, 32, 1), 160, 0); '16x15x32:256:march' -> (..., 1)."""
    parts = text.split(":")
    if len(parts) not in (2, 3) or (len(parts) == 3 and parts[2] != "march"):
        raise ValueError(f"bad launch {text!r}: expected TILE:THREADS[:march]")
    tile = tuple(int(x) for x in parts[0].lower().split("x"))
    if len(tile) != dim:
        raise ValueError(f"bad launch {text!r}: a {dim}D tile has {dim} extents")
    if dim == 2:
        tile = tile + (1,)
    march = 1 if len(parts) == 3 else 0
    if march and dim != 3:
        raise ValueError(f"bad launch {text!r}: the marching kernel is 3D only")
    return tile, int(parts[1]), march


def launch_with(fv, g, tile, threads, march=0):
    """The default launch of grid g with one tile shape and thread count for
    all three RK stages."""
    d = fv.launch_to_dict(fv.fv_default_launch(g if not isinstance(g, list) else g[0]))
    for st in d["stage"]:
        st.update(tile=tuple(tile), threads=threads, march=march)
    return d


def kernel_source_hash() -> str:
    """Hash of the stage kernel's code (comments and blank lines removed, so a
    comment edit does not retire a recorded measurement)."""
    h = hashlib.sha256()
    for f in ("fv_stage.cuh", "fv_device.cuh", "fv_emu.h", "fv_internal.h", "fv_stage2d.cu", "fv_stage2d_wide.cu",
              "fv_stage3d.cu"):
        with open(os.path.join(ROOT, "paper_2306_14011_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.path = None
        if shutil.which("nvidia-smi") is None:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id is not None:
            cmd += ["-i", str(gpu_id)]
        self.out = open(self.path, "w")
        self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("[N/A]", ""))}


def gpu_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself at N = 1."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (weak scaling)."""
    return world * units_per_rank / seconds_max


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        return dist, rank, world
    return None, rank, world


def run_ours(args):
    import torch

    from paper_2306_14011_gb300 import fv
    from paper_2306_14011_gb300 import inputs as I

    dist, rank, world = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    W = make_workload(args, I)
    g, U0 = W["grid"], W["U0"]
    cells = W["cells"]
    split = args.mode == "split"
    if split and W["batched"]:
        raise SystemExit("--mode split: batched contexts run the fused persistent kernel only")
    launch = None
    if args.launch:
        tile, thr, march = parse_launch(args.launch, g.dim if not W["batched"] else 2)
        launch = launch_with(fv, g, tile, thr, march)
    solver = fv.Solver(g, stream=stream, mode=fv.FV_SPLIT if split else None, launch=launch)
    U = torch.from_numpy(U0).to(dev) if not W["batched"] else solver.pack(
        [torch.from_numpy(u).to(dev) for u in W["states"]])
    if W["batched"]:
        U0 = U.cpu().numpy()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up: untimed steps (first call captures the graphs)
    solver.run(U, args.warmup)
    barrier()

    clocks = ClockSampler(gpu_uuid(torch))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    solver.run(U, args.steps)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, dist, dev)
    solver.sync()  # reports non-physical / timeout flags of the timed region

    # dominant kernel.  Single grid (fused stage kernel): average launch
    # duration over the timed region = (timed region - K x the time-step
    # reduction) / (3 K); the reduction (memset + dt kernel) is timed alone with
    # CUDA events right after.  Batch: the one persistent launch of the timed
    # region, per RK stage (it also runs the per-problem CFL phases).
    dt_ms = 0.0
    if not W["batched"]:
        dtbuf = torch.zeros(1, dtype=torch.float64, device=dev)
        reps = max(3, min(args.steps, 20))
        fv.fv_time_step(solver.ctx, U, dtbuf)
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(reps):
            fv.fv_time_step(solver.ctx, U, dtbuf)
        e3.record(stream)
        torch.cuda.synchronize()
        dt_ms = e2.elapsed_time(e3) / reps
    stage_ms = (ms - args.steps * dt_ms) / (3 * args.steps)

    # end to end through the C ABI with a pinned host state
    e2e = None
    if args.e2e_steps > 0:
        Uh_t = torch.from_numpy(U.cpu().numpy()).pin_memory()
        Uh = Uh_t.numpy()
        solver.run(Uh, 1)  # warm (allocates the staging buffers, captures graphs)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            solver.run(Uh, 1)  # H2D copy, one SSP-RK3 step, D2H copy, wait
        t1 = time.perf_counter()
        e2e = {"value": whole_job_rate(cells * 3 * args.e2e_steps, world, max_over_ranks(t1 - t0, dist, dev)),
               "unit": UNIT,
               "h2d_bytes_per_step": int(U0.nbytes), "d2h_bytes_per_step": int(U0.nbytes),
               "steps": args.e2e_steps}

    if rank != 0:
        solver.close()
        return None

    value = whole_job_rate(cells * 3 * args.steps, world, ms_max / 1e3)
    flops_per_launch = W["flop"] * cells
    achieved_tflops = flops_per_launch / (stage_ms / 1e3) / 1e12
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    achieved_gbs = W["bytes"] * cells / (stage_ms / 1e3) / 1e9
    st0 = solver.launch["stage"][0]
    traffic = STAGE_TRAFFIC["bytes"] if (not split and STAGE_TRAFFIC["source_hash"] == kernel_source_hash() and
                                         list(st0["tile"]) == STAGE_TRAFFIC["tile"] and
                                         st0["threads"] == STAGE_TRAFFIC["threads"]) else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": W["data"],
        "config": {"workload": W["desc"], "cells": cells, "launch": args.launch or "default",
                   "launch_params": solver.launch,
                   "kernel_structure": ("split: per stage %d kernels (limiter and flux per axis, source, RHS, "
                                        "update; Sec. 3.4), intermediates in HBM" % (2 * g.dim + 3)) if split
                   else "fused: one kernel per RK stage",
                   "l2": "state (%.0f MB) larger than L2, no flush" % (U0.nbytes / 1e6),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": traffic if W["name"] == "kh4096" else None,
                     "kernel": ("all %d split kernels of one stage (per-kernel times: profiles)" % (2 * g.dim + 3))
                     if split else W["kernel"], "stage_ms": stage_ms, "dt_kernel_ms": dt_ms,
                     "flop_per_cell_stage": W["flop"],
                     "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz",
                     "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": (achieved_gbs / hbm_peak) if hbm_peak else None,
                     "bytes_per_cell_stage": W["bytes"]},
        "e2e": e2e,
        "gpu_launches": ((2 + 3 * (2 * g.dim + 3)) if split else W["launches_per_step"]) * args.steps
        if not W["batched"] else 1,
        "clocks": clk,
        "impl": "ours",
    }
    if not W["batched"] and not split:
        # the kernel's FP64 instruction rate against a DFMA stream kernel on
        # the same device and clock (the issue-rate ceiling in practice)
        stream_rate = fv.fv_debug_fp64_rate(0)
        int_rate, mixed_rate = fv.fv_debug_fp64_rate(2), fv.fv_debug_fp64_rate(3)
        inst = STAGE_FP64_INST["2d" if g.dim == 2 else "3d"]
        if STAGE_FP64_INST["source_hash"] != kernel_source_hash():
            inst = None
        rate = inst * cells / (stage_ms / 1e3) if inst else None
        key = "2d" if g.dim == 2 else "3d"
        prod = INT_PIPE_PRODUCTS[key] * cells / (stage_ms / 1e3) if inst else None
        line["roofline"]["fp64_stream"] = {
            "dfma_stream_lane_ops_per_s": stream_rate, "kernel_fp64_inst_per_cell_stage": inst,
            "kernel_fp64_lane_ops_per_s": rate, "frac_of_stream": rate / stream_rate if rate else None,
            "int_pipe_products_per_cell_stage": INT_PIPE_PRODUCTS[key] if inst else None,
            "kernel_int_pipe_products_per_s": prod,
            "int_pipe_product_stream_ops_per_s": int_rate, "dfma_beside_int_products_stream_ops_per_s": mixed_rate,
            # the kernels' FP64 instructions plus their integer-pipe products
            # per second, against DFMA chains beside integer-pipe product
            # chains: the ceiling of the two pipes working together
            "combined_frac_of_mixed_stream": (rate + prod) / mixed_rate if rate else None,
            "note": "FP64 pipe share of the work; the flux products run on the integer pipe beside it"}
    if args.workload != "kh4096":
        line["metric"] = W["metric"]
    if world == 1 and not W["batched"] and args.tune_samples > 0:
        line["tuned"] = tuned_comparison(args, fv, solver, U, g, stream, W)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = W["cpu_baseline"]()
    solver.close()
    del U
    if world == 1 and W["name"] == "kh4096" and not split and args.workloads:
        line["workloads"] = other_workloads(args)
    return line


def tuned_comparison(args, fv, solver, U, g, stream, W):
    """The metric's second half, tuned vs default launch (Sec. 3.4-3.6): run
    the autotuner on the workload with a bounded sample, then time four
    launches interleaved -- the naive default (32x8 threads, one cell per
    thread), the library's default, the search's own pick and the exhaustive
    best of the reduced space -- each the median of `tune_replays` graph
    replays of `tune_steps` SSP-RK3 steps (CUDA events on the solver's
    stream), with clocks sampled during the comparison.  The launch the tuner
    returns (the fastest of search, default and exhaustive best in its own
    final timing) is left installed."""
    import torch
    default = solver.launch
    t0 = time.perf_counter()
    best, rep = solver.tune(U, samples=args.tune_samples, steps=2, candidates=args.tune_candidates, top=16, rounds=3,
                            refine=1, exhaustive=1, final_repeats=5, seed=7)
    tuner_s = time.perf_counter() - t0
    # the naive default: fused 2D kernels at one cell per thread (in the split
    # structure the library default already is one item per thread)
    naive = launch_with(fv, g, NAIVE_TILE_2D, NAIVE_THREADS_2D) if g.dim == 2 and args.mode == "fused" else None
    launches = {"naive_default": naive, "current_default": default, "search": rep["search_best"],
                "exhaustive_best": rep["exhaustive_best"]}
    for k in list(launches):
        if launches[k] is None:
            del launches[k]
    times = {k: [] for k in launches}
    clocks = ClockSampler(gpu_uuid(torch))
    for _ in range(args.tune_replays):
        for k, l in launches.items():
            solver.launch = l
            solver.run(U, 2)  # captures this launch's graphs; untimed
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.run(U, args.tune_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            times[k].append(e0.elapsed_time(e1) / args.tune_steps)
    clk = clocks.stop()
    solver.launch = best
    solver.sync()
    med = {k: statistics.median(v) for k, v in times.items()}
    cells = g.ncells

    def entry(k):
        return {"ms_per_step": med[k], "value": cells * 3 / (med[k] / 1e3), "replays_ms_per_step": times[k],
                "launch": launches[k]}

    out = {
        "workload": W["name"] + (" (split kernels, the paper's space)" if args.mode == "split" else "") +
                    "; the state as evolved by the timed run",
        "unit": UNIT,
        "current_default": dict(entry("current_default"), note="the library's hand-set default, itself the outcome "
                                                               "of earlier tuner runs and launch sweeps"),
        "tuned": dict(entry("search"), note="the FCNN search's own pick (surrogate rounds + refinement)"),
        "speedup_vs_current_default": med["current_default"] / med["search"],
        "r2_train": rep["r2_train"], "r2_test": rep["r2_test"],
        "n_params": rep["n_params"], "space_size": rep["space_size"], "samples": args.tune_samples,
        "n_train": rep["n_train"], "n_test": rep["n_test"], "n_measured": rep["n_measured"],
        "n_exhaustive": rep["n_exhaustive"], "candidates_scored": args.tune_candidates, "epochs": rep["epochs"],
        "tuner_seconds": tuner_s, "returned": ("search", "current_default", "exhaustive_best")[rep["chosen"]],
        "replays": args.tune_replays, "steps_per_replay": args.tune_steps, "clocks": clk,
    }
    if "naive_default" in med:
        out["naive_default"] = dict(entry("naive_default"), note="32x8 threads, one cell per thread, one CTA per "
                                                                 "32x8 tile covering the domain")
        out["speedup_vs_naive_default"] = med["naive_default"] / med["search"]
    if "exhaustive_best" in med:
        out["exhaustive_best"] = dict(entry("exhaustive_best"),
                                      note="best of the reduced space: one tile and thread count for all stages, "
                                           "box tiles, TMA loads, default time-step kernel")
        out["vs_exhaustive"] = med["exhaustive_best"] / med["search"]
        if "naive_default" in med:
            out["speedup_exhaustive_vs_naive_default"] = med["naive_default"] / med["exhaustive_best"]
    return out


def other_workloads(args):
    """Short timed runs of the other configurations: 3D Taylor-Green 384^3 and
    the 96-grid batched Sod set (forward, like the main line, with their own
    clocks and CPU-oracle baselines) and the adjoint gradient (1024^2 vortex,
    400 steps, checkpoints every 20)."""
    out = {}
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "config", "roofline", "clocks",
            "cpu_baseline", "gpu_launches")
    for name in ("tgv384", "sod96", "adjoint1024"):
        a = argparse.Namespace(**vars(args))
        a.workload, a.n, a.launch, a.mode, a.workloads = name, N_CELLS_SIDE, None, "fused", False
        a.e2e_steps, a.cpu_seconds, a.tune_samples = 0, args.workload_cpu_seconds, 0
        if name == "adjoint1024":
            a.steps, a.warmup = 1, 1
            ln = run_adjoint(a)
            out[name] = {k: ln[k] for k in keep + ("adjoint",) if k in ln}
        else:
            a.steps, a.warmup = args.workload_steps, 3
            ln = run_ours(a)
            out[name] = {k: ln[k] for k in keep if k in ln}
    return out


def make_workload(args, I):
    """The benchmark workloads: the metric's KH 4096^2 (default), the 3D
    Taylor-Green 384^3 and the batched rotated-Sod set (96 grids)."""
    if args.workload == "kh4096":
        n = args.n
        g, U0 = I.kelvin_helmholtz(n, seed=1)
        return dict(name="kh4096", grid=g, U0=U0, cells=g.ncells, batched=False, flop=FLOP_PER_CELL_STAGE_2D,
                    data="synthetic (seeded Kelvin-Helmholtz initial condition)",
                    bytes=BYTES_PER_CELL_STAGE_2D, kernel="fvk::stage_kernel<2, stage>", launches_per_step=5,
                    metric=METRIC,
                    desc=f"2D Euler Kelvin-Helmholtz {n}x{n} periodic, FP64, MUSCL-minmod + Roe + SSP-RK3, CFL 0.5; "
                         f"1 bench step = 1 SSP-RK3 step (dt reduction + 3 fused stage kernels) replayed from a "
                         f"CUDA graph",
                    cpu_baseline=lambda: cpu_baseline(args, U0, g))
    if args.workload == "tgv384":
        n = 384 if args.n == N_CELLS_SIDE else args.n
        g, U0 = I.taylor_green(n, seed=2)
        return dict(name="tgv384", grid=g, U0=U0, cells=g.ncells, batched=False, flop=FLOP_PER_CELL_STAGE_3D,
                    data="synthetic (Taylor-Green vortex initial condition, seeded pressure noise)",
                    bytes=BYTES_PER_CELL_STAGE_3D, kernel="fvk::stage_kernel<3, stage>", launches_per_step=5,
                    metric=f"FP64 cell-updates/s per RK stage (3D Euler Taylor-Green {n}^3)",
                    desc=f"3D Euler Taylor-Green {n}^3 periodic, M=0.1, 1e-4 pressure noise, FP64, MUSCL-minmod + "
                         f"Roe + SSP-RK3, CFL 0.5; 1 bench step = 1 SSP-RK3 step replayed from a CUDA graph",
                    cpu_baseline=lambda: cpu_baseline_3d(args, U0, g))
    specs = I.batched_sod(96, seed=3)
    probs = [I.sod_rotated(nn, th) for nn, th in specs]
    grids = [p[0] for p in probs]
    cells = sum(gg.ncells for gg in grids)
    return dict(name="sod96", grid=grids, U0=None, states=[p[1] for p in probs], cells=cells, batched=True,
                data="synthetic (rotated Sod shock-tube initial conditions, seeded sizes and angles)",
                flop=FLOP_PER_CELL_STAGE_2D, bytes=BYTES_PER_CELL_STAGE_2D,
                kernel="fvk::batch_run_kernel (persistent, all steps)", launches_per_step=1,
                metric="FP64 cell-updates/s per RK stage (96 batched 2D Sod grids, 64^2..2048^2)",
                desc=f"96 rotated 2D Sod problems, sizes log-uniform in [64, 2048] (seed 3), {cells} cells, "
                     f"transmissive, FP64, per-problem CFL 0.5; all bench steps in one persistent cooperative "
                     f"launch under a CUDA graph",
                cpu_baseline=lambda: cpu_baseline_batch(args, probs))


def cpu_baseline_3d(args, U0, g):
    """The oracle on a z-slab of the 3D state (periodic in x, y; transmissive at
    the slab's z faces), ~10 s of CPU work."""
    from oracle import oracle as O
    from paper_2306_14011_gb300 import inputs as I
    nz = 32
    gb = I.GridSpec(3, (g.n[0], g.n[1], nz), (g.length[0], g.length[1], g.length[2] * nz / g.n[2]),
                    ((0, 0), (0, 0), (1, 1)))
    Ub = np.ascontiguousarray(U0[:, :nz])
    steps, t0 = 0, time.perf_counter()
    while True:
        Ub, _ = O.run(gb, Ub, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= args.cpu_seconds or steps >= 20:
            break
    return {"value": gb.ncells * 3 * steps / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{steps} SSP-RK3 step(s) of the C++ oracle on a {g.n[0]}x{g.n[1]}x{nz} slab ({el:.1f} s)"}


def cpu_baseline_batch(args, probs):
    """The oracle stepping the batch's problems one after another (smallest
    first) for ~10 s."""
    from oracle import oracle as O
    order = sorted(range(len(probs)), key=lambda i: probs[i][0].ncells)
    cells, t0, done = 0, time.perf_counter(), 0
    for i in order:
        g, U = probs[i]
        O.run(g, U, 1)
        cells += g.ncells
        done += 1
        if time.perf_counter() - t0 >= args.cpu_seconds:
            break
    el = time.perf_counter() - t0
    return {"value": cells * 3 / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"one SSP-RK3 step of the {done} smallest problems with the C++ oracle ({el:.1f} s)"}


def _band(U0, g, rows):
    """A band of `rows` rows of the workload state, periodic in x and
    transmissive at the band's y edges (same per-cell work as the full grid)."""
    from paper_2306_14011_gb300 import inputs as I
    n = g.n[0]
    y0 = (g.n[1] - rows) // 2
    gb = I.GridSpec(2, (n, rows, 1), (g.length[0], g.length[1] * rows / g.n[1], 1.0),
                    ((I.BC_PERIODIC, I.BC_PERIODIC), (I.BC_TRANSMISSIVE, I.BC_TRANSMISSIVE),
                     (I.BC_PERIODIC, I.BC_PERIODIC)))
    return gb, np.ascontiguousarray(U0[:, y0:y0 + rows, :])


def cpu_baseline(args, U0, g):
    """The oracle as it stands, on the host cores, for ~10-30 s of CPU work:
    SSP-RK3 steps of a 1024-row band of the workload."""
    from oracle import oracle as O
    gb, Ub = _band(U0, g, args.cpu_rows)
    steps, t0 = 0, time.perf_counter()
    while True:
        Ub, _ = O.run(gb, Ub, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= args.cpu_seconds or steps >= 50:
            break
    return {"value": gb.ncells * 3 * steps / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{steps} SSP-RK3 step(s) of the C++ oracle on a {gb.n[0]}x{gb.n[1]} band of the "
                      f"{g.n[0]}x{g.n[1]} KH state ({el:.1f} s)"}


def run_reference(args):
    """Reference arm: the CPU oracle, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2306_14011_gb300 import inputs as I
    g, U0 = I.kelvin_helmholtz(args.n, seed=1)
    gb, Ub = _band(U0, g, args.ref_rows)
    for _ in range(args.warmup):
        Ub, _ = O.run(gb, Ub, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Ub, _ = O.run(gb, Ub, 1)
    el = time.perf_counter() - t0
    value = gb.ncells * 3 * args.steps / el
    sample = (f"each step: one SSP-RK3 step of the C++ oracle on a {gb.n[0]}x{gb.n[1]} band of the "
              f"{g.n[0]}x{g.n[1]} KH state")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Kelvin-Helmholtz initial condition)",
        "config": {"workload": f"2D Euler Kelvin-Helmholtz {g.n[0]}x{g.n[1]} periodic, FP64 (CPU oracle, "
                               f"{gb.n[1]}-row band per step)", "cells": gb.ncells},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_adjoint(args):
    """Discrete-adjoint workload: the gradient of the kinetic energy after 400
    fixed-dt SSP-RK3 steps of the 1024^2 periodic isentropic vortex with
    respect to the initial state, through FvRunFunction with checkpoints every
    20 steps (forward with checkpoints; per segment, recompute and 20 RK-step
    VJPs).  One bench step = one whole gradient; value = differentiated
    cell-stages per second (cells x 3 x 400 / gradient time).  Also times one
    residual VJP, one RK-step VJP and one RK step alone (CUDA events)."""
    import torch

    from paper_2306_14011_gb300 import fv
    from paper_2306_14011_gb300 import inputs as I
    from paper_2306_14011_gb300.autograd import FvRunFunction, kinetic_energy

    dist, rank, world = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    n, nsteps, every = (args.n if args.n != N_CELLS_SIDE else 1024), 400, 20
    g, U0 = I.isentropic_vortex(n, noise=0.0)
    solver = fv.Solver(g, stream=stream)
    Ud = torch.from_numpy(U0).to(dev)
    dt = solver.time_step(Ud)

    def gradient():
        X = Ud.clone().requires_grad_()
        kinetic_energy(FvRunFunction.apply(X, solver, nsteps, dt, every), g).backward()
        return X.grad

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        gradient()
    barrier()
    clocks = ClockSampler(gpu_uuid(torch))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        gradient()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    solver.sync()

    def timed(f, reps=10):
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            f()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    lam = torch.randn_like(Ud)
    out = torch.empty_like(Ud)
    R = torch.empty_like(Ud)
    X = Ud.clone()
    t_res = timed(lambda: solver.residual(Ud, R))
    t_rvjp = timed(lambda: solver.residual_vjp(Ud, lam, out))
    t_step = timed(lambda: solver.rk_step(X, dt))
    t_svjp = timed(lambda: solver.rk_step_vjp(Ud, lam, dt, out))
    solver.close()
    if rank != 0:
        return None
    cells = g.ncells
    # kernels per gradient: forward 400 x 3 stage launches; backward, per
    # segment, 19 recomputed steps x 3 and 20 RK-step VJPs x (2 stage
    # recomputations + 3 adjoint launches)
    launches = nsteps * 3 + (nsteps // every) * ((every - 1) * 3 + every * 5)
    return {
        "metric": f"differentiated FP64 cell-stages/s (gradient of the kinetic energy after {nsteps} SSP-RK3 steps, "
                  f"2D Euler vortex {n}^2, checkpoints every {every})",
        "value": whole_job_rate(cells * 3 * nsteps * args.steps, world, ms / 1e3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (isentropic vortex initial condition)",
        "config": {"workload": f"gradient of J = kinetic energy after {nsteps} fixed-dt SSP-RK3 steps of the {n}x{n} "
                               f"periodic isentropic vortex w.r.t. U0; FvRunFunction, checkpoints every {every}; "
                               "1 bench step = 1 gradient", "cells": cells, "launch": "default",
                   "parallelism": f"replicas x{world}"},
        "roofline": None,
        "adjoint": {"residual_ms": t_res, "residual_vjp_ms": t_rvjp, "rk_step_ms": t_step, "rk_step_vjp_ms": t_svjp,
                    "vjp_over_residual": t_rvjp / t_res, "step_vjp_over_step": t_svjp / t_step,
                    "gradient_over_forward_run": (ms / args.steps) / (nsteps * t_step)},
        "e2e": None,
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "impl": "ours",
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=N_CELLS_SIDE, help="grid cells per side (default: the workload's 4096)")
    ap.add_argument("--workload", choices=("kh4096", "tgv384", "sod96", "adjoint1024"), default="kh4096",
                    help="kh4096: the metric's configuration (default); tgv384: 3D Taylor-Green; "
                         "sod96: 96 batched Sod grids; adjoint1024: gradient through 400 steps (one bench step "
                         "= one gradient)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-rows", type=int, default=1024)
    ap.add_argument("--ref-rows", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=("fused", "split"), default="fused",
                    help="kernel structure: fused (one kernel per RK stage) or split (the paper's per-stage kernels)")
    ap.add_argument("--launch", default=None,
                    help="TILE:THREADS[:march] for all three RK stages (e.g. 32x8:256) instead of the default launch")
    ap.add_argument("--tune-samples", type=int, default=300,
                    help="random launches the autotuner times for the tuned comparison (0: no tuned object)")
    ap.add_argument("--tune-candidates", type=int, default=1000000,
                    help="random launches the trained network scores")
    ap.add_argument("--tune-replays", type=int, default=7)
    ap.add_argument("--tune-steps", type=int, default=5)
    ap.add_argument("--no-workloads", dest="workloads", action="store_false",
                    help="skip the short runs of the other configurations")
    ap.add_argument("--workload-steps", type=int, default=5)
    ap.add_argument("--workload-cpu-seconds", type=float, default=5.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "adjoint1024":
        line = run_adjoint(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
