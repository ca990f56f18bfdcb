#!/usr/bin/env python
"""Benchmark of the space-time Vanka-multigrid FGMRES solver on GB300.

Workload (default): the 2D channel [0, 2.2] x [0, 0.41] with 704 x 128 quads and
four levels (88 x 16 coarse), Q2/P1disc, dG(1), nu = 1e-3, tau = 0.005, the
Newton Jacobian at a seeded smooth linearisation velocity, V(2,2) averaged
Vanka with omega = 0.7, FGMRES(30) to a relative residual of 1e-8.

One step = one linearised solve on data resident in HBM:
  stg_update_linearisation(w)  (assembly of every level, all local inverses
                                J_K^{-1}, coarse factorisation)
  stg_gmres_solve(b)           (FGMRES preconditioned by V-cycles)
The headline form stores J_K^{-1} and runs the V-cycle in FP32 with FGMRES,
residuals and the coarse solve in FP64; the all-FP64 form is measured on the
same inputs for the time-to-tolerance comparison.

value = Vanka-smoothed space-time DoFs per second over the whole job: the
DoFs smoothed by all V-cycles of a step (iterations x sum over levels >= 1 of
(nu1 + nu2) N_l) times steps times ranks, divided by the slowest rank's time.
With several GPUs each rank solves its own seeded replica (no collective on
the data path; weak scaling).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import stg_inputs as si  # noqa: E402

METRIC = "Vanka-smoothed space-time DoFs/s; FGMRES time-to-1e-8 (FP32/batched vs FP64)"
UNIT = "smoothed space-time DoF/s"
WORKLOAD = "channel704_k1"
CPU_SAMPLE_FACTOR = 2     # cpu_baseline: 352 x 64 channel, same four-level hierarchy
REF_STEP_FACTOR = 4       # --impl reference: 176 x 32 channel per step


def describe(cfg, spec) -> str:
    return (f"2D channel [0,2.2]x[0,0.41], {spec.n[0]}x{spec.n[1]} quads, {spec.n_levels} levels "
            f"(coarse {spec.cells(0)[0]}x{spec.cells(0)[1]}), Q2/P1disc, dG({cfg['k']}), Newton Jacobian at seeded "
            f"smooth w, nu={cfg['nu']}, tau={cfg['tau']}, inflow/walls Dirichlet (Nitsche), do-nothing outflow, "
            f"V({cfg['nu1']},{cfg['nu2']}) averaged Vanka omega=0.7, FGMRES(30) rtol 1e-8")


# ----------------------------------------------------------------------------- oracle (CPU)
def oracle_step_cli(factor: int, repeats: int) -> None:
    """Runs the oracle's full step on the channel scaled down by `factor` (child process)."""
    import numpy as np  # noqa: F401
    import oracle
    from oracle import fgmres

    cfg = si.WORKLOADS[WORKLOAD]
    spec = si.scaled(cfg["spec"], factor)
    times, its_all = [], []
    for r in range(repeats):
        w = si.channel_w(spec, cfg["k"], seed=si.BASE_SEED + r)
        t0 = time.perf_counter()
        h = oracle.Hierarchy(spec, cfg["k"], cfg["nu"], cfg["tau"], w, newton=cfg["newton"], nu1=cfg["nu1"],
                             nu2=cfg["nu2"])
        b = h.apply(si.reference_solution(spec, cfg["k"]))
        x, its, rel, ok = fgmres.fgmres(h.apply, h.vcycle, b)
        times.append(time.perf_counter() - t0)
        its_all.append(its)
    sm = si.smoothed_dofs_per_cycle(spec, cfg["k"], cfg["nu1"], cfg["nu2"])
    print(json.dumps({"times": times, "iters": its_all, "smoothed_per_cycle": sm, "cells": list(spec.n),
                      "n_dofs": si.n_dofs(2, spec.n, cfg["k"])}))


def _oracle_env() -> dict:
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def run_oracle(factor: int, repeats: int, timeout: float = 900.0) -> dict:
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-step", str(factor), str(repeats)],
                         capture_output=True, text=True, env=_oracle_env(), timeout=timeout, cwd=ROOT)
    if out.returncode:
        raise RuntimeError("oracle run failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def available_memory_bytes() -> int:
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_oracle_all_cores(factor: int, gb_per_process: float, timeout: float = 900.0) -> dict:
    """The unmodified oracle step on every host core at once: one single-threaded process per core
    (as many as the free memory holds), each solving the same sample; the rate is the smoothed DoFs
    of all processes over the wall time from the first start to the last finish."""
    cores = os.cpu_count() or 1
    procs = max(1, min(cores, int(available_memory_bytes() / (gb_per_process * 1e9)) or 1))
    t0 = time.perf_counter()
    ps = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-step", str(factor), "1"],
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=_oracle_env(), cwd=ROOT)
          for _ in range(procs)]
    outs = []
    for p in ps:
        so, se = p.communicate(timeout=timeout)
        if p.returncode:
            raise RuntimeError("oracle run failed: " + se[-2000:])
        outs.append(json.loads(so.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    dofs = sum(o["smoothed_per_cycle"] * sum(o["iters"]) for o in outs)
    return {"value": dofs / wall, "processes": procs, "host_cores": cores, "wall_s": wall, "cells": outs[0]["cells"],
            "n_dofs": outs[0]["n_dofs"]}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # the sampler's start-up (NVML initialisation) stays out of the timed region: wait for its
        # first sample (at most 3 s)
        t_end = time.perf_counter() + 3.0
        while self.proc and time.perf_counter() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- GPU arm
def dist_setup():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    # NCCL reduces device tensors; a gloo group (the CPU tests of this path) host tensors
    t = torch.tensor([value], dtype=torch.float64, device="cpu" if dist.get_backend() == "gloo" else "cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank_step: float, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units every rank processed in `steps` steps, divided by the
    slowest rank's time (ms)."""
    return units_per_rank_step * steps * world / (ms_max * 1e-3)


# DRAM bytes per patch (dram__bytes_read.sum + dram__bytes_write.sum, ncu) of the colour-kernel
# variants captured on the 352x64 copy of the workload (5632 patches per launch, factors larger
# than L2); the traffic of a full-size launch scales with its patch count.
# Keyed by (form, variant).
MEASURED_TRAFFIC_PER_PATCH = {("f32", 11): 43.10e6 / 5632, ("f32", 15): 43.11e6 / 5632, ("f32", 10): 43.11e6 / 5632,
                              ("bf16", 15): 22.93e6 / 5632, ("f64", 11): 85.46e6 / 5632}


def colour_kernel_name(variant: int) -> str:
    """Kernel behind a colour-kernel variant number of the library's autotuner (2D, k = 1, FP32)."""
    if variant >= 9:
        stages, rows = ((4, 1), (3, 1), (2, 1), (6, 1), (4, 2), (3, 2), (2, 2), (6, 2))[variant - 9]
        return (f"vanka_colour_bulk_kernel<float,float,{stages},{rows}> (finest level, bulk-copy staged, "
                f"{rows} row(s) per thread)")
    return (f"vanka_colour_kernel<float,float,2,{(4, 8, 16)[(variant // 3) % 3]}> "
            f"({128 << (variant % 3)} threads, finest level)")


def q2_block_couplings(cells: tuple) -> int:
    """Number of (node, node) blocks of the Q2 velocity operator: two Q2 nodes couple when they
    share a cell, which factorises over the directions (a vertex line couples with the nodes
    within two steps, a cell-interior line with those within one)."""
    total = 1
    for c in cells:
        m = 2 * c + 1
        total *= sum(min(i + (2 if i % 2 == 0 else 1), m - 1) - max(i - (2 if i % 2 == 0 else 1), 0) + 1
                     for i in range(m))
    return total


def sweep_bytes(dim: int, cells: tuple, k: int, form: str) -> dict:
    """Algorithmic bytes of one averaged Vanka sweep on a level (each array read or written once):
    the residual r = b - J x (operator + x, b read, r written), the colour kernels (every J_K^{-1}
    read, r gathered, z read and written per patch) and the update (d, z read and written)."""
    nt = k + 1
    ncell = int(np.prod(cells))
    n = nt * (3 ** dim * dim + dim + 1)
    N = si.n_dofs(dim, cells, k)
    nnzb = q2_block_couplings(cells)
    vs = 8 if form == "f64" else 4
    fs = {"f64": 8, "f32": 4, "bf16": 2}[form]
    vp = ncell * 3 ** dim * nt * dim * (dim + 1)           # velocity-pressure (and pressure-velocity) entries
    if form == "f64" or dim == 3 or k == 0:
        op = nnzb * (nt * dim) ** 2 * vs + 2 * vp * vs       # dense node blocks
    else:
        op = nnzb * 4 + nnzb * nt * dim * dim * 4 + 2 * vp * 4   # Kronecker split: M_ij + per-node blocks
    residual = op + 3 * N * vs
    colour = ncell * (n * n * fs + 3 * n * vs)
    update = 4 * N * vs
    return {"residual": residual, "colour": colour, "update": update, "total": residual + colour + update}


def time_ms(torch, stream, fn, reps: int = 1) -> float:
    """Device time of fn() (reps times) on `stream`, CUDA events, synchronised on both sides."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal


def colour_fraction(k: int, form: str, ms: float, launches: int, patches: int, peak: float,
                    variant: int | None = None) -> dict:
    """HBM fraction of the finest level's colour kernels (2D): algorithmic bytes (every J_K^{-1}
    in the form's factor precision, r gathered, z read and written) over their CUDA-event time."""
    n = 21 * (k + 1)
    fs = {"f64": 8, "f32": 4, "bf16": 2}[form]
    vs = 8 if form == "f64" else 4
    per_launch = n * (n * fs + 3 * vs) * patches / max(launches, 1)
    avg = ms / max(launches, 1)
    gbs = per_launch / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
    out = {"bytes_per_launch": per_launch, "avg_launch_ms": avg, "gbs": gbs, "frac": gbs / peak,
           "launches": launches}
    per_patch = MEASURED_TRAFFIC_PER_PATCH.get((form, variant))
    if per_patch and k == 1:
        out["traffic"] = per_patch * patches / max(launches, 1)
        out["traffic_source"] = f"ncu dram bytes of variant {variant} on the 352x64 case, scaled by patches"
    if form == "f64":
        # the FP64 form's product J_K^{-1} r runs in FP64 FMAs: 2 n_K^2 flops per patch against the
        # GB300's nominal FP64 rate (no measured FP64 peak is recorded)
        flops = 2.0 * n * n * patches / max(launches, 1)
        tflops = flops / (avg * 1e-3) / 1e12 if avg > 0 else 0.0
        out["fp64"] = {"tflops": tflops, "peak_nominal_tflops": FP64_NOMINAL_TFLOPS,
                       "frac": tflops / FP64_NOMINAL_TFLOPS}
    return out


def smoother_report(solver, spec, k, cfg, form: str, peak: float, torch, sweeps: int = 20) -> dict:
    """Sweep- and cycle-level smoothed DoF/s and the finest sweep's HBM fraction.
    One sweep (residual + colour kernels + update) is timed as the difference of stg_smooth with
    2 + sweeps and 2 sweeps on the finest level (the C-ABI conversions cancel); a V-cycle as the
    mean of `sweeps` stg_vcycle calls."""
    top = spec.n_levels - 1
    N = si.n_dofs(spec.dim, spec.n, k)
    b = torch.from_numpy(si.random_vector(N, 31)).cuda()
    x0 = torch.zeros_like(b)
    solver.smooth(top, 2, b, x0)
    t_lo = min(time_ms(torch, solver.stream, lambda: solver.smooth(top, 2, b, x0)) for _ in range(3))
    t_hi = min(time_ms(torch, solver.stream, lambda: solver.smooth(top, 2 + sweeps, b, x0)) for _ in range(3))
    t_sweep = (t_hi - t_lo) / sweeps
    by = sweep_bytes(spec.dim, spec.n, k, form)
    out = solver.vcycle(b)
    t_cycle = time_ms(torch, solver.stream, lambda: solver.vcycle(b, out=out), reps=sweeps) / sweeps
    per_cycle = si.smoothed_dofs_per_cycle(spec, k, cfg["nu1"], cfg["nu2"])
    achieved = by["total"] / (t_sweep * 1e-3) / 1e9
    return {"sweep_ms": t_sweep, "sweep_dofs_per_s": N / (t_sweep * 1e-3),
            "vcycle_ms": t_cycle, "cycle_dofs_per_s": per_cycle / (t_cycle * 1e-3),
            "sweep_bytes": by, "sweep_gbs": achieved, "sweep_hbm_frac": achieved / peak}


def timed_steps(solver, w, b, x, steps: int, torch) -> tuple:
    """Runs `steps` steps on the solver's stream; returns (ms, iterations of the last step)."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    its = 0
    torch.cuda.synchronize()
    ev0.record(solver.stream)
    for _ in range(steps):
        solver.update_linearisation(w)
        _, its, rel, ok = solver.gmres_solve(b, out=x)
        if not ok:
            raise RuntimeError(f"FGMRES did not converge (rel {rel:.2e})")
    ev1.record(solver.stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), its


def gpu_arm(args) -> None:
    import torch

    from paper_2210_02690_gb300 import Solver

    world, rank, local = dist_setup()
    cfg = si.WORKLOADS[WORKLOAD]
    spec, k = cfg["spec"], cfg["k"]
    if args.scale > 1 or args.levels:  # smaller copy of the workload, for profiler captures only
        spec = si.scaled(spec, args.scale, args.levels or None)
    seed = si.BASE_SEED + rank
    w_np = si.channel_w(spec, k, seed=seed)
    xs_np = si.reference_solution(spec, k, seed=seed + 1)
    opts = dict(nu1=cfg["nu1"], nu2=cfg["nu2"], linearisation="newton", overlap_launches=args.overlap)
    w = torch.from_numpy(w_np.ravel()).cuda()
    forms = {"f32": dict(vcycle_prec="f32", factor_prec="f32"), "f64": dict(vcycle_prec="f64", factor_prec="f64"),
             "bf16": dict(vcycle_prec="f32", factor_prec="bf16")}
    n_dofs = si.n_dofs(2, spec.n, k)
    per_cycle = si.smoothed_dofs_per_cycle(spec, k, cfg["nu1"], cfg["nu2"])
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6800.0)
    results = {}
    main = None
    for name in args.forms:
        solver = Solver(spec, k, cfg["nu"], cfg["tau"], w, **opts, **forms[name])
        b = solver.apply_jacobian(torch.from_numpy(xs_np).cuda())
        x = torch.zeros_like(b)
        # the project's autotuner picks the colour-kernel variant per level (untimed); a profiler
        # run replays the plain run's choice instead (timings under a profiler differ)
        if args.colour_variants:
            solver.set_colour_variants([int(v) for v in args.colour_variants[name].split(",")])
            tuned = (solver.colour_variants()[-1], None)
        else:
            tuned = solver.autotune()
        timed_steps(solver, w, b, x, args.warmup, torch)
        steps = args.steps if name == "f32" else max(3, args.steps // 2)
        solver.profile(True)
        if name == "f32":
            launches0 = solver.kernel_launches()
        barrier(world)
        with ClockSampler(local) as clk:
            # profiler range (a no-op without a profiler): `ncu --profile-from-start off` sees
            # exactly the timed steps of the headline form
            if name == "f32":
                torch.cuda.profiler.start()
            ms, its = timed_steps(solver, w, b, x, steps, torch)
            if name == "f32":
                torch.cuda.profiler.stop()
                launches1 = solver.kernel_launches()
        barrier(world)
        clocks = clk.summary()
        ms_max = max_over_ranks(world, ms)
        # split of one step: setup and solve alone
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(solver.stream)
        solver.update_linearisation(w)
        e[1].record(solver.stream)
        _, its_s, rel_s, _ = solver.gmres_solve(b, out=x)
        e[2].record(solver.stream)
        torch.cuda.synchronize()
        res = {"ms_per_step": ms_max / steps, "iters": its, "steps": steps, "setup_ms": e[0].elapsed_time(e[1]),
               "autotune": {"finest_variant": tuned[0], "finest_sweep_ms": tuned[1],
                            "variants": ",".join(str(v) for v in solver.colour_variants())},
               "time_to_tol_ms": e[1].elapsed_time(e[2]), "rel_res": rel_s, "clocks": clocks,
               "value": aggregate_rate(per_cycle * its, steps, world, ms_max)}
        pms, plaunch, ppatch = solver.profile_read()
        res["colour_kernel"] = (pms, plaunch, ppatch)
        solver.profile(False)
        res["colour_kernel_frac"] = colour_fraction(k, name, pms, plaunch, ppatch, peak, tuned[0])
        if world == 1:
            res["smoother"] = smoother_report(solver, spec, k, cfg, name, peak, torch)
        if name == "f32":
            res["gpu_launches"] = launches1 - launches0
            # end to end through the public API: pinned host inputs, copies inside the timed region
            w_h = torch.from_numpy(w_np.ravel()).pin_memory()
            b_h = b.cpu().pin_memory()
            x_h = torch.empty_like(b_h).pin_memory()
            w_d, b_d = torch.empty_like(w), torch.empty_like(b)
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                w_d.copy_(w_h, non_blocking=True)
                b_d.copy_(b_h, non_blocking=True)
                solver.update_linearisation(w_d)
                solver.gmres_solve(b_d, out=x)
                x_h.copy_(x, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            e2e_ms = max_over_ranks(world, e0.elapsed_time(e1))
            res["e2e"] = {"value": aggregate_rate(per_cycle * its, steps, world, e2e_ms), "unit": UNIT,
                          "h2d_bytes_per_step": int(w_h.numel() * 8 + b_h.numel() * 8),
                          "d2h_bytes_per_step": int(x_h.numel() * 8),
                          "ms_per_step": e2e_ms / steps, "wall_s": time.perf_counter() - t0}
            main = solver
            results[name] = res
        else:
            results[name] = res
            solver.close()
    r32 = results["f32"]
    pms, plaunch, ppatch = r32["colour_kernel"]
    npatch = 21 * (k + 1)
    # algorithmic bytes of one colour-kernel launch: each patch streams its J_K^{-1}
    # (npatch^2 FP32 values), gathers npatch residual values and reads+writes npatch values of z
    bytes_per_patch = npatch * npatch * 4 + 3 * npatch * 4
    avg_ms = pms / max(plaunch, 1)
    per_launch_bytes = bytes_per_patch * ppatch / max(plaunch, 1)
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    variant = r32["autotune"]["finest_variant"]
    per_patch = MEASURED_TRAFFIC_PER_PATCH.get(("f32", variant))
    traffic = per_patch * ppatch / max(plaunch, 1) if per_patch else None
    roofline = {"bound": "hbm", "kernel": colour_kernel_name(variant),
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": "ncu dram bytes of the 352x64 case, scaled by patches"
                if per_patch else None,
                "bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms,
                "launches": plaunch, "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}
    if rank != 0:
        if main:
            main.close()
        return
    out = {
        "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world, "steps": r32["steps"],
        "warmup": args.warmup, "ms_per_step": r32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 factors + f32 V-cycle; f64 FGMRES/residuals/coarse solve",
        "data": "synthetic (seeded Poiseuille + curl perturbation w, N(0,1) x*, b = J x*)",
        "config": {"workload": f"{WORKLOAD}: " + describe(cfg, spec), "n_dofs": n_dofs,
                   "smoothed_dofs_per_vcycle": per_cycle, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (FP32 J_K^{-1} of the finest level: "
                         f"{spec.n[0] * spec.n[1] * npatch * npatch * 4 / 1e6:.0f} MB)",
                   "step": "update_linearisation (assembly + local inverses + coarse factorisation) + FGMRES to 1e-8",
                   "launch_overlap": bool(args.overlap)},
        "fgmres_iters": r32["iters"], "rel_res": r32["rel_res"], "setup_ms": r32["setup_ms"],
        "autotune": r32["autotune"],
        "time_to_tol_ms": r32["time_to_tol_ms"],
        "roofline": roofline, "e2e": r32["e2e"], "gpu_launches": r32["gpu_launches"], "clocks": r32["clocks"],
    }
    if "smoother" in r32:
        out["smoother"] = r32["smoother"]
    out["colour_kernel_frac"] = r32["colour_kernel_frac"]
    keys = ("value", "ms_per_step", "iters", "setup_ms", "time_to_tol_ms", "rel_res", "autotune",
            "colour_kernel_frac", "smoother")
    if "f64" in results:
        out["f64_form"] = {k_: results["f64"][k_] for k_ in keys if k_ in results["f64"]}
        out["speedup_time_to_tol_f32_vs_f64"] = results["f64"]["time_to_tol_ms"] / r32["time_to_tol_ms"]
        out["speedup_step_f32_vs_f64"] = results["f64"]["ms_per_step"] / r32["ms_per_step"]
    if "bf16" in results:
        out["bf16_factor_form"] = {k_: results["bf16"][k_] for k_ in keys if k_ in results["bf16"]}
    if main:
        main.close()
    if world == 1 and not args.no_cpu_baseline:
        o = run_oracle(CPU_SAMPLE_FACTOR, 1)
        t = sum(o["times"])
        out["cpu_baseline"] = {"value": o["smoothed_per_cycle"] * sum(o["iters"]) / t, "unit": UNIT, "cores": 1,
                               "kind": "oracle",
                               "sample": f"oracle full step (assembly, LAPACK local inverses, coarse LU, FGMRES to "
                                         f"1e-8) on the same channel at {o['cells'][0]}x{o['cells'][1]} quads "
                                         f"({o['n_dofs']} DoFs, 4 levels), 1 thread, {t:.1f} s"}
        a = run_oracle_all_cores(CPU_SAMPLE_FACTOR, 2.5)
        out["cpu_baseline"]["all_cores"] = {
            "value": a["value"], "unit": UNIT, "cores": a["processes"], "host_cores": a["host_cores"],
            "kind": "oracle",
            "sample": f"{a['processes']} single-threaded oracle processes at once, each the full step on the "
                      f"{a['cells'][0]}x{a['cells'][1]} channel; {a['wall_s']:.1f} s wall"}
    if world == 1 and not args.no_workloads:
        import torch
        out["square256"] = square256_report(peak, torch)
        out["cube48"] = cube48_report(peak, torch)
        out["order4"] = order4_report(peak, torch)
    if world == 1 and not args.no_workloads:
        out["obstacle_march"] = obstacle_march_report()
    if world == 1 and not args.no_warm_start:
        out["warm_start"] = warm_start_report()
    if world == 1 and not args.no_batch:
        out["batched"] = batch_report()
    print(json.dumps(out), flush=True)


FORMS = {"f32": dict(vcycle_prec="f32", factor_prec="f32"), "f64": dict(vcycle_prec="f64", factor_prec="f64"),
         "bf16": dict(vcycle_prec="f32", factor_prec="bf16")}


def workload_line(name: str, k: int, form: str, peak: float, torch, reps: int = 3) -> dict:
    """Set-up, FGMRES time-to-1e-8 and the smoother figures of one (workload, k, form)."""
    from paper_2210_02690_gb300 import Solver

    cfg = si.WORKLOADS[name]
    spec = cfg["spec"]
    w = torch.from_numpy(si.make_w(dict(cfg, k=k)).ravel()).cuda()
    s = Solver(spec, k, cfg["nu"], cfg["tau"], w, nu1=cfg["nu1"], nu2=cfg["nu2"],
               linearisation="newton" if cfg["newton"] else "oseen", **FORMS[form])
    b = s.apply_jacobian(torch.from_numpy(si.reference_solution(spec, k)).cuda())
    x = torch.zeros_like(b)
    variant, _ = s.autotune()
    s.update_linearisation(w)
    s.gmres_solve(b, out=x)
    t_setup = min(time_ms(torch, s.stream, lambda: s.update_linearisation(w)) for _ in range(reps))
    its = [0]

    def solve():
        _, its[0], rel, ok = s.gmres_solve(b, out=x)
        if not ok:
            raise RuntimeError(f"{name} k={k} {form}: FGMRES did not converge ({rel:.2e})")
    t_solve = min(time_ms(torch, s.stream, solve) for _ in range(reps))
    per_cycle = si.smoothed_dofs_per_cycle(spec, k, cfg["nu1"], cfg["nu2"])
    out = {"n_dofs": si.n_dofs(spec.dim, spec.n, k, spec.order), "setup_ms": t_setup, "time_to_tol_ms": t_solve,
           "iters": its[0], "finest_variant": variant,
           "value": per_cycle * its[0] / ((t_setup + t_solve) * 1e-3),
           "smoother": smoother_report(s, spec, k, cfg, form, peak, torch) if spec.order == 2 else None}
    s.close()
    return out


def square256_report(peak: float, torch) -> dict:
    """Unit square 256x256 (5 levels, 16x16 coarse), Oseen, k = 1..4 (patches of 42..105
    unknowns), local inverses in FP64, FP32 and BF16, outer FGMRES in FP64."""
    cfg = si.WORKLOADS["square256"]
    out = {"workload": "unit square 256x256 quads, 5 levels (coarse 16x16), Q2/P1disc, dG(k), Oseen at seeded "
                       f"Fourier w, nu={cfg['nu']}, tau={cfg['tau']}, Dirichlet on all faces, V(2,2), FGMRES to 1e-8"}
    for k in (1, 2, 3, 4):
        for form in ("f64", "f32", "bf16"):
            out[f"k{k}_{form}"] = workload_line("square256", k, form, peak, torch)
    return out


def order4_report(peak: float, torch) -> dict:
    """The paper's 2D element (Q4)^2 x P3disc (local systems of 60 (k+1) unknowns) on the channel,
    352x64 quads -> 44x8: FP64 and FP32 forms, k = 1, 2."""
    cfg = si.WORKLOADS["channel_q4"]
    spec = cfg["spec"]
    out = {"workload": f"channel [0,2.2]x[0,0.41], {spec.n[0]}x{spec.n[1]} quads, {spec.n_levels} levels, "
                       "(Q4)^2 x P3disc, Newton Jacobian at the seeded channel w, nu=1e-3, tau=0.005, V(2,2), "
                       "FGMRES to 1e-8"}
    for k in (1, 2):
        for form in ("f64", "f32"):
            out[f"k{k}_{form}"] = workload_line("channel_q4", k, form, peak, torch)
    return out


def cube48_report(peak: float, torch) -> dict:
    """Unit cube 48^3 (levels 6^3 .. 48^3), Oseen, dG(1) (170 x 170 local matrices), FP32 local
    inverses and V-cycle, FP64 outer FGMRES."""
    cfg = si.WORKLOADS["cube48_k1"]
    out = {"workload": "unit cube 48^3 hexes, 4 levels (coarse 6^3), Q2/P1disc, dG(1), Oseen at seeded "
                       f"divergence-free w, nu={cfg['nu']}, tau={cfg['tau']}, Dirichlet on all faces, V(2,2), "
                       "FGMRES to 1e-8"}
    out["k1_f32"] = workload_line("cube48_k1", 1, "f32", peak, torch)
    # robustness in the time degree (Sec. 4 runs dG(0..2) in 3D): the 32^3 cube keeps the k = 2
    # operators (9 x 9 FP64 node blocks) within memory
    for k in (0, 1, 2):
        out[f"cube32_k{k}_f32"] = workload_line("cube32", k, "f32", peak, torch)
    return out


def batch_report() -> dict:
    """64 uneven problems (rectangles of 32..256 square cells per side, k in {1, 2}) solved to 1e-8:
    batched FP32 form (one graph launch per FGMRES iteration for all problems) against the
    same problems solved one after another in the FP32 form and in the plain FP64 form."""
    import torch

    from paper_2210_02690_gb300 import Batch, Solver

    probs = si.batch_problems()

    def make(spec, k, sd, **form):
        w = torch.from_numpy(si.fourier_w(spec, k, seed=sd).ravel()).cuda()
        s = Solver(spec, k, 1e-3, 0.01, w, nu1=2, nu2=2, **form)
        b = s.apply_jacobian(torch.from_numpy(si.reference_solution(spec, k, seed=sd + 1)).cuda())
        return s, b

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    f32 = dict(vcycle_prec="f32", factor_prec="f32")
    pairs = [make(spec, k, sd, **f32) for spec, k, sd in probs]
    solvers, rhs = [p[0] for p in pairs], [p[1] for p in pairs]
    for s, b in pairs:  # warm-up
        s.gmres_solve(b)
    seq, t_seq = timed(lambda: [s.gmres_solve(b) for s, b in pairs])
    batch = Batch(solvers)
    batch.gmres_solve(rhs)
    (xs, its_b, rel_b, ok_b), t_batch = timed(lambda: batch.gmres_solve(rhs))
    batch.close()
    for s in solvers:
        s.close()
    t64, its64 = 0.0, []
    for spec, k, sd in probs:
        s, b = make(spec, k, sd)
        s.gmres_solve(b)
        (_, it, _, _), t = timed(lambda: s.gmres_solve(b))
        t64 += t
        its64.append(it)
        s.close()
    dofs = sum(si.n_dofs(2, spec.n, k) for spec, k, _ in probs)
    return {"workload": f"{len(probs)} rectangles of square cells, n_x, n_y in {{32..256}}, k in {{1, 2}}, "
                        f"{dofs} space-time DoFs in total; FGMRES to 1e-8 relative",
            "batched_f32_s": t_batch, "sequential_f32_s": t_seq, "sequential_f64_s": t64,
            "speedup_batched_vs_sequential_f32": t_seq / t_batch, "speedup_batched_f32_vs_plain_f64": t64 / t_batch,
            "iters_batched": [int(v) for v in its_b], "iters_f32": [int(r[1]) for r in seq],
            "iters_f64": its64, "all_converged": bool(ok_b)}


def obstacle_march_report(slabs: int | None = None) -> dict:
    """Newton time march on the channel with an obstacle (the structured stand-in for the flow
    around an obstacle of Sec. 4): from rest with the Poiseuille inflow switched on at t = 0,
    dG(k) for k = 0..4, FP32 form, the paper's absolute tolerances (Newton 1e-8, GMRES 1e-9).
    Reports the mean Newton steps per slab and GMRES iterations per Newton step (the statistics
    of Tables 3.1 and 3.2) and the drag and lift coefficients at the end of the march."""
    import torch
    from paper_2210_02690_gb300.march import March, summary

    cfg = si.OBSTACLE
    spec = cfg["spec"]
    n_slabs = cfg["slabs"] if slabs is None else slabs
    box = spec.obstacle_cells(0)
    h0 = ((spec.hi[0] - spec.lo[0]) / spec.cells(0)[0], (spec.hi[1] - spec.lo[1]) / spec.cells(0)[1])
    diameter = (box[3] - box[2]) * h0[1]
    u_mean = 2.0 * cfg["u_max"] / 3.0
    out = {"workload": f"channel [0,2.2]x[0,0.41], {spec.n[0]}x{spec.n[1]} quads, {spec.n_levels} levels, "
                       f"obstacle of {box[1] - box[0]}x{box[3] - box[2]} coarse cells around (0.2, 0.2) "
                       f"(D = {diameter:.4f}), nu = {cfg['nu']}, Poiseuille inflow U_max = {cfg['u_max']} "
                       f"(Re = U_mean D / nu = {u_mean * diameter / cfg['nu']:.0f}), tau = {cfg['tau']}, "
                       f"{n_slabs} slabs from rest; FP32 form; Newton 1e-8, GMRES 1e-9 absolute"}
    for k in range(5):
        m = March(spec, k, cfg["nu"], cfg["tau"], np.zeros(2 * np.prod([2 * c + 1 for c in spec.n])),
                  si.obstacle_inflow(spec, k, cfg["u_max"]), vcycle_prec="f32", factor_prec="f32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.run(n_slabs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        sm = summary(m.stats)
        F = m.solver.obstacle_forces(m.X[-1])
        c = 2.0 * F[-1] / (u_mean ** 2 * diameter)
        out[f"k{k}"] = {"dofs_per_slab": int(m.N), "mean_newton": sm["mean_newton"],
                        "mean_gmres_per_newton": sm["mean_gmres_per_newton"], "seconds": wall,
                        "c_drag_end": float(c[0]), "c_lift_end": float(c[1])}
        m.close()
    return out


def warm_start_report() -> dict:
    """Time march with the learned warm start (2D channel 128x32, dG(1), 400 slabs; network
    trained on slabs 1-200, every slab 201-400 solved from three guesses to the absolute
    tolerances of Sec. 4)."""
    from paper_2210_02690_gb300.march import March, summary

    cfg = si.MARCH
    spec, k = cfg["spec"], cfg["k"]
    t0 = time.perf_counter()
    m = March(spec, k, cfg["nu"], cfg["tau"], si.march_initial_velocity(spec, pert=cfg["pert"]),
              si.march_inflow(spec, k), vcycle_prec="f32", factor_prec="f32")
    m.run(cfg["slabs"])
    march_s = time.perf_counter() - t0
    net, sv, losses, train_s = m.train(cfg["channels"], si.cnn_init(cfg["channels"]),
                                       list(range(2, cfg["train_slabs"])))
    ev = m.evaluate(list(range(cfg["train_slabs"], cfg["slabs"])), net, sv)
    out = {"workload": f"channel {spec.n[0]}x{spec.n[1]} quads, dG({k}), tau {cfg['tau']}, {cfg['slabs']} slabs; "
                       f"network {cfg['channels']} trained on slabs 1-{cfg['train_slabs']}, evaluated on "
                       f"{cfg['train_slabs'] + 1}-{cfg['slabs']}",
           "tolerances": "Newton absolute 1e-8, GMRES absolute 1e-9 (Sec. 4), same for every guess",
           "march_s": march_s, "train_s": train_s, "train_steps": len(losses),
           "train_loss_first_median_last20": [float(losses[0]), float(np.median(losses[-20:]))]}
    for name, rows in ev.items():
        sm = summary(rows)
        out[name] = {key: sm[key] for key in ("newton_steps", "gmres_iters", "mean_r0", "seconds",
                                              "max_final_over_tol", "all_converged")}
    out["gmres_iters_saved_vs_fallback"] = 1.0 - out["network"]["gmres_iters"] / out["fallback"]["gmres_iters"]
    out["time_to_tol_speedup_vs_fallback"] = out["fallback"]["seconds"] / out["network"]["seconds"]
    keys = ("newton_steps", "gmres_iters", "mean_r0", "seconds", "max_final_over_tol", "all_converged")
    eval_slabs = list(range(cfg["train_slabs"], cfg["slabs"]))
    # the plain FP64 form (FP64 local inverses and V-cycle) from the fallback guess: the method
    # without reduced precision and without the learned part, on the same slabs and tolerances
    f64 = m.companion_solver(vcycle_prec="f64", factor_prec="f64")
    ev64 = m.evaluate(eval_slabs, net, sv, solver=f64, names=("fallback",))
    f64.close()
    out["plain_f64_fallback"] = {key: summary(ev64["fallback"])[key] for key in keys}
    out["time_to_tol_speedup_warm_f32_vs_plain_f64"] = out["plain_f64_fallback"]["seconds"] / out["network"]["seconds"]
    # a tighter regime in which the guesses differ in cost: Newton to 1e-10, GMRES to 1e-11 absolute
    tight = m.companion_solver(vcycle_prec="f32", factor_prec="f32", gmres_atol=1e-11)
    evt = m.evaluate(eval_slabs, net, sv, solver=tight, atol=1e-10)
    tight.close()
    out["tight"] = {"tolerances": "Newton absolute 1e-10, GMRES absolute 1e-11, FP32 form"}
    for name, rows in evt.items():
        out["tight"][name] = {key: summary(rows)[key] for key in keys}
    net.close()
    m.close()
    return out


def setup_profile(args) -> None:
    """One re-linearisation (assembly, local inverses, coarse factorisation) of a workload inside
    the profiler range (`ncu --profile-from-start off`), after an untimed one."""
    import torch

    from paper_2210_02690_gb300 import Solver

    cfg = si.WORKLOADS[args.setup_profile]
    spec = cfg["spec"]
    if args.scale > 1 or args.levels:
        spec = si.scaled(spec, args.scale, args.levels or None)
    k = cfg["k"] if args.k is None else args.k
    w = torch.from_numpy(si.make_w(dict(cfg, spec=spec, k=k)).ravel()).cuda()
    s = Solver(spec, k, cfg["nu"], cfg["tau"], w, nu1=cfg["nu1"], nu2=cfg["nu2"],
               linearisation="newton" if cfg["newton"] else "oseen", **FORMS["f32"])
    s.update_linearisation(w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record(s.stream)
    s.update_linearisation(w)
    e1.record(s.stream)
    torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.setup_profile, "cells": list(spec.n), "levels": spec.n_levels, "k": k,
                      "setup_ms": e0.elapsed_time(e1)}), flush=True)
    s.close()


def vcycle_profile(args) -> None:
    """One V-cycle of the headline channel (with --scale/--levels) in one precision form inside the
    profiler range (`ncu --profile-from-start off`), after three untimed ones; the colour-kernel
    variants of --colour-variants (that form's entry) replace the autotuner's choice."""
    import torch

    from paper_2210_02690_gb300 import Solver

    form = args.vcycle_profile
    cfg = si.WORKLOADS[WORKLOAD]
    spec = cfg["spec"]
    if args.scale > 1 or args.levels:
        spec = si.scaled(spec, args.scale, args.levels or None)
    k = cfg["k"]
    w = torch.from_numpy(si.channel_w(spec, k).ravel()).cuda()
    s = Solver(spec, k, cfg["nu"], cfg["tau"], w, nu1=cfg["nu1"], nu2=cfg["nu2"], linearisation="newton",
               **FORMS[form])
    if args.colour_variants:
        s.set_colour_variants([int(v) for v in args.colour_variants[form].split(",")])
    else:
        s.autotune()
    b = s.apply_jacobian(torch.from_numpy(si.reference_solution(spec, k)).cuda())
    for _ in range(3):
        s.vcycle(b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record(s.stream)
    s.vcycle(b)
    e1.record(s.stream)
    torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    print(json.dumps({"form": form, "cells": list(spec.n), "levels": spec.n_levels,
                      "variants": s.colour_variants(), "vcycle_ms": e0.elapsed_time(e1)}), flush=True)
    s.close()


# ----------------------------------------------------------------------------- reference arm
def reference_arm(args) -> None:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = si.WORKLOADS[WORKLOAD]
    o = run_oracle(REF_STEP_FACTOR, args.warmup + args.steps, timeout=3600)
    times = o["times"][args.warmup:]
    its = o["iters"][args.warmup:]
    t = sum(times)
    value = o["smoothed_per_cycle"] * sum(its) / t
    sample = (f"oracle full step on the same channel at {o['cells'][0]}x{o['cells'][1]} quads ({o['n_dofs']} DoFs, "
              f"4 levels) per step, 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: " + describe(cfg, cfg["spec"]), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--oracle-step":
        oracle_step_cli(int(sys.argv[2]), int(sys.argv[3]))
        return
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm-start report")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve report")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the lines of the 256x256 square (k = 1..4) and the 48^3 cube")
    ap.add_argument("--setup-profile", default=None, metavar="WORKLOAD",
                    help="profiler case: one untimed and one profiled re-linearisation (FP32 form) of a "
                         "workload of stg_inputs.WORKLOADS (with --scale/--levels), then exit")
    ap.add_argument("--k", type=int, default=None,
                    help="with --setup-profile: the time degree (default: the workload's)")
    ap.add_argument("--vcycle-profile", default=None, choices=["f32", "f64", "bf16"],
                    help="profiler case: one V-cycle of the headline channel (with --scale/--levels) in "
                         "this form inside the profiler range, after three untimed ones, then exit")
    ap.add_argument("--colour-variants", default=None, metavar="F32;F64;BF16",
                    help="skip the autotuner and set the colour-kernel variants of levels 1.. per form, "
                         "e.g. '11,11,11;4,4,4;11,11,11' (the 'variants' a plain run reports), for "
                         "profiler runs")
    ap.add_argument("--forms", default="f32,f64,bf16",
                    help="precision forms to time (f32, the headline, always runs; e.g. 'f32' for profiler runs)")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the finest mesh by this factor (small cases for profiler captures)")
    ap.add_argument("--overlap", type=int, choices=[0, 1], default=1,
                    help="overlap_launches of the headline workload's solvers (programmatic dependent "
                         "launch of the V-cycle kernels; 1 is the library default)")
    ap.add_argument("--levels", type=int, default=0,
                    help="with --scale: number of levels of the smaller copy (e.g. --scale 4 --levels 2 "
                         "keeps the 88x16 coarse level)")
    args = ap.parse_args()
    if args.colour_variants:
        parts = args.colour_variants.split(";")
        args.colour_variants = {"f32": parts[0], "f64": parts[min(1, len(parts) - 1)],
                                "bf16": parts[min(2, len(parts) - 1)]}
    args.forms = ["f32"] + [f for f in args.forms.split(",") if f in ("f64", "bf16")]
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.setup_profile:
        setup_profile(args)
    elif args.vcycle_profile:
        vcycle_profile(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
