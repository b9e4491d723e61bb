#!/usr/bin/env python
"""Benchmark of the FLD radiation-energy update on GB300.

Workload (default): the 512^3 periodic lognormal-density grid with Kramers opacity,
dt = 100x the explicit limit, one full update per step (coefficients, multigrid
diffusion to 1e-8 relative residual, exchange).  `value` is the mixed-precision
solver (FP32 V-cycles inside the FP64 defect-correction loop); the plain FP64 GPU
solver on the same inputs and accuracy is reported beside it, with the error of the
mixed result against it.  Inputs (1 GiB per field) are larger than L2 (129 MB), so no
explicit flush is needed between steps.

One JSON line on rank 0.  `--impl reference` times the plain CPU oracle instead.
Multi-GPU: replicas only (one independent grid per GPU, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "implicit FLD cell-updates/s at 1e-8 residual (FP64 vs mixed); % HBM peak"
UNIT = "cell-updates/s"

# Per-kernel roofline model, per cell of the launch's level.  HBM-bound kernels: algorithmic
# (minimum) bytes.  FP64-bound kernels: the FP64 operations the formula needs (an FMA counts as
# 2, a reciprocal or square root as 1), compared with the nominal FP64 rate.
FP64_PEAK_GFLOPS = 1250.0  # GB300 nominal dense FP64 (1.25 TFLOP/s)
KERNEL_MODEL = {
    # one colour of a red-black sweep on the finest level: the colour's r and x (write), the other
    # colour's x, the 3 face arrays (the FP32 sweep rebuilds 1/diag from them; FP64 reads 1/diag)
    "smooth_L0": {"bound": "hbm", "bytes_f32": 3 * 0.5 * 4 + 3 * 4, "bytes_f64": 4 * 0.5 * 8 + 3 * 8},
    "smooth_L0_zero": {"bound": "hbm", "bytes_f32": 3 * 0.5 * 4, "bytes_f64": 3 * 0.5 * 8},
    # one full red-black sweep in one pass (wavefront): r, 3 faces, x in, x out (the FP64 sweep
    # also reads 1/diag); from x = 0 the first colour reads 1/diag instead of x; the last sweep of a
    # cycle also updates the FP64 iterate (read + write 16 B)
    "wave_L0": {"bound": "hbm", "bytes_f32": 4 + 12 + 4 + 4, "bytes_f64": 8 + 24 + 8 + 8 + 8},
    "wave_L0_zero": {"bound": "hbm", "bytes_f32": 4 + 12 + 2 + 4, "bytes_f64": 8 + 24 + 8 + 8},
    "wave_L0_update": {"bound": "hbm", "bytes_f32": 4 + 12 + 4 + 4 + 16, "bytes_f64": 8 + 24 + 8 + 8 + 8 + 16},
    # the tiled sweep of the mixed solver's finest 3-D level: r, the cell coefficient dc and x in,
    # x out (16 B); from x = 0 no x in (12 B); the last sweep of a cycle also updates the FP64 iterate
    "sweep_L0": {"bound": "hbm", "bytes_f32": 4 + 4 + 4 + 4, "bytes_f64": None},
    "sweep_L0_zero": {"bound": "hbm", "bytes_f32": 4 + 4 + 4, "bytes_f64": None},
    "sweep_L0_update": {"bound": "hbm", "bytes_f32": 4 + 4 + 4 + 4 + 16, "bytes_f64": None},
    "restrict_L0": {"bound": "hbm", "bytes_f32": 2 * 4 + 3 * 4 + 4 / 8, "bytes_f64": 2 * 8 + 3 * 8 + 8 / 8},
    "prolong_L0": {"bound": "hbm", "bytes_f32": 2 * 4 + 4 / 8, "bytes_f64": 2 * 8 + 8 / 8},
    # first outer residual.  Mixed: one double-float pass that also builds the diagonal: weights hi
    # and lo (24), E_old (8; the step solves in place, so no copy into the FP64 iterate), diagonal
    # hi and lo and 1/diag (12), r hi and lo (8).  FP64: r = b - d x + sum_6 w x_nb from w (24), x,
    # b, diag (24), r (8)
    "residual": {"bound": "hbm", "bytes_f32": 24 + 8 + 12 + 8, "bytes_f64": 24 + 24 + 8},
    # mixed solver's double-float residual update r -= A d and x += d: d (4, neighbours from cache),
    # r hi/lo in and out (16), weights hi and lo (24), diagonal hi and lo (8), the FP64 iterate (16)
    "residual_update": {"bound": "hbm", "bytes_f32": 4 + 16 + 24 + 8 + 16, "bytes_f64": 4 + 16 + 24 + 8 + 16},
    # E, rho, eps in; kappa and D out (double-float arithmetic on the FP32 pipe: issue-bound, far
    # below this bound)
    "coeffs": {"bound": "hbm", "bytes_f32": 40, "bytes_f64": 40},
    # D in; weights out (mixed: hi and lo floats and the tiled sweep's cell coefficient; FP64:
    # doubles and their FP32 copies)
    "faces": {"bound": "hbm", "bytes_f32": 8 + 24 + 4, "bytes_f64": 8 + 24 + 12},
    # rho, kappa, eps, E in; eps, E out (double-float, issue-bound like coeffs)
    "exchange": {"bound": "hbm", "bytes_f32": 48, "bytes_f64": 48},
    # FP64 operator set-up: weights (24) and E_old (8) in; b, diag (16), 1/diag and diag hi/lo (12) out
    "fine_setup": {"bound": "hbm", "bytes_f32": 24 + 8 + 16 + 12, "bytes_f64": 24 + 8 + 16 + 16},
}


GOLDEN_DT = os.path.join(ROOT, "tests", "golden", "explicit_dt.json")


def stored_dt(key):
    """Explicit diffusion limit of a full-size recipe's initial state, written by the oracle
    (tests/golden/make_explicit_dt.py): the workloads' dt is a multiple of it."""
    with open(GOLDEN_DT) as f:
        table = json.load(f)
    if key not in table:
        raise SystemExit(f"no stored explicit limit for {key}; run tests/golden/make_explicit_dt.py")
    return table[key]


def host_cpu():
    """CPU model and the cores this process may use."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:  # Arm hosts list no model name in /proc/cpuinfo; lscpu decodes the part number
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.strip().lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
            else os.cpu_count()}


def load_traffic(n: int, precision: str) -> dict:
    """DRAM bytes per launch of each traced scope at n^3, from single-kernel ncu captures
    (profiles/traffic.json; a scope's own captured_n, else the file's) scaled by the cells a launch
    processes.  A scope whose kernel changed since its capture is absent there, so its traffic is
    reported as null."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return {}
    if t.get("precision") != precision:
        return {}
    return {k: v["dram_bytes_per_launch"] * (n / v.get("captured_n", t["captured_n"])) ** 3
            for k, v in t.get("scopes", {}).items()}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, one sample every `interval_ms`, each stamped with
    the host's monotonic clock when it arrives.  The sampler starts before the warm-up (nvidia-smi
    takes a few hundred ms to deliver its first line), and `window()` brackets the timed region:
    the summary covers the samples that arrived inside it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device: int, interval_ms: int = 50):
        self.device = device
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []  # (monotonic seconds, line)
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.interval_ms), "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def begin(self):
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        # two intervals, so that the first sample after a window shorter than one has arrived
        time.sleep(2 * self.interval_ms * 1e-3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summary(self.lines, self.t0, self.t1, self.interval_ms)

    @classmethod
    def summary(cls, lines, t0, t1, interval_ms) -> dict:
        """Median SM clock, maximum clock and the throttle reasons seen, over the samples that
        arrived in [t0, t1]; when the window is shorter than one interval and holds none, over the
        first sample after t0 (`"window": "next sample"`)."""
        rows = []
        for t, ln in lines:
            parts = [q.strip() for q in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        lo = t0 if t0 is not None else -math.inf
        hi = t1 if t1 is not None else math.inf
        inside = [r for r in rows if lo <= r[0] <= hi]
        note = "timed region"
        if not inside:
            later = [r for r in rows if r[0] >= lo]
            inside, note = later[:1], "next sample"
        sm = sorted(r[1] for r in inside)
        reasons = sorted({nm for r in inside for nm, v in zip(cls.REASONS, r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": inside[-1][2] if inside else None,
                "reasons": reasons, "samples": len(sm), "interval_ms": interval_ms, "window": note}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, cells_per_rank: int, steps: int, local_ms: float):
    """Replicas: every rank advances its own grid.  The job's time is the slowest rank's; the
    job's throughput is all ranks' cell-updates over it.  Returns (max_ms, cell-updates/s)."""
    ms = allreduce_max(world, local_ms)
    return ms, world * cells_per_rank * steps / (ms * 1e-3)


# ----------------------------------------------------------------------------- oracle leg

def oracle_sample(n: int, steps: int, rtol: float):
    """The CPU oracle on the same recipe at n^3 (a bounded sample of the workload)."""
    import oracle
    from paper_2104_03968_gb300 import inputs
    case = inputs.lognormal_3d(n=n, seed=2)
    g, p = case["grid"], case["phys"]
    # dt = 100x the explicit limit of this sample's initial state (the oracle's limited D)
    D0 = oracle.coeffs(g, p, case["E"], case["rho"], oracle.opacity(p, case["rho"], case["eps"]))
    inputs.with_explicit_dt(case, inputs.explicit_dt(D0, 1.0, 3))
    del D0
    eps, E = case["eps"], case["E"]
    t0 = time.perf_counter()
    for _ in range(steps):
        eps, E, _ = oracle.step(g, p, case["dt"], case["rho"], eps, E, rtol=rtol)
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt, dt


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    n = args.oracle_n
    for _ in range(args.warmup):
        oracle_sample(n, 1, args.rtol)
    val, secs = oracle_sample(n, args.steps, args.rtol)
    sample = f"lognormal {n}^3 (same recipe as the {args.n}^3 workload), {args.steps} steps, rtol {args.rtol:g}"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_cpu()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, nu=None):
    """nu: the (nu1, nu2) the library's autotuner chose (reported by the solve), if known."""
    cfg = {"workload": f"lognormal-density Kramers-opacity periodic grid {args.n}^3, dt = 100x the explicit limit "
                       f"min(dx^2/(2 d D_cell)) with the initial state's Levermore-Pomraning D_cell, "
                       f"full FLD step (coeffs + multigrid diffusion to {args.rtol:g} + exchange)",
           "grid": [args.n] * 3, "cells": args.n ** 3, "rtol": args.rtol, "precision": args.precision,
           "multigrid": "FMG first cycle, V-cycles after; red-black Gauss-Seidel sweep counts autotuned",
           "l2_flush": "inputs larger than L2 (1 GiB per field)", "parallelism": "replicas"}
    if nu is not None:
        cfg["nu1"], cfg["nu2"], cfg["nu1_coarse"], cfg["nu2_coarse"] = nu
    return cfg


# ----------------------------------------------------------------------------- GPU leg

def timed_steps(torch, fld, ctx, g, p, dt, rho, eps, E, steps, trace=False):
    """`steps` full updates on the device, timed with CUDA events on torch's current stream (the
    library's stream).  Untraced, the steps are enqueued back to back (each one's outcome arrives
    in its Info in stream order) and checked after the final synchronisation.  Traced, every
    kernel is bracketed by events (the host-driven solve, which waits on the stream per cycle):
    the per-kernel device times for the roofline."""
    stream = torch.cuda.current_stream()
    if trace:
        # finest-level and per-step kernels only: the coarse levels' small launches are where the
        # event records would cost host time
        fld.trace_enable(ctx, True, major_only=True)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    pending = [fld.step(ctx, g, p, dt, rho, eps, E, sync=False) for _ in range(steps)]
    t1.record(stream)
    torch.cuda.synchronize()
    infos = [fld.outcome(ctx, i, allow_unconverged=False) for i in pending]
    rep = None
    if trace:
        fld.trace_enable(ctx, False)
        rep = fld.trace_report(ctx)
    return t0.elapsed_time(t1), infos, rep


def roofline(rep: dict, ncell: int, precision: str, peaks: dict, traffic: dict, bound=None):
    """Roofline of the modelled kernel with the largest traced time (restricted to one bound
    when `bound` is given): algorithmic bytes or FP64 flops per launch over its mean launch time."""
    if not rep:
        return None
    cands = [k for k in rep if k in KERNEL_MODEL and (bound is None or KERNEL_MODEL[k]["bound"] == bound)]
    if not cands:
        return None
    name = max(cands, key=lambda k: rep[k][1])
    launches, ms = rep[name]
    model = KERNEL_MODEL[name]
    avg_s = ms / launches * 1e-3
    out = {"kernel": name, "bound": model["bound"], "avg_launch_ms": ms / launches, "launches": launches,
           "share_of_traced_ms": ms / sum(v[1] for v in rep.values())}
    if model["bound"] == "hbm":
        per_cell = model["bytes_f32" if precision == "mixed" else "bytes_f64"]
        achieved = per_cell * ncell / avg_s / 1e9
        out.update({"achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "peak_source": peaks["source"] + " copy bandwidth", "traffic": traffic.get(name),
                    "algorithmic_bytes_per_launch": per_cell * ncell})
    else:
        achieved = model["flops"] * ncell / avg_s / 1e9
        out.update({"achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                    "frac": achieved / FP64_PEAK_GFLOPS, "peak_source": "nominal FP64 rate of GB300",
                    "traffic": traffic.get(name), "algorithmic_flops_per_launch": model["flops"] * ncell})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--nu1", type=int, default=0, help="finest pre-sweeps (0 with --nu2 0: autotuned)")
    ap.add_argument("--nu2", type=int, default=0, help="finest post-sweeps")
    ap.add_argument("--oracle-n", type=int, default=192, dest="oracle_n")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 2-D and column workloads")
    ap.add_argument("--workload", default="lognormal3d", choices=["lognormal3d", "batched2d", "columns"],
                    help="lognormal3d: the headline 512^3 grid; batched2d / columns: the batched workloads")
    ap.add_argument("--ngrids", type=int, default=512)
    ap.add_argument("--ncol", type=int, default=4096)
    args = ap.parse_args()
    if args.workload != "lognormal3d":
        return run_batched_workload(args)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    from paper_2104_03968_gb300 import build as _b
    if rank == 0:
        _b.build()
    barrier(world)
    from paper_2104_03968_gb300 import fld, inputs

    torch.cuda.set_device(local)
    ctx = fld.Context(local)
    case = inputs.lognormal_3d(n=args.n, seed=2, device=f"cuda:{local}",
                               dt_exp=stored_dt(f"lognormal_3d_{args.n}_seed2"))
    g, phys, dt = case["grid"], case["phys"], case["dt"]
    rho0, eps0, E0 = case["rho"], case["eps"], case["E"]
    ncell = args.n ** 3
    p = dict(phys, precision=args.precision, rtol=args.rtol)
    if args.nu1 or args.nu2:
        p.update(nu1=args.nu1, nu2=args.nu2)

    def fresh():
        return eps0.clone(), E0.clone()

    # ---- main arm: warm-up, then exactly K timed steps
    eps, E = fresh()
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        fld.step(ctx, g, p, dt, rho0, eps, E)
    barrier(world)
    torch.cuda.synchronize()
    n_before = fld.launch_count()
    clocks.begin()
    ms, infos, _ = timed_steps(torch, fld, ctx, g, p, dt, rho0, eps, E, args.steps)
    clocks.end()
    n_after = fld.launch_count()
    clk = clocks.stop()
    barrier(world)
    ms, value = replica_throughput(world, ncell, args.steps, ms)
    launches = (n_after - n_before) * world
    # the same number of steps again, traced kernel by kernel (outside the timed region)
    _, _, rep = timed_steps(torch, fld, ctx, g, p, dt, rho0, eps, E, args.steps, trace=True)
    traffic = load_traffic(args.n, args.precision)
    peaks = load_peaks()
    roof = roofline(rep, ncell, args.precision, peaks, traffic)
    roof_hbm = roofline(rep, ncell, args.precision, peaks, traffic, bound="hbm")

    # ---- same inputs, one step of each precision, to report the mixed error against FP64
    extra = {}
    if not args.no_fp64 and args.precision == "mixed":
        ctx64 = fld.Context(local)
        p64 = dict(phys, precision="fp64", rtol=args.rtol)
        e1, E1 = fresh()
        fld.step(ctx, g, p, dt, rho0, e1, E1)
        e2, E2 = fresh()
        fld.step(ctx64, g, p64, dt, rho0, e2, E2)
        dE = (E1 - E2)
        extra["mixed_vs_fp64"] = {"E_max_rel": float(dE.abs().max() / E2.abs().max()),
                                  "E_l2_rel": float(dE.norm() / E2.norm()),
                                  "eps_max_rel": float((e1 - e2).abs().max() / e2.abs().max())}
        del e1, E1, e2, E2, dE
        eps64, E64 = fresh()
        for _ in range(args.warmup):
            fld.step(ctx64, g, p64, dt, rho0, eps64, E64)
        barrier(world)
        ms64, infos64, _ = timed_steps(torch, fld, ctx64, g, p64, dt, rho0, eps64, E64, args.steps)
        ms64 = allreduce_max(world, ms64)
        extra["fp64"] = {"value": world * ncell * args.steps / (ms64 * 1e-3), "ms_per_step": ms64 / args.steps,
                         "cycles_per_step": [i["cycles"] for i in infos64]}
        del eps64, E64
        ctx64.close()

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hr = rho0.cpu().pin_memory()
        he = eps0.cpu().pin_memory()
        hE = E0.cpu().pin_memory()
        fld.step(ctx, g, p, dt, hr, he, hE)  # warm
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fld.step(ctx, g, p, dt, hr, he, hE)
        torch.cuda.synchronize()
        secs = allreduce_max(world, time.perf_counter() - t0)
        e2e = {"value": world * ncell * args.steps / secs, "unit": UNIT, "h2d_bytes_per_step": 3 * ncell * 8,
               "d2h_bytes_per_step": 2 * ncell * 8}

    # ---- the batched 2-D grids and the wind columns, mixed and FP64 (outside the headline's timing)
    secondary = {}
    if not args.no_batched:
        secondary = secondary_workloads(torch, np, fld, inputs, ctx, args, peaks)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        val, secs = oracle_sample(args.oracle_n, 1, args.rtol)
        cpu = {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full step of the same recipe at {args.oracle_n}^3 ({secs:.1f} s, single thread)",
               **host_cpu()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64+f32 (FP32 V-cycles; coefficients, weights, residuals and exchange in double-float "
                         "f32 pairs; FP64 iterate and norms)" if args.precision == "mixed"
                else "f64",
                "data": "synthetic", "config": workload_config(args, (infos[0]["nu1"], infos[0]["nu2"], infos[0]["nu1_coarse"],
                                                                 infos[0]["nu2_coarse"])), "roofline": roof,
                "roofline_hbm": roof_hbm, "cpu_baseline": cpu,
                "e2e": e2e, "clocks": clk, "gpu_launches": launches,
                "kernels_ms": {k: [v[0], round(v[1], 3)] for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1])},
                "cycles_per_step": [i["cycles"] for i in infos],
                "rel_residual": [i["rel_residual"] for i in infos], **extra, **secondary}
        print(json.dumps(line), flush=True)
    ctx.close()
    barrier(world)
    return 0


# ----------------------------------------------------------------------------- batched workloads

# Column step (one fused kernel per column): rho, eps, E in (24 B) and eps, E out (16 B) per cell.
COLUMN_BYTES = 40


def batched_inputs(torch, np, inputs, kind, ngrids, ncol):
    """Device inputs of a secondary workload: 512 uneven periodic 2-D grids or the wind columns."""
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    if kind == "batched2d":
        dtx = stored_dt("batched_2d_512_seed3")
        if ngrids > len(dtx):
            raise SystemExit(f"stored explicit limits cover {len(dtx)} batched grids")
        cases = inputs.batched_2d(ngrids=ngrids, seed=3, dt_exp=dtx)
        return {"kind": kind, "grids": [c["grid"] for c in cases], "phys": [c["phys"] for c in cases],
                "dts": [c["dt"] for c in cases], "rho": [dev(c["rho"]) for c in cases],
                "eps": [dev(c["eps"]) for c in cases], "E": [dev(c["E"]) for c in cases],
                "cells": sum(int(c["rho"].size) for c in cases),
                "desc": f"{ngrids} independent periodic 2-D grids, n log-uniform in [64, 512], kappa0 = 10^U(-2,4), "
                        f"dt = 10^U(1,3) x each grid's explicit limit, one graph launch per step"}
    dtx = stored_dt("wind_columns_4096x2048_seed4")
    if ncol > len(dtx):
        raise SystemExit(f"stored explicit limits cover {len(dtx)} columns")
    case = inputs.wind_columns(ncol=ncol, ncell=2048, seed=4, dt_exp=dtx[:ncol])
    return {"kind": kind, "phys": case["phys"], "bc": tuple(case["bc"]), "rf": dev(case["r_faces"]),
            "vlo": dev(case["bc_lo"]), "vhi": dev(case["bc_hi"]), "dt": dev(case["dt"]), "rho": dev(case["rho"]),
            "eps": dev(case["eps"]), "E": dev(case["E"]), "cells": int(case["rho"].size),
            "desc": f"{ncol} spherical wind-like columns x 2048 cells, r = 1..100 R*, tabulated opacity, "
                    f"dt = 100x each column's explicit limit, direct tridiagonal diffusion + exchange"}


def time_batched(torch, fld, ctx, W, precision, rtol, steps, warmup, peaks):
    """Warm-up, then `steps` timed steps of a secondary workload from its initial state, with the
    device time of the library's traced scopes."""
    if W["kind"] == "batched2d":
        params = [dict(p, precision=precision, rtol=rtol) for p in W["phys"]]
        eps = [t.clone() for t in W["eps"]]
        E = [t.clone() for t in W["E"]]

        def step():
            return fld.step_batched(ctx, W["grids"], params, W["dts"], W["rho"], eps, E)
    else:
        p = dict(W["phys"], precision=precision)
        eps, E = W["eps"].clone(), W["E"].clone()

        def step():
            return [fld.columns_step(ctx, W["rf"], "spherical", W["bc"], W["vlo"], W["vhi"], p, W["dt"], W["rho"],
                                     eps, E)]
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    fld.trace_enable(ctx, True)
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    n0 = fld.launch_count()
    t0.record(stream)
    per_step = []
    for _ in range(steps):
        per_step.append(step())
    t1.record(stream)
    torch.cuda.synchronize()
    n1 = fld.launch_count()
    fld.trace_enable(ctx, False)
    rep = fld.trace_report(ctx)
    ms = t0.elapsed_time(t1)
    out = {"value": W["cells"] * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "gpu_launches": n1 - n0, "status": sorted({i["status"] for infos in per_step for i in infos}),
           "kernels_ms": {k: [v[0], round(v[1], 3)] for k, v in rep.items()}}
    if W["kind"] == "batched2d":
        out["max_cycles_per_step"] = [max(i["cycles"] for i in infos) for infos in per_step]
        out["mean_cycles_per_step"] = [sum(i["cycles"] for i in infos) / len(infos) for infos in per_step]
    else:
        name = "columns_mixed" if precision == "mixed" else "columns"
        if name in rep:
            launches, kms = rep[name]
            achieved = COLUMN_BYTES * W["cells"] / (kms / launches * 1e-3) / 1e9
            out["roofline"] = {"kernel": "k_columns", "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                               "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                               "peak_source": peaks["source"] + " copy bandwidth", "traffic": None,
                               "algorithmic_bytes_per_launch": COLUMN_BYTES * W["cells"],
                               "note": "one fused kernel per step (coefficients, tridiagonal solve, exchange); "
                                       "bound by FP64 arithmetic, not by HBM"}
    return out


def secondary_workloads(torch, np, fld, inputs, ctx, args, peaks):
    """The batched 2-D grids and the wind columns, mixed and FP64, for the headline line."""
    out = {}
    for kind in ("batched2d", "columns"):
        W = batched_inputs(torch, np, inputs, kind, args.ngrids, args.ncol)
        res = {"config": {"workload": W["desc"], "cells": W["cells"], "rtol": args.rtol}}
        for prec in ("mixed", "fp64"):
            res[prec] = time_batched(torch, fld, ctx, W, prec, args.rtol, args.steps, args.warmup, peaks)
        res["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
        out[kind] = res
        del W
        torch.cuda.empty_cache()
    return out


def run_batched_workload(args):
    """A line of its own for one secondary workload and precision."""
    import numpy as np
    import torch

    from paper_2104_03968_gb300 import build as _b
    _b.build()
    from paper_2104_03968_gb300 import fld, inputs

    ctx = fld.Context(0)
    W = batched_inputs(torch, np, inputs, args.workload, args.ngrids, args.ncol)
    r = time_batched(torch, fld, ctx, W, args.precision, args.rtol, args.steps, args.warmup, load_peaks())
    line = {"metric": f"{args.workload} cell-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
            "config": {"workload": W["desc"], "cells": W["cells"], "rtol": args.rtol}, **r}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
