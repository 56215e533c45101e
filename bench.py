"""Benchmark: cells/s per CFD time step for the batched finite-rate chemistry solve.

Workload (one "step"): one chem_integrate call over dt = 1e-5 s for the 256 x 256 (65 536
cells) shear-layer field of the 53-species / 325-reaction synthetic mechanism at 40 atm,
rtol 1e-6, atol 1e-10, cold start (every step starts from the same initial field, copied in
outside the timed region).

Reported: `value` = cells / (device time of the integrate call, CUDA events on the launching
stream) with the field resident in HBM; `e2e` = the same cells / (wall time of one
chem_integrate call through the C ABI with pinned HOST arrays: the library copies the field in,
integrates and copies it back inside the call); `roofline` = achieved FP64 FLOP/s of the integrate
kernel (algorithmic FLOPs from the oracle's per-step operation count, times the kernel's own
per-cell step counts) against the FP64 pipe peak; `cpu_baseline` = the CPU oracle on a bounded
sample of the same field on the host cores, and on one core.

Warm-up calls run on a slice of the field (one wave of cells, the same options and launch path);
one more untimed full-size call with a one-attempt step cap allocates the library's per-cell and
staging buffers before the timed region.  A wall-time budget (`--budget-s`) stops the timed loop
early, and says so in the line (`steps` < `steps_requested`), if the remaining steps cannot finish
in time.

`--impl reference` times the CPU oracle itself (the reference implementation of this repo's
method) on a bounded sample per step.

`--workload adjoint` times the differentiated solve instead: 16 384 cells of the igniting band
(53 species, T ~ U[1000, 1300] K, 20 atm, dt = 1e-4 s); one step = chem_integrate_record +
chem_adjoint for a random dL/dphi(dt), reporting the forward and backward times, their ratio
and the checkpoint memory.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

T_START = time.monotonic()
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cells/s per CFD Δt (53 sp, rtol 1e-6), batched/mixed vs plain FP64; % roofline"
L2_BYTES = 129 * 2 ** 20
OPCOUNT_FILE = os.path.join(ROOT, "tests", "golden", "opcount_mech53.json")
# FLOPs per operation.  Unit weights: add, mul, div, exp and log count one each (the conservative
# count, `roofline.frac`).  Weighted: an exp or log counts its cost in FMA flops, the measured FP64
# pipe throughput of the library exp and log relative to DFMA on GB300 (17 and 31 DFMA),
# reported beside it as `roofline.frac_weighted`.
UNIT_WEIGHTS = {"add": 1, "mul": 1, "div": 1, "exp": 1, "log": 1}
FLOP_WEIGHTS = {"add": 1, "mul": 1, "div": 1, "exp": 2 * 17, "log": 2 * 31}
# DRAM bytes (read + write) of the integrate kernel as a function of the cells of a launch,
# fitted to two ncu captures (dram__bytes_read.sum + dram__bytes_write.sum, the timed launch of
# `bench.py --cells n --dt 1e-9 --warmup 1 --steps 1`) of the current kernel on evenly spaced
# slices of the shear-layer field: 1 566 720 B read / 0 B written at 608 cells and 3 371 264 B /
# 0 B at 4864 cells, i.e. fixed bytes (mechanism tables, the CTAs' first touches) plus bytes per
# cell (its state; the rest of the state is read from L2, where the library's staging copy in
# the same call left it, and the results stay in L2 until the copy back).
TRAFFIC_FIT = {"fixed": 1566720 - 608 * (3371264 - 1566720) / (4864 - 608),
               "per_cell": (3371264 - 1566720) / (4864 - 608), "cells": (608, 4864)}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--precision", choices=["fp64", "mixed", "ff"], default="fp64",
                    help="linear solves: FP64, FP32 LU + FP64 refinement, or FP32-pair LU + FP64 refinement")
    ap.add_argument("--refine-sweeps", type=int, default=-1, help="refinement sweeps per stage solve (mixed, ff)")
    ap.add_argument("--solver", choices=["rosenbrock", "seulex"], default="rosenbrock",
                    help="integrator: the Rosenbrock method or the paper's Seulex")
    ap.add_argument("--cells", type=int, default=0, help="cells per rank (0 = the full field of the workload)")
    ap.add_argument("--warm-cells", type=int, default=608,
                    help="cells of each warm-up call (a slice of the field; 608 = 4 cells on each of 152 SMs)")
    ap.add_argument("--budget-s", type=float, default=1740.0,
                    help="wall-time budget of the whole run in seconds (the timed loop stops early if the rest "
                         "cannot finish inside it)")
    ap.add_argument("--dt", type=float, default=0.0, help="override the CFD time step (profiling small cases)")
    ap.add_argument("--workload", choices=["shear", "uneven", "adjoint", "0d"], default="shear",
                    help="shear: 53-species shear layer (the headline); uneven: 100-species igniting/cold/burnt field")
    ap.add_argument("--order", choices=["shuffled", "blocked"], default="blocked", help="cell order of --workload uneven")
    ap.add_argument("--batch-cells", type=int, default=0,
                    help="also time one launch per batch of this many cells (static assignment) against the queue")
    ap.add_argument("--autotune", action="store_true", help="pick warps/cell and cells/CTA with the autotuner first")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rtol", type=float, default=0.0, help="override the workload's rtol (work-precision runs)")
    ap.add_argument("--accuracy-sample", type=int, default=0,
                    help="error of the timed result on this many evenly spaced cells against a converged FP64 "
                         "solve of the same cells (Rosenbrock at rtol 1e-10, atol 1e-14)")
    ap.add_argument("--map", action="store_true",
                    help="shear layer: zonal reference-cell mapping of the cells within 1e-9 of an unmixed "
                         "stream (chem_integrate_mapped), timed against the plain solve")
    ap.add_argument("--vs-fp64", action="store_true",
                    help="also run the plain FP64 Rosenbrock path once (untimed result, timed call) and report "
                         "the speed ratio and the largest deviation of T and Y from it")
    ap.add_argument("--warm-start", action="store_true",
                    help="also time the next CFD step: from the state at dt, with the carried-over sub-step h")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle's all-core sample")
    return ap.parse_args(argv)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------------------------------
# CPU legs: the oracle (plain FP64 C++, one cell per thread at a time) on bounded samples

def _oracle_seconds(ora, w, idx, nthreads):
    T, Y = w["T"][idx], w["Y"][:, idx]
    t0 = time.perf_counter()
    ora.integrate(w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], nthreads=nthreads)
    return time.perf_counter() - t0


def sample_sizes(rate_all: float, cores: int, target_s: float, n_field: int):
    """All-core sample of about target_s seconds (a multiple of the core count, at least one cell
    per core, at most the field) and a single-core sample of about target_s / 2 seconds
    (2..64 cells), from a measured all-core rate in cells/s."""
    n_all = int(rate_all * target_s) // cores * cores
    n_all = max(cores, min(n_all, n_field))
    n_one = int(rate_all / cores * target_s / 2)
    n_one = max(2, min(n_one, 64, n_field))
    return n_all, n_one


def cpu_baseline(w, target_s: float = 15.0):
    """The CPU oracle on bounded, evenly spaced samples of the field: all host cores (threads over
    cells), and one core (labelled; the rate of a single-threaded solve)."""
    import oracle
    cores = os.cpu_count() or 1
    ora = oracle.OracleMechanism(w["mech"].write_temp())
    n = w["T"].shape[0]
    probe = np.linspace(0, n - 1, cores).astype(np.int64)
    rate0 = cores / _oracle_seconds(ora, w, probe, cores)
    n_all, n_one = sample_sizes(rate0, cores, target_s, n)
    idx = np.linspace(0, n - 1, n_all).astype(np.int64)
    s_all = _oracle_seconds(ora, w, idx, cores)
    idx1 = np.linspace(0, n - 1, n_one).astype(np.int64)
    s_one = _oracle_seconds(ora, w, idx1, 1)
    return {"value": n_all / s_all, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_all} cells evenly spaced over the same {n}-cell field, one integrate each, "
                      f"{cores} threads (one cell per thread at a time)", "seconds": s_all,
            "single_core": {"value": n_one / s_one, "unit": "cells/s", "cores": 1, "cells": n_one,
                            "seconds": s_one,
                            "sample": f"{n_one} cells evenly spaced over the field, one thread"}}


def run_reference(args, w, world, rank):
    """The oracle as the reference arm: each step a bounded sample of the workload on all host
    cores (rank 0 only; other ranks exit without work)."""
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    ora = oracle.OracleMechanism(w["mech"].write_temp())
    n = w["T"].shape[0]
    probe = np.linspace(0, n - 1, cores).astype(np.int64)
    for _ in range(max(0, args.warmup)):
        rate0 = cores / _oracle_seconds(ora, w, probe, cores)
    if args.warmup <= 0:
        rate0 = cores / _oracle_seconds(ora, w, probe, cores)
    # about 120 s of timed CPU work in total, at least one cell per core per step
    per_step = max(cores, int(rate0 * 120.0 / max(1, args.steps)) // cores * cores)
    per_step = min(per_step, n)
    idx = np.linspace(0, n - 1, per_step).astype(np.int64)
    tot_s = 0.0
    for _ in range(args.steps):
        tot_s += _oracle_seconds(ora, w, idx, cores)
    value = per_step * args.steps / tot_s
    sample = (f"{per_step} cells evenly spaced over the same {n}-cell field per step, one integrate each, "
              f"{cores} threads (one cell per thread at a time)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, "fp64", None, "rosenbrock"),
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# Host-side arithmetic of the line

def _per_part(weights):
    with open(OPCOUNT_FILE) as fh:
        oc = json.load(fh)
    return {k: sum(weights[o] * v[o] for o in weights) for k, v in oc["counts"].items()}, oc["N"]


def algorithmic_flops(steps: np.ndarray, rejects: np.ndarray, weights=None):
    """FP64 FLOPs the method needs for the given per-cell step counts (oracle operation count per
    rate evaluation, Jacobian, LU and solve, with the given operation weights)."""
    per, N = _per_part(FLOP_WEIGHTS if weights is None else weights)
    # per attempt: W = I/(gamma h) - J (N^2 + N), LU, 4 stage solves + 1 error-filter solve,
    # 2 rate evaluations (stages 2 and 3; stage 4 reuses stage 3), stage combinations and error
    # norm (~ 30 N); per accepted step: one Jacobian (with its own rate evaluation).
    attempt = N * N + N + per["lu"] + 5 * per["solve"] + 2 * per["rates"] + 30 * N
    accepted = per["jacobian"]
    total_steps = int(steps.sum())
    total_attempts = total_steps + int(rejects.sum())
    return attempt * total_attempts + accepted * total_steps, {"per_attempt": attempt, "per_accepted": accepted}


def traffic_bytes(n_cells: int):
    """DRAM bytes of one integrate launch of n_cells from the two-capture fit (None without one)."""
    if TRAFFIC_FIT is None:
        return None
    return TRAFFIC_FIT["fixed"] + TRAFFIC_FIT["per_cell"] * n_cells


class Budget:
    """Wall-time budget of the run: the timed loop takes another step only if it, the steps that
    would follow, and the work after the loop (`reserve_s`) still fit."""

    def __init__(self, limit_s: float, t0: float = None):
        self.limit = float(limit_s)
        self.t0 = T_START if t0 is None else t0

    def elapsed(self, now=None):
        return (time.monotonic() if now is None else now) - self.t0

    def may_continue(self, done: int, requested: int, step_s: float, reserve_s: float, now=None) -> bool:
        if done >= requested:
            return False
        if done == 0:
            return True  # at least one timed step
        return self.elapsed(now) + step_s + reserve_s <= self.limit

    def projection(self, done: int, requested: int, step_s: float, reserve_s: float, now=None) -> dict:
        """The steps that fit at the measured step time (all requested ones, or fewer) and the
        projected end of the run, for the log line after the first timed step."""
        t = self.elapsed(now)
        n = done
        while n < requested and t + step_s + reserve_s <= self.limit:
            t += step_s
            n += 1
        return {"steps_that_fit": n, "requested": requested, "projected_end_s": t + reserve_s,
                "limit_s": self.limit}


def workload_config(w, precision, refine_sweeps, solver, **extra):
    K = w["mech"].K
    cfg = {"workload": w["name"], "cells": int(w["T"].shape[0]), "species": K, "reactions": w["mech"].R,
           "dt_s": w["dt"], "p_atm": w["p_Pa"] / 101325.0, "rtol": w["rtol"], "atol": w["atol"],
           "precision": precision, "refine_sweeps": refine_sweeps, "solver": solver,
           "start": "cold (every step from the initial field)"}
    cfg.update(extra)
    return cfg


def roofline_block(steps_np, rej_np, kern_ms_per_launch, peak, rosen, n_cells, traffic_ok):
    """The `roofline` object of the line: FP64-ALU bound, achieved FLOP/s of one launch from the
    algorithmic count (unit weights for `frac`, transcendental-weighted beside it)."""
    if rosen:
        f_unit, per_unit = algorithmic_flops(steps_np, rej_np, UNIT_WEIGHTS)
        f_w, per_w = algorithmic_flops(steps_np, rej_np, FLOP_WEIGHTS)
    else:
        f_unit = f_w = float("nan")
        per_unit = per_w = {"per_attempt": None, "per_accepted": None}
    sec = kern_ms_per_launch / 1e3
    a_unit = f_unit / sec / 1e12
    a_w = f_w / sec / 1e12
    ok = np.isfinite(a_unit)
    return {"bound": "alu", "achieved": a_unit if ok else None, "peak": peak["tflops"], "unit": "TFLOP/s",
            "frac": a_unit / peak["tflops"] if ok else None,
            "traffic": traffic_bytes(n_cells) if traffic_ok else None,
            "peak_source": peak["source"], "peak_measured": peak["measured_tflops"],
            "frac_of_measured": a_unit / peak["measured_tflops"] if ok else None,
            "weights": "add, mul, div, exp, log count 1 flop each",
            "achieved_weighted": a_w if ok else None,
            "frac_weighted": a_w / peak["tflops"] if ok else None,
            "frac_weighted_of_measured": a_w / peak["measured_tflops"] if ok else None,
            "weights_weighted": "exp 34 and log 62 flops (17 and 31 DFMA of FP64 pipe time)",
            "flops_per_attempt": per_unit["per_attempt"], "flops_per_accepted_step": per_unit["per_accepted"],
            "flops_per_attempt_weighted": per_w["per_attempt"],
            "flops_per_accepted_step_weighted": per_w["per_accepted"]}


def forward_line(*, w, world, args, steps_done, kern_ms, e2e, clk, st_np, steps_np, rej_np, peak, opts_info,
                 dtype, rosen, traffic_ok, lowp_stats, warm_cells, budget_stopped):
    """The JSON line of the forward workloads from the measured pieces (host arithmetic only)."""
    n_total = int(w["T"].shape[0])
    cells = n_total * world * steps_done
    value = cells / (kern_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": steps_done,
        "warmup": args.warmup, "ms_per_step": kern_ms / steps_done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": workload_config(w, args.precision, opts_info.get("refine_sweeps"), args.solver,
                                  warps_per_cell=opts_info.get("warps_per_cell"),
                                  cells_per_cta=opts_info.get("cells_per_cta"), cuda_graph=True,
                                  scheduling="persistent kernel + device work queue",
                                  call="chem_integrate on pinned host arrays (C ABI host path)",
                                  l2="flushed between steps (256 MiB write)",
                                  warmup_cells=warm_cells),
        "e2e": e2e,
        "gpu_launches": 1 * steps_done,
        "roofline": roofline_block(steps_np, rej_np, kern_ms / steps_done, peak, rosen, n_total, traffic_ok),
        "clocks": clk,
        "cells_status": {str(k): int(v) for k, v in zip(*np.unique(st_np, return_counts=True))},
        "steps_per_cell": {"mean": float(steps_np.mean()), "max": int(steps_np.max()),
                           "rejects_mean": float(rej_np.mean())},
    }
    if steps_done != args.steps or budget_stopped:
        line["steps_requested"] = args.steps
        line["budget_stop"] = f"timed loop stopped after {steps_done} of {args.steps} steps: wall-time budget " \
                              f"{args.budget_s:.0f} s"
    if lowp_stats:
        line["refinement"] = lowp_stats
    return line


def adjoint_line(*, w, world, args, n, K, R, N, cap, fwd, bwd, tot, clk, ns, st, peak_bytes, warm, h2d, d2h):
    cells = n * world * args.steps
    return {
        "metric": "cells/s, forward with checkpoints + discrete adjoint (53 sp, igniting band, dt 1e-4 s)",
        "value": cells / ((fwd + bwd) / 1e3), "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": (fwd + bwd) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "cells": n, "species": K, "reactions": R, "dt_s": w["dt"],
                   "p_atm": w["p_Pa"] / 101325.0, "rtol": w["rtol"], "atol": w["atol"],
                   "warmup_cells": warm, "l2": "flushed between steps (256 MiB write)",
                   "gradient": "dL/d(T0, Y0) per cell and dL/dlnA summed over cells, L random linear"},
        "forward_ms": fwd / args.steps, "backward_ms": bwd / args.steps, "backward_over_forward": bwd / fwd,
        "checkpoint": {"bytes_allocated": int(n * cap * (N + 1) * 8), "bytes_used": int(ns.sum()) * (N + 1) * 8,
                       "steps_per_cell_max": int(ns.max()), "steps_per_cell_mean": float(ns.mean()),
                       "peak_device_bytes": int(peak_bytes)},
        "e2e": {"value": cells / (tot / 1e3), "unit": "cells/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 4 * args.steps,
        "roofline": None,
        "clocks": clk,
        "cells_status": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
    }


# ------------------------------------------------------------------------------------------------
# GPU workloads

def run_adjoint(args, world, rank, local):
    """Forward with checkpoints + discrete adjoint on the igniting band (see the module doc)."""
    import torch
    from paper_2105_12070_gb300 import chem, ranks, synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.cells or 16384
    w = synth.workload_igniting(n)
    if args.dt > 0:
        w["dt"] = args.dt
    mech = chem.Mechanism(w["mech"].write_temp())
    N, K, R = mech.N, mech.K, mech.R
    rng = np.random.default_rng(7)
    T_host = torch.from_numpy(w["T"].copy()).pin_memory()
    Y_host = torch.from_numpy(w["Y"].copy()).pin_memory()
    gT_host = torch.from_numpy(rng.normal(size=n) * 1e-3).pin_memory()
    gY_host = torch.from_numpy(rng.normal(size=(K, n))).pin_memory()
    outs = [torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty((K, n), dtype=torch.float64).pin_memory(),
            torch.empty(R, dtype=torch.float64).pin_memory()]
    T = torch.empty_like(T_host, device="cuda")
    Y = torch.empty_like(Y_host, device="cuda")
    gT, gY = torch.empty_like(gT_host, device="cuda"), torch.empty_like(gY_host, device="cuda")
    gT0, gY0 = torch.empty_like(gT), torch.empty_like(gY)
    g_lnA = torch.empty(R, dtype=torch.float64, device="cuda")
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    nsteps = torch.zeros(n, dtype=torch.int32, device="cuda")
    # checkpoint capacity: the accepted-step count of a plain FP64 pass, plus a margin
    T.copy_(T_host)
    Y.copy_(Y_host)
    chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], status=status)
    steps = torch.zeros(n, dtype=torch.int32, device="cuda")
    chem.chem_last_cell_counters(mech, steps, None)
    cap = int(steps.max().item()) + 16
    rec = torch.empty((n, cap, N + 1), dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def one_step(m):
        flush.fill_(1.0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(stream)
        T[:m].copy_(T_host[:m], non_blocking=True)
        Y[:, :m].copy_(Y_host[:, :m], non_blocking=True)
        gT[:m].copy_(gT_host[:m], non_blocking=True)
        gY[:, :m].copy_(gY_host[:, :m], non_blocking=True)
        e[1].record(stream)
        Ts, Ys = (T, Y) if m == n else (T[:m].contiguous(), Y[:, :m].contiguous())
        chem.chem_integrate_record(mech, w["p_Pa"], Ts, Ys, w["dt"], rec[:m], nsteps[:m], status[:m],
                                   rtol=w["rtol"], atol=w["atol"])
        e[2].record(stream)
        gTs, gYs = (gT, gY) if m == n else (gT[:m].contiguous(), gY[:, :m].contiguous())
        gT0s, gY0s = (gT0, gY0) if m == n else (gT0[:m].contiguous(), gY0[:, :m].contiguous())
        chem.chem_adjoint(mech, w["p_Pa"], rec[:m], nsteps[:m], status[:m], gTs, gYs, gT0s, gY0s, g_lnA=g_lnA)
        ranks.sum_lnA_grad(g_lnA)  # the one exchange step (N > 1): sum of the per-rank gradients
        e[3].record(stream)
        outs[0][:m].copy_(gT0s, non_blocking=True)
        outs[1][:, :m].copy_(gY0s, non_blocking=True)
        outs[2].copy_(g_lnA, non_blocking=True)
        e[4].record(stream)
        e[4].synchronize()
        return e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3]), e[0].elapsed_time(e[4])

    warm = min(n, 152)
    for _ in range(args.warmup):
        one_step(warm)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    clocks = ClockSampler(local)
    clocks.start()
    fwd = bwd = tot = 0.0
    for _ in range(args.steps):
        a, b, c = one_step(n)
        fwd += a
        bwd += b
        tot += c
    torch.cuda.synchronize()
    clk = clocks.stop()
    fwd, bwd, tot = ranks.max_over_ranks([fwd, bwd, tot], device="cuda")
    line = adjoint_line(w=w, world=world, args=args, n=n, K=K, R=R, N=N, cap=cap, fwd=fwd, bwd=bwd, tot=tot,
                        clk=clk, ns=nsteps.cpu().numpy(), st=status.cpu().numpy(),
                        peak_bytes=torch.cuda.max_memory_allocated(), warm=warm,
                        h2d=(T_host.numel() + Y_host.numel() + gT_host.numel() + gY_host.numel()) * 8,
                        d2h=(n + K * n + R) * 8)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_ablation(args, world, rank, local):
    """The paper's Fig. 3 experiment on the GPU (Sec. 2.3): a 0D reactor (the 53-species mechanism
    at 1200 K, 13.5 atm) advanced over CFD steps of 1e-6 s with the step carried over, timed for
    each absolute tolerance with (forward-difference Jacobian, FP64 LU), (analytical Jacobian, FP64
    LU), (analytical Jacobian, FP32 LU + FP64 refinement) and Seulex."""
    import torch
    from paper_2105_12070_gb300 import chem, ranks, synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.cells or 608
    w = synth.workload_0d(n)
    mech = chem.Mechanism(w["mech"].write_temp())
    ncfd = 50
    variants = [("fd_fp64", dict(jacobian=chem.CHEM_JAC_FD)),
                ("analytic_fp64", dict()),
                ("analytic_mixed", dict(precision=chem.CHEM_PREC_MIXED)),
                ("seulex", dict(solver=chem.CHEM_SOLVER_SEULEX))]
    atols = (1e-8, 1e-10, 1e-12, 1e-14)
    T = torch.empty(n, dtype=torch.float64, device="cuda")
    Y = torch.empty((mech.K, n), dtype=torch.float64, device="cuda")
    h = torch.zeros(n, dtype=torch.float64, device="cuda")
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    T0 = torch.from_numpy(w["T"]).cuda()
    Y0 = torch.from_numpy(w["Y"]).cuda()
    stream = torch.cuda.current_stream()
    rows = []
    clocks = ClockSampler(local)
    clocks.start()
    for name, kw in variants:
        opts = chem.default_opts(**kw)
        for atol in atols:
            for rep in range(2):  # the first pass warms the launch path, the second is timed
                T.copy_(T0)
                Y.copy_(Y0)
                h.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                steps = 0
                for _ in range(ncfd):
                    st = chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], atol, h_inout=h,
                                             status=status, opts=opts, want_stats=True)
                    steps += st.steps
                e1.record(stream)
                e1.synchronize()
            ms = e0.elapsed_time(e1)
            rows.append({"variant": name, "atol": atol, "ms": ms, "ms_per_cfd_step": ms / ncfd,
                         "steps_per_cell": steps / n, "T_final": float(T[0].item()),
                         "failed_cells": int((status != 0).sum().item())})
    clk = clocks.stop()
    ms_all = ranks.max_over_ranks([r["ms"] for r in rows], device="cuda")
    for r, m in zip(rows, ms_all):
        r["ms"] = m
    ref = {r["atol"]: r["ms"] for r in rows if r["variant"] == "analytic_fp64"}
    for r in rows:
        r["time_vs_analytic_fp64"] = r["ms"] / ref[r["atol"]]
    head = next(r for r in rows if r["variant"] == "analytic_fp64" and r["atol"] == 1e-10)
    line = {
        "metric": "0D reactor: time per CFD step vs absolute tolerance (Fig. 3 analogue)",
        "value": head["ms_per_cfd_step"], "unit": "ms per CFD step (608 reactors)", "n_gpus": world,
        "steps": ncfd, "warmup": 1, "ms_per_step": head["ms_per_cfd_step"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "cells": n, "species": mech.K, "reactions": mech.R, "dt_s": w["dt"],
                   "p_atm": 13.5, "T0_K": 1200.0, "rtol": w["rtol"], "cfd_steps": ncfd},
        "ablation": rows, "clocks": clk, "gpu_launches": None, "roofline": None,
        "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    world, rank, local = dist_setup(args)
    from paper_2105_12070_gb300 import synth
    if args.workload == "adjoint" and args.impl == "gpu":
        return run_adjoint(args, world, rank, local)
    if args.workload == "0d" and args.impl == "gpu":
        return run_ablation(args, world, rank, local)
    if args.workload == "uneven":
        w = synth.workload_uneven(args.cells or 262144, args.order)
    else:
        w = synth.workload_shear_layer()
    if args.dt > 0:
        w["dt"] = args.dt
    if args.rtol > 0:
        w["rtol_nominal"] = w["rtol"]
        w["rtol"] = args.rtol
    if args.impl == "reference":
        return run_reference(args, w, world, rank)
    return run_forward(args, w, world, rank, local)


def run_forward(args, w, world, rank, local):
    import torch
    from paper_2105_12070_gb300 import chem, ranks

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rtol_nominal = w.get("rtol_nominal", w["rtol"])
    budget = Budget(args.budget_s)
    mech = chem.Mechanism(w["mech"].write_temp())
    n_field = w["T"].shape[0]
    n_total = n_field if args.cells <= 0 else args.cells
    # weak scaling: every rank integrates its own copy of the field (cells are independent); a
    # smaller --cells takes evenly spaced cells of the field (profiling and parity slices)
    if n_total < n_field:
        idx = np.linspace(0, n_field - 1, n_total).astype(np.int64)
        w = dict(w, T=w["T"][idx].copy(), Y=w["Y"][:, idx].copy(), name=f"{w['name']}_sample{n_total}")
    elif n_total > n_field:
        idx = np.arange(n_total) % n_field
        w = dict(w, T=w["T"][idx].copy(), Y=w["Y"][:, idx].copy(), name=f"{w['name']}_tiled{n_total}")
    # the CPU oracle's legs first, on the host cores while the GPU is idle, so that the budget of
    # the timed loop needs no reserve for them (one process only: N = 1)
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, args.cpu_seconds)
        cb.pop("seconds", None)
    T_host = torch.from_numpy(w["T"].copy()).pin_memory()
    Y_host = torch.from_numpy(w["Y"].copy()).pin_memory()
    T = torch.empty_like(T_host, device="cuda")
    Y = torch.empty_like(Y_host, device="cuda")
    status = torch.zeros(n_total, dtype=torch.int32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    prec = {"fp64": chem.CHEM_PREC_FP64, "mixed": chem.CHEM_PREC_MIXED, "ff": chem.CHEM_PREC_MIXED_FF}[args.precision]
    solver = chem.CHEM_SOLVER_SEULEX if args.solver == "seulex" else chem.CHEM_SOLVER_ROSENBROCK
    if args.autotune:
        from paper_2105_12070_gb300 import autotune
        opts = autotune.autotune(mech, w["p_Pa"], w["T"], w["Y"], w["dt"], precision=prec)
        opts.solver = solver
    else:
        opts = chem.default_opts(precision=prec, solver=solver)
    if args.refine_sweeps >= 0:
        opts.refine_sweeps = args.refine_sweeps
    opts.use_graph = 1
    stream = torch.cuda.current_stream()
    lowp_stats = {}

    Tp = torch.empty_like(T_host).pin_memory()  # the caller's host arrays of the timed calls
    Yp = torch.empty_like(Y_host).pin_memory()
    sp = torch.empty(n_total, dtype=torch.int32).pin_memory()

    def host_call(m, o=None):
        """One step: the field (its first m cells) copied into pinned host arrays and L2 flushed
        outside the timing, then one chem_integrate call through the C ABI on those host arrays:
        the library stages them to the device, integrates and copies the result back.  Returns
        (device ms of the integrate launch from the library's events on the stream, wall ms of the
        whole call)."""
        if m == n_total:
            Ta, Ya, sa = Tp, Yp, sp
            Ta.copy_(T_host)
            Ya.copy_(Y_host)
        else:
            Ta = T_host[:m].clone().pin_memory()
            Ya = Y_host[:, :m].contiguous().pin_memory()
            sa = sp[:m]
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = chem.chem_integrate(mech, w["p_Pa"], Ta, Ya, w["dt"], w["rtol"], w["atol"], status=sa,
                                 opts=opts if o is None else o, want_stats=True, stream=stream.cuda_stream)
        wall_ms = (time.perf_counter() - t0) * 1e3
        if prec != chem.CHEM_PREC_FP64:
            lowp_stats.update(attempts=int(st.steps + st.rejects), refine_fallbacks=int(st.refine_fallbacks))
        return st.kernel_ms, wall_ms

    warm = min(args.warm_cells, n_total)
    for i in range(args.warmup):
        host_call(warm)
    # the library's per-cell and staging buffers for the full field, outside the timed region
    host_call(n_total, o=chem.default_opts(max_steps=1))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    kern_ms, wall_ms = 0.0, 0.0
    done = 0
    reserve = 20.0  # counters, the peak probe and the print after the loop (a few seconds)
    stopped = False
    while True:
        step_s = wall_ms / 1e3 / done if done else 0.0
        if not budget.may_continue(done, args.steps, step_s, reserve):
            stopped = done < args.steps
            break
        k, wms = host_call(n_total)
        kern_ms += k
        wall_ms += wms
        done += 1
        if done == 1 and rank == 0:
            pj = budget.projection(done, args.steps, wms / 1e3, reserve)
            print(f"bench: first timed step {wms / 1e3:.1f} s; {pj['steps_that_fit']} of {pj['requested']} steps "
                  f"fit, projected end {pj['projected_end_s']:.0f} s of the {pj['limit_s']:.0f} s budget",
                  file=sys.stderr, flush=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    T_out, Y_out = Tp.clone(), Yp.clone()
    st_np = sp.numpy().copy()
    steps = torch.zeros(n_total, dtype=torch.int32, device="cuda")
    rej = torch.zeros_like(steps)
    chem.chem_last_cell_counters(mech, steps, rej)
    steps_np, rej_np = steps.cpu().numpy(), rej.cpu().numpy()
    kern_ms, wall_ms = ranks.max_over_ranks([kern_ms, wall_ms], device="cuda")
    e2e = {"value": n_total * world * done / (wall_ms / 1e3), "unit": "cells/s",
           "h2d_bytes_per_step": int(T_host.numel() * 8 + Y_host.numel() * 8),
           "d2h_bytes_per_step": int(T_host.numel() * 8 + Y_host.numel() * 8 + n_total * 4),
           "how": "host wall time of the same timed chem_integrate calls on pinned host arrays (the C ABI's host "
                  "path: staging copies in and out inside each call); `value` is the device time of their "
                  "integrate launches"}
    rosen = solver == chem.CHEM_SOLVER_ROSENBROCK
    peak = fp64_peak_tflops()
    line = forward_line(
        w=w, world=world, args=args, steps_done=done, kern_ms=kern_ms, e2e=e2e, clk=clk, st_np=st_np,
        steps_np=steps_np, rej_np=rej_np, peak=peak,
        opts_info={"refine_sweeps": opts.refine_sweeps if prec != chem.CHEM_PREC_FP64 else None,
                   "warps_per_cell": opts.warps_per_cell, "cells_per_cta": opts.cells_per_cta},
        dtype={chem.CHEM_PREC_FP64: "f64", chem.CHEM_PREC_MIXED: "f64+f32"}.get(prec, "f64+f32x2"),
        rosen=rosen and mech.K == 53,
        traffic_ok=(mech.K == 53 and prec == chem.CHEM_PREC_FP64 and rosen and args.dt <= 0),
        lowp_stats=lowp_stats, warm_cells=warm, budget_stopped=stopped)
    if args.accuracy_sample > 0:
        # a converged FP64 solution of sampled cells (tight tolerances) on the same GPU path
        m_s = min(args.accuracy_sample, n_total)
        sidx = np.linspace(0, n_total - 1, m_s).astype(np.int64)
        Ts = torch.from_numpy(T_host.numpy()[sidx].copy()).cuda()
        Ys = torch.from_numpy(Y_host.numpy()[:, sidx].copy()).cuda()
        sst = torch.zeros(m_s, dtype=torch.int32, device="cuda")
        aopts = chem.default_opts(max_steps=2000000)
        chem.chem_integrate(mech, w["p_Pa"], Ts, Ys, w["dt"], 1e-10, 1e-14, status=sst, opts=aopts)
        Tt, Yt = Ts.cpu().numpy(), Ys.cpu().numpy()
        Tr, Yr = T_out.numpy()[sidx], Y_out.numpy()[:, sidx]
        scT = w["atol"] + rtol_nominal * np.abs(Tt)
        scY = w["atol"] + rtol_nominal * np.abs(Yt)
        eT = np.abs(Tr - Tt) / scT
        eY = np.abs(Yr - Yt) / scY
        per_cell = np.maximum(eT, eY.max(axis=0))
        line["accuracy"] = {"sample_cells": int(m_s), "reference": "GPU Rosenbrock FP64, rtol 1e-10, atol 1e-14",
                            "reference_status_ok": bool(np.all(sst.cpu().numpy() == 0)),
                            "units": f"atol + rtol |x| with the nominal rtol {rtol_nominal:g}",
                            "max_err": float(per_cell.max()), "median_err": float(np.median(per_cell)),
                            "max_rel_err_T": float((np.abs(Tr - Tt) / np.abs(Tt)).max())}
    if args.map and "streams" in w:
        (Tf, Yf), (To, Yo) = w["streams"]
        refs = np.array([np.concatenate([[Tf], Yf]), np.concatenate([[To], Yo])])
        T.copy_(T_host)
        Y.copy_(Y_host)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nm, _ = chem.chem_integrate_mapped(mech, w["p_Pa"], T, Y, w["dt"], refs, 1e-6, 1e-9, rtol=w["rtol"],
                                           atol=w["atol"], status=status, opts=opts)
        e1.record(stream)
        e1.synchronize()
        mms = e0.elapsed_time(e1)
        Tm, Ym = T.cpu().numpy(), Y.cpu().numpy()
        Tr, Yr = T_out.numpy(), Y_out.numpy()
        line["reference_mapping"] = {
            "tol_T_K": 1e-6, "tol_Y": 1e-9, "mapped_cells": int(nm), "ms_per_step": mms,
            "value": n_total / (mms / 1e3), "speedup": (kern_ms / done) / mms,
            "max_err_vs_solve_in_tol_units": float(max(
                (np.abs(Tm - Tr) / (w["atol"] + w["rtol"] * np.abs(Tr))).max(),
                (np.abs(Ym - Yr) / (w["atol"] + w["rtol"] * np.abs(Yr))).max()))}
    if args.vs_fp64:
        # the plain FP64 Rosenbrock path on the same field, for the comparison the precision and
        # solver options are compared against (speed and the state it produces)
        T_ref, Y_ref = T_out.clone(), Y_out.clone()
        fopts = chem.default_opts(precision=chem.CHEM_PREC_FP64, solver=chem.CHEM_SOLVER_ROSENBROCK)
        fopts.use_graph = 1
        T.copy_(T_host)
        Y.copy_(Y_host)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], status=status, opts=fopts)
        e1.record(stream)
        e1.synchronize()
        fms = e0.elapsed_time(e1)
        Tf, Yf = T.cpu().numpy(), Y.cpu().numpy()
        dT = np.abs(T_ref.numpy() - Tf) / np.abs(Tf)
        dY = np.abs(Y_ref.numpy() - Yf)
        line["vs_fp64"] = {"fp64_ms_per_step": fms, "speedup": fms / (kern_ms / done),
                           "max_rel_err_T": float(dT.max()),
                           "max_abs_err_Y": float(dY.max()),
                           "max_err_Y_in_tol_units": float((dY / (w["atol"] + w["rtol"] * np.abs(Yf))).max()),
                           "max_err_T_in_tol_units": float((np.abs(T_ref.numpy() - Tf) /
                                                            (w["atol"] + w["rtol"] * np.abs(Tf))).max())}
    if args.warm_start:
        # the next CFD step of the same field: an untimed cold call leaves T, Y at dt and the
        # controller's proposal in h; the timed call continues from there (Sec. 2.3: the previous
        # sub-step is the first guess of the next interval)
        hbuf = torch.zeros(n_total, dtype=torch.float64, device="cuda")
        T.copy_(T_host)
        Y.copy_(Y_host)
        chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], h_inout=hbuf, status=status,
                            opts=opts)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], h_inout=hbuf, status=status,
                            opts=opts)
        e1.record(stream)
        e1.synchronize()
        wms = e0.elapsed_time(e1)
        chem.chem_last_cell_counters(mech, steps, rej)
        wst = steps.cpu().numpy()
        line["warm_start"] = {"value": n_total / (wms / 1e3), "unit": "cells/s", "ms_per_step": wms,
                              "steps_per_cell_mean": float(wst.mean()), "steps_per_cell_max": int(wst.max()),
                              "cells_status": {str(k): int(v) for k, v in
                                               zip(*np.unique(status.cpu().numpy(), return_counts=True))}}
    if args.batch_cells > 0:
        # one launch per batch of consecutive cells, static assignment inside each launch
        bopts = chem.default_opts(precision=prec, use_queue=0, batch_cells=args.batch_cells,
                                  warps_per_cell=opts.warps_per_cell, cells_per_cta=opts.cells_per_cta,
                                  solver=solver)
        bopts.use_graph = 1
        bms = host_call(n_total, o=bopts)[0]
        line["batched_launches"] = {"batch_cells": args.batch_cells, "ms_per_step": bms,
                                    "value": n_total / (bms / 1e3), "queue_speedup": bms / (kern_ms / done)}
    if cb is not None:
        line["cpu_baseline"] = cb
    line["wall_s"] = budget.elapsed()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# FP64 peak from unit counts and clocks: GB300's nominal FP64 rate (1.25 TFLOP/s) is 2 FP64 FMA
# lanes per clock per SM (152 SMs x 2.07 GHz x 2 lanes x 2 flop = 1.259 TFLOP/s); one FP64 warp
# instruction per 64 clocks per SM sub-partition
FP64_LANES_PER_SM_CLK = 2
N_SMS = 152
SM_MAX_CLOCK_GHZ = 2.07


def fp64_peak_tflops():
    """The roofline denominator of the FP64-ALU-bound kernels: derived from the unit count and
    the maximum SM clock, with the DFMA throughput measured in this process beside it
    (chem_probe_fp64_peak: 8 independent DFMA chains per thread, 4 x 256 threads per SM)."""
    from paper_2105_12070_gb300 import chem
    derived = FP64_LANES_PER_SM_CLK * N_SMS * SM_MAX_CLOCK_GHZ * 2.0 / 1e3
    return {"tflops": derived, "measured_tflops": chem.chem_probe_fp64_peak(),
            "source": "derived: 2 FP64 FMA lanes/clk/SM x 152 SMs x 2.07 GHz x 2 flop (nominal 1.25 TFLOP/s)"}


if __name__ == "__main__":
    sys.exit(main())
