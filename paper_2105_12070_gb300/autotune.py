"""Autotuner for the integrate launch shape: warps per cell (G) and cells per CTA.

Every candidate the library accepts for the mechanism is timed on a sample of the caller's cells
over a short interval (the per-step cost is what the shape changes; the early, stiffest part of
the integration has the same per-step mix of rate, Jacobian, LU and solve work), and the one with
the most step attempts per second wins: each candidate is timed `repeats` times with CUDA events
and its median counts.  Results are cached in a JSON file per (species, reactions,
pressure-dependent reactions, solver, precision, device name): the per-cell shared-memory plan
depends on the first three, the kernel on the solver and precision.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import chem

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "chemgpu_autotune.json")


def _key(mech, precision: int, solver: int) -> str:
    import torch
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    return f"K{mech.K}-R{mech.R}-pd{mech.n_pd}-solver{solver}-prec{precision}-{name}"


def candidates():
    out = []
    for G in (1, 2, 4, 8):
        for cpc in range(1, 8 // G + 1):
            out.append((G, cpc))
    return out


def autotune(mech: chem.Mechanism, p_Pa: float, T, Y, dt: float, rtol: float = 1e-6, atol: float = 1e-10,
             precision: int = chem.CHEM_PREC_FP64, solver: int = chem.CHEM_SOLVER_ROSENBROCK,
             tune_dt: float = 1e-9, repeats: int = 5, cache_path: str | None = DEFAULT_CACHE, force: bool = False,
             verbose: bool = False) -> chem.ChemOpts:
    """Returns ChemOpts with the fastest (warps_per_cell, cells_per_cta) for this mechanism.
    T [n] and Y [K, n] are host (numpy) or device (torch) arrays of representative cells."""
    import torch
    key = _key(mech, precision, solver)
    if cache_path and not force and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if key in cache:
            c = cache[key]
            return chem.default_opts(precision=precision, solver=solver, warps_per_cell=c["G"],
                                     cells_per_cta=c["cells_per_cta"])
    T = torch.as_tensor(np.asarray(T.cpu() if hasattr(T, "cpu") else T), dtype=torch.float64)
    Y = torch.as_tensor(np.asarray(Y.cpu() if hasattr(Y, "cpu") else Y), dtype=torch.float64)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    n = min(T.shape[0], 2 * sms * 8)
    idx = torch.linspace(0, T.shape[0] - 1, n).long()
    T0 = T[idx].contiguous().cuda()
    Y0 = Y[:, idx].contiguous().cuda()
    results = []
    stream = torch.cuda.current_stream()
    for G, cpc in candidates():
        opts = chem.default_opts(precision=precision, solver=solver, warps_per_cell=G, cells_per_cta=cpc)
        try:
            Tt, Yt = T0.clone(), Y0.clone()
            chem.chem_integrate(mech, p_Pa, Tt, Yt, tune_dt, rtol, atol, opts=opts)  # warm-up / validity
            torch.cuda.synchronize()
        except chem.ChemError:
            continue
        rates = []
        for _ in range(max(1, repeats)):
            Tt, Yt = T0.clone(), Y0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = chem.chem_integrate(mech, p_Pa, Tt, Yt, tune_dt, rtol, atol, opts=opts, want_stats=True)
            e1.record(stream)
            e1.synchronize()
            rates.append((st.steps + st.rejects) / (e0.elapsed_time(e1) / 1e3))
        rate = float(np.median(rates))
        results.append((rate, G, cpc))
        if verbose:
            print(f"autotune G={G} cells/CTA={cpc}: {rate:.4g} step attempts/s (median of {len(rates)})")
    if not results:
        raise chem.ChemError("autotune: no launch shape fits this mechanism")
    rate, G, cpc = max(results)
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache = {}
        if os.path.exists(cache_path):
            try:
                with open(cache_path) as fh:
                    cache = json.load(fh)
            except (OSError, ValueError):
                cache = {}
        cache[key] = {"G": G, "cells_per_cta": cpc, "attempts_per_s": rate,
                      "all": [{"G": g, "cells_per_cta": c, "attempts_per_s": r} for r, g, c in results]}
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return chem.default_opts(precision=precision, solver=solver, warps_per_cell=G, cells_per_cta=cpc)
