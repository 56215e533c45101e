"""Per-phase cycle counters of the integrate kernel (a profiling aid; needs a GPU).

Builds a second copy of the library with -DCHEM_PHASE_TIMERS (thread 0 of each cell group adds
clock64() deltas per phase), integrates an evenly spaced sample of the 53-species shear-layer
field over a short interval in each precision mode, and prints the cycles per step attempt of one
cell group for: the rate evaluation with Jacobian data, the Jacobian assembly, W and its LU, the
stage solves (with any refinement), the two stage rate evaluations and the step control.  The
timers perturb the kernel a little; compare phases, not absolute speed.

    python -m paper_2105_12070_gb300.phases [--cells 1216] [--dt 1e-8] [--define NAME ...] [--modes 0,2]

--define adds a preprocessor macro to the timer build (e.g. CHEM_LU_VARIANT=0: the LU column by
column, =2: in 8-column panels; CHEM_LU_RCP_DIVISION: FP64 pivot reciprocals by division).
"""
from __future__ import annotations

import argparse
import ctypes
import os

import numpy as np

PHASES = ["rates+Jdata", "J assembly", "W+LU", "solves", "stage rates", "control"]
# (precision, refinement sweeps) pairs: FP64, FP32 + refinement, FP32 pairs with 2 / 1 / 0 sweeps
MODES = [(0, 2), (1, 2), (2, 2), (2, 1), (2, 0)]


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cells", type=int, default=1216)
    ap.add_argument("--dt", type=float, default=1e-8)
    ap.add_argument("--define", action="append", default=[], help="extra macro of the timer build")
    ap.add_argument("--modes", default="", help="comma-separated indices into MODES (default: all)")
    args = ap.parse_args(argv)

    from . import build
    tag = "_".join(["phase_timers"] + [d.lower().replace("=", "") for d in args.define])
    out = os.path.join(build.BUILD, tag, "libchemgpu.so")
    build.build(defines=["CHEM_PHASE_TIMERS"] + list(args.define), out=out, force=True)
    build.LIB = out  # this process loads the timer build
    import torch

    from . import chem, synth
    lib = chem.load_library(build_if_missing=False)
    lib.chem_debug_phase_cycles.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
    w = synth.workload_shear_layer()
    mech = chem.Mechanism(w["mech"].write_temp())
    n = min(args.cells, w["T"].shape[0])
    idx = np.arange(n) * (w["T"].shape[0] // n)
    buf = (ctypes.c_ulonglong * 8)()
    modes = [MODES[int(i)] for i in args.modes.split(",")] if args.modes else MODES
    print("defines: " + (" ".join(args.define) or "(none)"), flush=True)
    for prec, sweeps in modes:
        T = torch.from_numpy(w["T"][idx].copy()).cuda()
        Y = torch.from_numpy(w["Y"][:, idx].copy()).cuda()
        opts = chem.default_opts(warps_per_cell=2, precision=prec, refine_sweeps=sweeps)
        lib.chem_debug_phase_cycles(buf)  # reset
        st = chem.chem_integrate(mech, w["p_Pa"], T, Y, args.dt, w["rtol"], w["atol"], opts=opts, want_stats=True)
        torch.cuda.synchronize()
        lib.chem_debug_phase_cycles(buf)
        attempts = st.steps + st.rejects
        c = np.array(list(buf)[:len(PHASES)], dtype=np.float64) / max(attempts, 1)
        print(f"precision {prec} sweeps {sweeps}: {attempts} attempts, {st.refine_fallbacks} fallbacks; cycles per "
              "attempt: " + ", ".join(f"{name} {v:.0f}" for name, v in zip(PHASES, c)) + f"; total {c.sum():.0f}",
              flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
