"""Differentiable chemistry solve: torch.autograd.Function over chem_integrate_record /
chem_adjoint (the discrete adjoint of the accepted Rosenbrock steps, step sizes frozen).

    T1, Y1, status = integrate(mech, p_Pa, T0, Y0, lnA, dt)  # forward on the GPU, checkpoints kept
    loss(T1, Y1).backward()                               # reverse sweep on the GPU

gives dloss/dT0, dloss/dY0 (zero for the last species, which the solve recomputes as
1 - sum of the others) and dloss/dlnA (R,), lnA the ln of the pre-exponential factors of the
forward rate constants (of k_inf for fall-off reactions) in the mechanism file's reaction
order.  Marshalling only: both sweeps run in libchemgpu.
"""
from __future__ import annotations

import numpy as np
import torch

from . import chem

_MAX_STEPS_REC = 4096


def _ensure_lnA(mech: chem.Mechanism, lnA: torch.Tensor):
    want = lnA.detach().to("cpu", torch.float64).numpy()
    cur = getattr(mech, "_lnA_cache", None)
    if cur is None:
        cur = chem.chem_get_lnA(mech)
    if not np.array_equal(cur, want):
        chem.chem_set_lnA(mech, want)
        cur = want.copy()
    mech._lnA_cache = cur


class ChemIntegrateFunction(torch.autograd.Function):
    """(T0, Y0, lnA) -> (T(dt), Y(dt)) for every cell; see the module docstring."""

    @staticmethod
    def forward(ctx, T0, Y0, lnA, mech, p_Pa, dt, rtol, atol, max_steps_rec, opts):
        _ensure_lnA(mech, lnA)
        n = int(T0.shape[0])
        T = T0.detach().to(torch.float64).contiguous().clone()
        Y = Y0.detach().to(torch.float64).contiguous().clone()
        dev = T.device
        rec = torch.empty((n, max_steps_rec, mech.N + 1), dtype=torch.float64, device=dev)
        nsteps = torch.empty(n, dtype=torch.int32, device=dev)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        chem.chem_integrate_record(mech, p_Pa, T, Y, dt, rec, nsteps, status, rtol=rtol, atol=atol, opts=opts)
        ctx.save_for_backward(rec, nsteps, status)
        ctx.mech, ctx.p_Pa = mech, p_Pa
        ctx.lnA_values = mech._lnA_cache.copy()
        ctx.mark_non_differentiable(status)
        return T, Y, status

    @staticmethod
    def backward(ctx, gT, gY, _gstatus):
        rec, nsteps, status = ctx.saved_tensors
        mech = ctx.mech
        if not np.array_equal(mech._lnA_cache, ctx.lnA_values):
            chem.chem_set_lnA(mech, ctx.lnA_values)
            mech._lnA_cache = ctx.lnA_values.copy()
        n = int(nsteps.shape[0])
        dev = rec.device
        gT = torch.zeros(n, dtype=torch.float64, device=dev) if gT is None else gT.to(torch.float64).contiguous()
        gY = (torch.zeros((mech.K, n), dtype=torch.float64, device=dev) if gY is None
              else gY.to(torch.float64).contiguous())
        gT0 = torch.empty_like(gT)
        gY0 = torch.empty_like(gY)
        g_lnA = torch.empty(mech.R, dtype=torch.float64, device=dev)
        chem.chem_adjoint(mech, ctx.p_Pa, rec, nsteps, status, gT, gY, gT0, gY0, g_lnA=g_lnA)
        return gT0, gY0, g_lnA, None, None, None, None, None, None, None


def integrate(mech: chem.Mechanism, p_Pa: float, T0: torch.Tensor, Y0: torch.Tensor, lnA: torch.Tensor, dt: float,
              rtol: float = 1e-6, atol: float = 1e-10, max_steps_rec: int = _MAX_STEPS_REC, opts=None):
    """Differentiable chem_integrate: returns (T(dt), Y(dt), status).  status (int32, not
    differentiable) is CHEM_CELL_* per cell; a cell that needs more than max_steps_rec accepted
    steps ends with status record_full, and any cell whose status is not ok gets NaN gradients."""
    return ChemIntegrateFunction.apply(T0, Y0, lnA, mech, float(p_Pa), float(dt), float(rtol), float(atol),
                                       int(max_steps_rec), opts)
