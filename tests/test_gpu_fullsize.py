"""Parity at the full benchmark size, in the benchmark's launch configuration.

The whole 65 536-cell shear-layer field goes through one chem_integrate call with the
benchmark's options (persistent kernel, device work queue, CUDA graph; automatic launch shape).
The oracle integrates a sample of 32 cells spread over the field one by one, and the GPU values
of those cells must match within the integrate tolerance 1e-6 |x| + 1e-10.  Every cell of the
field must end with status OK, T and Y finite, sum Y = 1 to 1e-12 and its element totals kept to
1e-12, and every 64th cell its mixture enthalpy kept to 2e-5 of its scale (properties of Eq. 1
that hold at any size).  The discrete adjoint gets the same treatment at its benchmark size (16 384 igniting
cells): the dot-product identity against the oracle's tangent-linear replay on two sampled cells.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def test_full_shear_field_in_benchmark_configuration():
    w = synth.workload_shear_layer()
    path = w["mech"].write_temp()
    mech, om = chem.Mechanism(path), O.OracleMechanism(path)
    n = w["T"].shape[0]
    T = torch.from_numpy(w["T"].copy()).cuda()
    Y = torch.from_numpy(w["Y"].copy()).cuda()
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    opts = chem.default_opts()
    opts.use_graph = 1
    chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], status=status, opts=opts)
    torch.cuda.synchronize()
    Tg, Yg, st = T.cpu().numpy(), Y.cpu().numpy(), status.cpu().numpy()
    assert np.all(st == 0)
    assert np.all(np.isfinite(Tg)) and np.all(np.isfinite(Yg))
    assert np.max(np.abs(Yg.sum(axis=0) - 1.0)) <= 1e-12
    # invariants of Eq. 1 on every cell: element totals (linear invariants, kept by the method to
    # rounding) and the mixture enthalpy at constant pressure (kept to the integration tolerance)
    gen = w["mech"]
    e0 = gen.comp.T @ (w["Y"] / gen.W[:, None])
    e1 = gen.comp.T @ (Yg / gen.W[:, None])
    assert np.max(np.abs(e1 - e0) / np.abs(e0).max(axis=0)) <= 1e-12
    ru = 8.314462618e7
    for c in range(0, n, 64):
        h = []
        for Tc, Yc in ((w["T"][c], w["Y"][:, c]), (Tg[c], Yg[:, c])):
            _, hRT, _ = om.thermo(Tc)
            hk = hRT * ru * Tc / gen.W
            h.append(((Yc * hk).sum(), np.abs(Yc * hk).sum()))
        assert abs(h[1][0] - h[0][0]) <= 2e-5 * h[0][1], c
    idx = np.random.default_rng(11).choice(n, size=32, replace=False)
    To, Yo, so, _, _ = om.integrate(w["p_Pa"], w["T"][idx], w["Y"][:, idx], w["dt"], w["rtol"], w["atol"],
                                    nthreads=16)
    assert np.all(so == 0)
    assert np.all(np.abs(Tg[idx] - To) <= 1e-6 * np.abs(To) + 1e-10)
    assert np.all(np.abs(Yg[:, idx] - Yo) <= 1e-6 * np.abs(Yo) + 1e-10)


def test_full_adjoint_configuration_sampled():
    w = synth.workload_igniting(16384)
    path = w["mech"].write_temp()
    mech, om = chem.Mechanism(path), O.OracleMechanism(path)
    n = w["T"].shape[0]
    cap = 4096
    T = torch.from_numpy(w["T"].copy()).cuda()
    Y = torch.from_numpy(w["Y"].copy()).cuda()
    rec = torch.empty((n, cap, mech.N + 1), dtype=torch.float64, device="cuda")
    nsteps = torch.empty(n, dtype=torch.int32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    chem.chem_integrate_record(mech, w["p_Pa"], T, Y, w["dt"], rec, nsteps, status, rtol=w["rtol"], atol=w["atol"])
    rng = np.random.default_rng(12)
    gT = rng.normal(size=n) * 1e-3
    gY = rng.normal(size=(mech.K, n))
    gT0 = torch.empty(n, dtype=torch.float64, device="cuda")
    gY0 = torch.empty((mech.K, n), dtype=torch.float64, device="cuda")
    gA = torch.empty(mech.R, dtype=torch.float64, device="cuda")
    chem.chem_adjoint(mech, w["p_Pa"], rec, nsteps, status, torch.from_numpy(gT).cuda(),
                      torch.from_numpy(gY).cuda(), gT0, gY0, g_lnA=gA)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert np.all(st == 0)
    g0, gy0 = gT0.cpu().numpy(), gY0.cpu().numpy()
    assert np.all(np.isfinite(g0)) and np.all(np.isfinite(gy0)) and np.all(np.isfinite(gA.cpu().numpy()))
    ns = nsteps.cpu().numpy()
    for c in rng.choice(n, size=2, replace=False):
        hs = rec[c, :ns[c], -1].cpu().numpy()
        phi0 = np.concatenate([[w["T"][c]], w["Y"][:-1, c]])
        lam = np.concatenate([[gT[c]], gY[:-1, c] - gY[-1, c]])
        d = rng.normal(size=mech.N) * np.maximum(np.abs(phi0), 1e-8)
        _, tl = om.replay(w["p_Pa"], phi0, hs, dphi=d)
        lhs = lam @ tl
        rhs = g0[c] * d[0] + gy0[:-1, c] @ d[1:]
        assert abs(lhs - rhs) <= 1e-8 * (np.abs(lam) @ np.abs(tl)), (c, lhs, rhs)
