"""Pins of the oracle's Seulex integrator (the paper's extrapolated linearly implicit Euler,
Sec. 2.3; Hairer & Wanner IV.9).

* closed-form kinetics: A = B isomerisation (elementary and Lindemann forms) and the A -> B -> C
  chain are reproduced to 10 rtol at rtol 1e-6 and to 1e-9 at rtol 1e-12;
* on the A -> B -> C chain (a linear system), column j of the tableau is the rational function
  (1 - z/n_j)^(-n_j) of z = H lambda, so the extrapolated value T_jj is accurate to order j:
  the observed error falls with tighter tolerance and the step count grows slowly (high order);
* an independent method pins the nonlinear case: Seulex and the 4-stage Rosenbrock method agree
  at tight tolerance on the 10-species mechanism;
* tolerance proportionality and the h carry-over.
"""
import os

import numpy as np

import oracle as O
from paper_2105_12070_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RC = 8.314462618 / 4.184
RU = 8.314462618e7


def _kf(A, b, Ea, T):
    return A * T ** b * np.exp(-Ea / (RC * T))


def _isomer(path, kf_eff):
    mech = O.OracleMechanism(path)
    T0 = np.array([1200.0, 1500.0, 900.0])
    Y = np.array([[0.9, 0.05, 0.5], [0.1, 0.95, 0.5]])
    p, dt = 2.0e5, 1e-5
    for rtol, bound in ((1e-6, None), (1e-12, 1e-9)):
        Tn, Yn, st, steps, rej = mech.integrate(p, T0, Y, dt, rtol=rtol, atol=1e-20 if rtol < 1e-8 else 1e-10,
                                                solver="seulex")
        assert np.all(st == 0)
        np.testing.assert_array_equal(Tn, T0)
        kf = kf_eff(T0, p)
        kr = kf / 4.0
        yeq = kr / (kf + kr)
        exact = yeq + (Y[0] - yeq) * np.exp(-(kf + kr) * dt)
        err = np.abs(Yn[0] - exact)
        if bound is None:
            assert np.all(err <= 10 * rtol * np.abs(exact) + 1e-10), err
        else:
            assert np.all(err <= bound), err


def test_closed_form_isomer():
    _isomer(os.path.join(GOLDEN, "isomer_AB.txt"), lambda T, p: _kf(3000.0, 0.5, 10000.0, T))


def test_closed_form_isomer_lindemann():
    def keff(T, p):
        kinf = _kf(1.0e5, 0.0, 2000.0, T)
        k0 = _kf(5.0e11, 0.0, 1000.0, T)
        M = 1.5 * (p * 10.0) / (RU * T)
        Pr = k0 * M / kinf
        return kinf * Pr / (1.0 + Pr)
    _isomer(os.path.join(GOLDEN, "isomer_AB_lindemann.txt"), keff)


def test_closed_form_chain_and_order():
    mech = O.OracleMechanism(os.path.join(GOLDEN, "chain_ABC.txt"))
    k1, k2 = 2.0e5, 7.0e4
    T0 = np.array([1000.0, 1700.0])
    Y = np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    dt = 4e-5
    ya = np.exp(-k1 * dt)
    yb = k1 / (k2 - k1) * (np.exp(-k1 * dt) - np.exp(-k2 * dt))
    exact = np.array([ya, yb, 1.0 - ya - yb])
    errs, steps = [], []
    for rtol in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12):
        Tn, Yn, st, nst, _ = mech.integrate(1e5, T0, Y, dt, rtol=rtol, atol=1e-20, solver="seulex")
        assert np.all(st == 0)
        e = np.max(np.abs(Yn - exact[:, None]) / np.maximum(np.abs(exact[:, None]), 1e-3))
        assert e <= 10 * rtol, (rtol, e)
        errs.append(e)
        steps.append(int(nst.max()))
    assert errs[-1] < 1e-9
    # a high-order method: eight orders of magnitude of tolerance cost well under a 10x step count
    assert steps[-1] < 10 * steps[0], steps


def test_agrees_with_rosenbrock_at_tight_tolerance():
    w = synth.workload_small()
    mech = O.OracleMechanism(w["mech"].write_temp())
    idx = np.arange(0, 256, 32)
    T, Y = w["T"][idx], w["Y"][:, idx]
    Ts, Ys, st, _, _ = mech.integrate(w["p_Pa"], T, Y, w["dt"], rtol=1e-10, atol=1e-16, solver="seulex",
                                      max_steps=400000)
    Tr, Yr, st2, _, _ = mech.integrate(w["p_Pa"], T, Y, w["dt"], rtol=1e-10, atol=1e-16, max_steps=400000)
    assert np.all(st == 0) and np.all(st2 == 0)
    np.testing.assert_allclose(Ts, Tr, rtol=1e-8)
    assert np.max(np.abs(Ys - Yr)) <= 1e-8


def test_tolerance_proportionality_and_carry_over():
    w = synth.workload_small()
    mech = O.OracleMechanism(w["mech"].write_temp())
    idx = np.arange(0, 256, 64)
    T, Y = w["T"][idx], w["Y"][:, idx]
    Tref, Yref, _, _, _ = mech.integrate(w["p_Pa"], T, Y, w["dt"], rtol=1e-11, atol=1e-17, max_steps=400000)
    errs = []
    for rtol in (1e-5, 1e-7, 1e-9):
        Tn, Yn, st, _, _ = mech.integrate(w["p_Pa"], T, Y, w["dt"], rtol=rtol, atol=rtol * 1e-4, solver="seulex")
        assert np.all(st == 0)
        errs.append(np.max(np.abs(Yn - Yref)))
    assert errs[0] > errs[1] > errs[2], errs
    # carry-over: a positive h_inout is the first step tried, and it is updated with the proposal
    h = np.full(idx.shape[0], 1e-7)
    mech.integrate(w["p_Pa"], T, Y, w["dt"], h_inout=h, solver="seulex")
    assert np.all(h > 0.0) and np.all(h != 1e-7)
