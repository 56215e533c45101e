"""Pins of the oracle's thermochemistry, rates and analytical Jacobian (Sec. 2.1 Eq. 1, Sec. 2.3).

* thermo: d(h/R)/dT = cp/R and d(s/R)/dT = cp/(R T) by complex step (a dropped or wrong NASA
  term breaks one of them);
* Jacobian: complex-step derivative of the rate function to 1e-12 row-normwise, and central
  finite differences (the paper's "Standard" Jacobian, Sec. 2.3) to ~1e-5;
* invariants of Eq. 1: element conservation, sum Y = 1 and constant mixture enthalpy under the
  adiabatic constant-pressure integration;
* equilibrium: the long-time state equals the Gibbs minimum found by an independent element-
  potential solve (pins Kc including its (Patm/(Ru T))^dnu factor), and every reversible
  reaction is in detailed balance there;
* fall-off: Pr -> inf gives kinf, Pr -> 0 gives k0 [M], and the Troe F equals Fcent at the
  centre log10 Pr = -c.
"""
import os

import numpy as np
import pytest
from scipy.optimize import fsolve

import oracle as O
from paper_2105_12070_gb300 import synth

RU = 8.314462618e7
RC = 8.314462618 / 4.184
PATM = 1.01325e6


@pytest.fixture(scope="module")
def small():
    m = synth.mechanism_small()
    return m, O.OracleMechanism(m.write_temp())


@pytest.fixture(scope="module")
def mech53():
    m = synth.mechanism_53()
    return m, O.OracleMechanism(m.write_temp())


def test_thermo_complex_step(small, mech53):
    for gen, ora in (small, mech53):
        for T in (350.0, 800.0, 999.0, 1001.0, 1500.0, 2600.0, 4000.0):
            cp, hRT, sR = ora.thermo(T)
            dhR, dsR = ora.thermo_cs(T)
            np.testing.assert_allclose(dhR, cp, rtol=1e-13, atol=0)
            np.testing.assert_allclose(dsR * T, cp, rtol=1e-12, atol=0)
        # the generator fitted continuous polynomials at Tmid: the oracle evaluates both sides
        lo = ora.thermo(1000.0)
        hi = ora.thermo(1000.0 + 1e-9)
        for a, b in zip(lo, hi):
            np.testing.assert_allclose(a, b, rtol=1e-9)


def _states(gen, n, seed, T_range=(900.0, 1800.0)):
    T, Y = synth.cells_uniform(seed, gen.K, n, T_range)
    return T, Y


@pytest.mark.parametrize("which", ["small", "mech53"])
def test_jacobian_complex_step(which, request):
    gen, ora = request.getfixturevalue(which)
    T, Y = _states(gen, 4, 7)
    for p in (1.01325e5, 4.0e6):
        J = ora.jacobian(p, T, Y)
        for c in range(len(T)):
            Jcs = ora.jacobian_cs(p, T[c], Y[:, c])
            scale = np.abs(Jcs).max(axis=1)
            err = np.abs(J[c] - Jcs).max(axis=1) / scale
            assert err.max() < 1e-12, err.max()


def test_jacobian_central_differences(small):
    gen, ora = small
    T, Y = _states(gen, 2, 8)
    p = 1.01325e5
    J = ora.jacobian(p, T, Y)
    N = ora.N
    for c in range(2):
        phi = np.concatenate([[T[c]], Y[:-1, c]])
        Jfd = np.zeros((N, N))
        for j in range(N):
            hstep = 1e-6 * max(abs(phi[j]), 1e-3)
            up, dn = phi.copy(), phi.copy()
            up[j] += hstep
            dn[j] -= hstep
            fu = ora.rates(p, up[:1], np.concatenate([up[1:], [1 - up[1:].sum()]])[:, None])[:, 0]
            fd = ora.rates(p, dn[:1], np.concatenate([dn[1:], [1 - dn[1:].sum()]])[:, None])[:, 0]
            Jfd[:, j] = (fu - fd) / (2 * hstep)
        err = np.abs(J[c] - Jfd).max(axis=1) / np.abs(J[c]).max(axis=1)
        assert err.max() < 1e-5, err.max()


def _element_totals(gen, Y):
    return gen.comp.T @ (Y / gen.W[:, None])  # mol of each element per gram


def _mix_enthalpy(ora, gen, T, Y):
    h = np.zeros(len(T))
    scale = np.zeros(len(T))
    for c in range(len(T)):
        _, hRT, _ = ora.thermo(T[c])
        hk = hRT * RU * T[c] / gen.W
        h[c] = (Y[:, c] * hk).sum()
        scale[c] = np.abs(Y[:, c] * hk).sum()
    return h, scale


@pytest.mark.parametrize("rtol,tol_h", [(1e-6, 2e-5), (1e-10, 1e-8)])
def test_invariants_small(small, rtol, tol_h):
    gen, ora = small
    w = synth.workload_small()
    n = 32
    T0, Y0 = w["T"][:n], w["Y"][:, :n]
    Tn, Yn, st, steps, _ = ora.integrate(w["p_Pa"], T0, Y0, w["dt"], rtol=rtol, atol=1e-10 * rtol / 1e-6,
                                         nthreads=4)
    assert np.all(st == 0)
    e0 = _element_totals(gen, Y0)
    e1 = _element_totals(gen, Yn)
    assert np.abs(e1 - e0).max() / np.abs(e0).max() < 1e-12
    assert np.abs(Yn.sum(0) - 1.0).max() < 1e-13
    h0, sc = _mix_enthalpy(ora, gen, T0, Y0)
    h1, _ = _mix_enthalpy(ora, gen, Tn, Yn)
    assert np.all(np.abs(h1 - h0) <= tol_h * sc), np.abs(h1 - h0) / sc
    assert np.abs(Tn - T0).max() > 10.0  # the test is not vacuous: chemistry happened


def test_invariants_mech53(mech53):
    gen, ora = mech53
    w = synth.workload_shear_layer(16)
    idx = np.arange(0, 256, 37)
    T0, Y0 = w["T"][idx], w["Y"][:, idx]
    Tn, Yn, st, _, _ = ora.integrate(w["p_Pa"], T0, Y0, 1e-7, nthreads=4)
    assert np.all(st == 0)
    e0 = _element_totals(gen, Y0)
    e1 = _element_totals(gen, Yn)
    assert np.abs(e1 - e0).max() / np.abs(e0).max() < 1e-12
    h0, sc = _mix_enthalpy(ora, gen, T0, Y0)
    h1, _ = _mix_enthalpy(ora, gen, Tn, Yn)
    assert np.all(np.abs(h1 - h0) <= 2e-5 * sc)


def _gibbs_equilibrium(ora, gen, T, p_cgs, b_el):
    """Ideal-gas Gibbs minimum at (T, p) for element totals b_el (mol/g), by the element-potential
    method: n_k = N exp(-g_k/RT - ln(p/Patm) + sum_e lambda_e a_ek), sum n_k = N, A n = b."""
    _, hRT, sR = ora.thermo(T)
    g = hRT - sR
    A = gen.comp.T.astype(float)
    E = A.shape[0]

    def resid(x):
        lam, lnN = x[:E], x[E]
        lnx = -g - np.log(p_cgs / PATM) + lam @ A
        xk = np.exp(lnx)
        n = np.exp(lnN) * xk
        return np.concatenate([(A @ n - b_el) / b_el, [xk.sum() - 1.0]])

    best = None
    for trial in range(20):
        x0 = np.concatenate([np.random.default_rng(trial).normal(0, 5, E) - 5, [np.log(b_el.sum())]])
        x, info, ier, _ = fsolve(resid, x0, full_output=True, xtol=1e-14)
        if ier == 1 and np.abs(resid(x)).max() < 1e-11:
            best = x
            break
    assert best is not None
    lam, lnN = best[:E], best[E]
    xk = np.exp(-g - np.log(p_cgs / PATM) + lam @ A)
    return xk


def test_equilibrium_and_detailed_balance(small):
    gen, ora = small
    w = synth.workload_small()
    c = 3
    p = w["p_Pa"]
    T0, Y0 = w["T"][c:c + 1], w["Y"][:, c:c + 1]
    Tn, Yn, st, _, _ = ora.integrate(p, T0, Y0, 10.0, rtol=1e-11, atol=1e-22)
    assert st[0] == 0
    # mole fractions of the integrated long-time state
    x_int = (Yn[:, 0] / gen.W) / (Yn[:, 0] / gen.W).sum()
    x_eq = _gibbs_equilibrium(ora, gen, Tn[0], p * 10.0, _element_totals(gen, Yn)[:, 0])
    big = x_eq > 1e-8
    np.testing.assert_allclose(x_int[big], x_eq[big], rtol=1e-6)
    kf, kr, qf, qr = ora.reaction_rates(p, Tn[0], Yn[:, 0])
    assert np.all(np.abs(qf - qr) <= 1e-7 * np.maximum(qf, qr) + 1e-300)


def _falloff_mech(troe, params="0.6 200.0 1200.0 5000.0"):
    extra = f"troe {params}\n" if troe else ""
    rtype = 3 if troe else 2
    txt = ("CHEMMECH 1\nelements 1\nX 20.0\nspecies 2\n"
           "A 20.0 300.0 1000.0 5000.0 1 3.5 0 0 0 0 -1000.0 10.0 3.5 0 0 0 0 -1000.0 10.0\n"
           "B 20.0 300.0 1000.0 5000.0 1 3.5 0 0 0 0 -1000.0 11.0 3.5 0 0 0 0 -1000.0 11.0\n"
           f"reactions 1\n{rtype} 1 0 -1 1 1 -1 1.0e6 0.3 3000.0\neff 1.0 1.0\nlow 1.0e13 -0.5 1000.0\n{extra}end\n")
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".txt")
    os.write(fd, txt.encode())
    os.close(fd)
    return path


def test_troe_broadening_width():
    """The width of Troe's broadening curve (Gilbert, Luther & Troe 1983, the CHEMKIN form).  In
    u = log10 Pr + c the curve is log10 F = log10 Fcent / (1 + f^2), f = u / (n - d u).  Solving
    f = +1 and f = -1 by hand gives the two half-depth points u = n / (1 + d) and u = -n / (1 - d),
    where F = Fcent^(1/2) exactly, 2 n / (1 - d^2) apart; f = +-2 gives u = 2n / (1 + 2d) and
    -2n / (1 - 2d), where F = Fcent^(1/5).  The oracle's rate constants are evaluated at the
    pressures that put log10 Pr there, over several broadening centres.  The width
    n = 0.75 - 1.27 log10 Fcent and the slope d = 0.14 set where these points lie, so a wrong sign
    or term in either moves them off (planted mistakes 11 and 12)."""
    T = 1300.0
    Y = np.array([0.3, 0.7])
    kinf = 1.0e6 * T ** 0.3 * np.exp(-3000.0 / (RC * T))
    k0 = 1.0e13 * T ** -0.5 * np.exp(-1000.0 / (RC * T))
    d = 0.14
    for a, T3, T1, T2 in ((0.6, 200.0, 1200.0, 5000.0), (0.2, 100.0, 3000.0, 9000.0), (0.9, 800.0, 800.0, 2000.0)):
        ora = O.OracleMechanism(_falloff_mech(True, f"{a} {T3} {T1} {T2}"))
        Fcent = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + np.exp(-T2 / T)
        L = np.log10(Fcent)
        c = -0.4 - 0.67 * L
        n = 0.75 - 1.27 * L
        for u, power in ((n / (1 + d), 0.5), (-n / (1 - d), 0.5), (2 * n / (1 + 2 * d), 0.2),
                         (-2 * n / (1 - 2 * d), 0.2)):
            Pr = 10.0 ** (u - c)
            p = Pr * kinf / k0 * RU * T / 10.0  # [M] = p / (Ru T) with p in dyn/cm^2, efficiencies 1
            kf = ora.reaction_rates(p, T, Y)[0][0]
            F = kf / (kinf * Pr / (1 + Pr))
            assert abs(np.log10(F) / L - power) < 1e-10, (a, u, power, np.log10(F) / L)


@pytest.mark.parametrize("troe", [False, True])
def test_falloff_limits(troe):
    ora = O.OracleMechanism(_falloff_mech(troe))
    T = 1300.0
    Y = np.array([0.3, 0.7])
    kinf = 1.0e6 * T ** 0.3 * np.exp(-3000.0 / (RC * T))
    k0 = 1.0e13 * T ** -0.5 * np.exp(-1000.0 / (RC * T))
    if not troe:
        # high pressure: k -> kinf;  low pressure: k -> k0 [M]
        kf_hi = ora.reaction_rates(1e16, T, Y)[0][0]
        assert abs(kf_hi / kinf - 1.0) < 1e-4
        p_lo = 1e-8
        M = p_lo * 10.0 / (RU * T)
        kf_lo = ora.reaction_rates(p_lo, T, Y)[0][0]
        assert abs(kf_lo / (k0 * M) - 1.0) < 1e-4
    else:
        # Fcent -> 1 (alpha = 1, T1 and T2 -> inf) reduces Troe to Lindemann at every pressure
        lind = O.OracleMechanism(_falloff_mech(False))
        flat = O.OracleMechanism(_falloff_mech(True, "1.0 200.0 1e300 1e300"))
        for p in (1e-2, 1e3, 1e5, 1e7, 1e9):
            a = lind.reaction_rates(p, T, Y)[0][0]
            b = flat.reaction_rates(p, T, Y)[0][0]
            assert abs(a / b - 1.0) < 1e-14
        a, T3, T1, T2 = 0.6, 200.0, 1200.0, 5000.0
        Fcent = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + np.exp(-T2 / T)
        c = -0.4 - 0.67 * np.log10(Fcent)
        Pr = 10.0 ** (-c)
        M = Pr * kinf / k0
        p = M * RU * T / 10.0
        kf = ora.reaction_rates(p, T, Y)[0][0]
        F = kf / (kinf * Pr / (1 + Pr))
        assert abs(F / Fcent - 1.0) < 1e-12
        # off-centre the broadening is between Fcent and 1
        kf2 = ora.reaction_rates(p * 100, T, Y)[0][0]
        F2 = kf2 / (kinf * 100 * Pr / (1 + 100 * Pr))
        assert Fcent < F2 < 1.0
