"""Pins of the oracle's Rosenbrock integrator (Sec. 2.3, Eq. 2 in its Rosenbrock form).

* the coefficient table satisfies the Rosenbrock order conditions (Hairer & Wanner, Solving
  ODEs II, Table IV.7.1) up to order 4, and its embedded weights up to order 3;
* the stability function has R(inf) = 0 (L-stable) and |R(iy)| <= 1 (A-stable);
* closed-form kinetics: A = B isomerisation (elementary, third-body and Lindemann forms) and the
  A -> B -> C chain are reproduced to 10 rtol at rtol 1e-6 and to 1e-9 at rtol 1e-12.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RC = 8.314462618 / 4.184
RU = 8.314462618e7


def _order_residuals(alpha, gam, b, g):
    """Order conditions for (I - g h J) k_i = h f(y + sum alpha_ij k_j) + h J sum gam_ij k_j."""
    beta = alpha + gam
    one = np.ones(4)
    ai = alpha @ one
    bi = beta @ one
    return np.array([
        b @ one - 1.0,
        b @ bi - (0.5 - g),
        b @ ai ** 2 - 1.0 / 3.0,
        b @ beta @ bi - (1.0 / 6.0 - g + g * g),
        b @ ai ** 3 - 0.25,
        b @ (ai * (alpha @ bi)) - (1.0 / 8.0 - g / 3.0),
        b @ beta @ ai ** 2 - (1.0 / 12.0 - g / 3.0),
        b @ beta @ beta @ bi - (1.0 / 24.0 - g / 2.0 + 1.5 * g * g - g ** 3),
    ])


def test_order_conditions():
    g, alpha, gam, b, bhat = O.ros_coefficients()
    assert np.all(np.triu(alpha) == 0) and np.all(np.triu(gam) == 0)
    assert np.abs(_order_residuals(alpha, gam, b, g)).max() < 1e-14
    emb = _order_residuals(alpha, gam, bhat, g)
    assert np.abs(emb[:4]).max() < 1e-14  # order 3
    assert np.abs(emb[4:]).max() > 1e-3  # and genuinely not order 4 (a distinct estimate)
    # stage 4 reuses stage 3's argument, so one rate evaluation per step is saved
    np.testing.assert_array_equal(alpha[3], alpha[2])


def _stability(alpha, gam, weights, g, z):
    B = alpha + gam + g * np.eye(4)
    return 1.0 + z * weights @ np.linalg.solve(np.eye(4) - z * B, np.ones(4))


def test_l_and_a_stability():
    g, alpha, gam, b, bhat = O.ros_coefficients()
    B = alpha + gam + g * np.eye(4)
    r_inf = 1.0 - b @ np.linalg.solve(B, np.ones(4))
    rhat_inf = 1.0 - bhat @ np.linalg.solve(B, np.ones(4))
    assert abs(r_inf) < 1e-13
    assert abs(rhat_inf - 0.5) < 1e-13
    for y in np.logspace(-3, 8, 500):
        assert abs(_stability(alpha, gam, b, g, 1j * y)) <= 1.0 + 1e-12
    for x in -np.logspace(-3, 8, 200):
        assert abs(_stability(alpha, gam, b, g, x)) <= 1.0 + 1e-12
    # matches exp(z) to order 4 near 0
    z = 1e-2
    assert abs(_stability(alpha, gam, b, g, z) - np.exp(z)) < 1e-10 * 10


def _kf(A, b, Ea, T):
    return A * T ** b * np.exp(-Ea / (RC * T))


def _isomer_case(path, kf_eff):
    mech = O.OracleMechanism(path)
    T0 = np.array([1200.0, 1500.0, 900.0])
    Y = np.array([[0.9, 0.05, 0.5], [0.1, 0.95, 0.5]])
    p = 2.0e5
    dt = 1e-5
    out = {}
    for rtol in (1e-6, 1e-12):
        Tn, Yn, st, steps, rej = mech.integrate(p, T0, Y, dt, rtol=rtol, atol=1e-20 if rtol < 1e-8 else 1e-10)
        assert np.all(st == 0)
        np.testing.assert_array_equal(Tn, T0)  # dH = 0: the temperature equation is exactly zero
        kf = kf_eff(T0, p)
        kr = kf / 4.0
        yeq = kr / (kf + kr)
        exact = yeq + (Y[0] - yeq) * np.exp(-(kf + kr) * dt)
        out[rtol] = np.abs(Yn[0] - exact)
        assert np.allclose(Yn.sum(0), 1.0, atol=1e-15, rtol=0)
    assert np.all(out[1e-6] <= 10 * 1e-6 * np.abs(Yn[0]) + 1e-10), out
    assert np.all(out[1e-12] <= 1e-9), out
    return out


def test_closed_form_isomer_elementary():
    _isomer_case(os.path.join(GOLDEN, "isomer_AB.txt"), lambda T, p: _kf(3000.0, 0.5, 10000.0, T))


def test_closed_form_isomer_third_body():
    # [M] = 2 * total concentration = 2 p / (Ru T) in mol/cm^3 (p in dyn/cm^2)
    _isomer_case(os.path.join(GOLDEN, "isomer_AB_third_body.txt"),
                 lambda T, p: _kf(2.0e10, 0.0, 5000.0, T) * 2.0 * (p * 10.0) / (RU * T))


def test_closed_form_isomer_lindemann():
    def keff(T, p):
        kinf = _kf(1.0e5, 0.0, 2000.0, T)
        k0 = _kf(5.0e11, 0.0, 1000.0, T)
        M = 1.5 * (p * 10.0) / (RU * T)
        Pr = k0 * M / kinf
        return kinf * Pr / (1.0 + Pr)
    _isomer_case(os.path.join(GOLDEN, "isomer_AB_lindemann.txt"), keff)


def test_closed_form_chain():
    mech = O.OracleMechanism(os.path.join(GOLDEN, "chain_ABC.txt"))
    k1, k2 = 2.0e5, 7.0e4
    T0 = np.array([1000.0, 1700.0])
    Y = np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    for dt in (1e-6, 1e-5, 4e-5):
        for rtol, tol in ((1e-6, 1e-5), (1e-12, 1e-9)):
            Tn, Yn, st, _, _ = mech.integrate(1e5, T0, Y, dt, rtol=rtol, atol=1e-20 if rtol < 1e-8 else 1e-10)
            assert np.all(st == 0)
            ya = np.exp(-k1 * dt)
            yb = k1 / (k2 - k1) * (np.exp(-k1 * dt) - np.exp(-k2 * dt))
            exact = np.array([ya, yb, 1.0 - ya - yb])
            err = np.abs(Yn - exact[:, None])
            assert np.all(err <= tol * np.maximum(np.abs(exact[:, None]), 1e-3)), (dt, rtol, err)


def test_tolerance_proportionality():
    """The global error on the closed-form case shrinks with rtol (the controller works)."""
    mech = O.OracleMechanism(os.path.join(GOLDEN, "chain_ABC.txt"))
    k1, k2, dt = 2.0e5, 7.0e4, 4e-5
    yb = k1 / (k2 - k1) * (np.exp(-k1 * dt) - np.exp(-k2 * dt))
    errs = []
    for rtol in (1e-4, 1e-6, 1e-8):
        _, Yn, _, steps, _ = mech.integrate(1e5, np.array([1300.0]), np.array([[1.0], [0.0], [0.0]]), dt,
                                            rtol=rtol, atol=1e-20)
        errs.append(abs(Yn[1, 0] - yb) / yb)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-7
