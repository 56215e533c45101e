"""Pins of the oracle's discrete sensitivities (the tangent-linear model of the accepted
Rosenbrock steps, which the discrete adjoint of the integrator must transpose).

* replaying the recorded accepted step sizes reproduces the adaptive integration exactly;
* the tangent-linear result along a state direction and along a ln A direction equals central
  differences of the replay (the replay is a smooth function of both once the steps are fixed);
* on the A -> B -> C chain, the sensitivities of the Bateman solution with respect to ln k1,
  ln k2 and the initial Y_A are reproduced to the integration tolerance (closed forms).
"""
import os

import numpy as np

import oracle as O
from paper_2105_12070_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_cell(c):
    w = synth.workload_small()
    mech = O.OracleMechanism(w["mech"].write_temp())
    phi = np.concatenate([[w["T"][c]], w["Y"][:-1, c]])
    return mech, w["p_Pa"], phi, w["dt"]


def test_replay_reproduces_integrate():
    mech, p, phi, dt = _small_cell(5)
    out, hs, st = mech.integrate_record(p, phi, dt)
    assert st == 0 and hs.shape[0] > 10
    assert abs(hs.sum() - dt) <= 1e-12 * dt
    Yfull = np.concatenate([phi[1:], [1.0 - phi[1:].sum()]])
    T1, Y1, st1, steps, _ = mech.integrate(p, phi[:1], Yfull[:, None], dt)
    assert st1[0] == 0 and steps[0] == hs.shape[0]
    assert np.array_equal(out, np.concatenate([T1, Y1[:-1, 0]]))
    assert np.array_equal(mech.replay(p, phi, hs), out)


def test_tangent_linear_matches_central_differences():
    mech, p, phi, dt = _small_cell(9)
    _, hs, st = mech.integrate_record(p, phi, dt)
    assert st == 0
    rng = np.random.default_rng(4)
    dphi = rng.normal(size=mech.N) * np.maximum(np.abs(phi), 1e-6)
    dlnA = rng.normal(size=mech.R)
    for dx, dl in ((dphi, None), (None, dlnA), (dphi, dlnA)):
        _, tl = mech.replay(p, phi, hs, dphi=dx, dlnA=dl)
        eps = 1e-4  # the replay is smooth: truncation ~eps^2, roundoff ~1e-16/eps
        fwd = mech.replay(p, phi + eps * (dx if dx is not None else 0.0), hs,
                          lnA_shift=eps * dl if dl is not None else None)
        bwd = mech.replay(p, phi - eps * (dx if dx is not None else 0.0), hs,
                          lnA_shift=-eps * dl if dl is not None else None)
        fd = (fwd - bwd) / (2 * eps)
        assert np.max(np.abs(fd - tl)) <= 1e-6 * np.max(np.abs(tl)), (dx is None, dl is None)


def test_closed_form_chain_sensitivities():
    mech = O.OracleMechanism(os.path.join(GOLDEN, "chain_ABC.txt"))
    k1, k2, t = 2.0e5, 7.0e4, 2e-5
    phi = np.array([1200.0, 1.0, 0.0])
    _, hs, st = mech.integrate_record(1e5, phi, t, rtol=1e-12, atol=1e-20)
    assert st == 0
    e1, e2 = np.exp(-k1 * t), np.exp(-k2 * t)
    # d/d ln k1 and d/d ln k2 of Y_A = e^{-k1 t}, Y_B = k1/(k2-k1) (e^{-k1 t} - e^{-k2 t})
    dA_l1 = -k1 * t * e1
    dB_l1 = k1 * (k2 / (k2 - k1) ** 2 * (e1 - e2) + k1 / (k2 - k1) * (-t * e1))
    dB_l2 = k2 * (-k1 / (k2 - k1) ** 2 * (e1 - e2) + k1 / (k2 - k1) * (t * e2))
    _, d1 = mech.replay(1e5, phi, hs, dlnA=np.array([1.0, 0.0]))
    _, d2 = mech.replay(1e5, phi, hs, dlnA=np.array([0.0, 1.0]))
    _, da = mech.replay(1e5, phi, hs, dphi=np.array([0.0, 1.0, 0.0]))
    tol = 1e-8
    assert abs(d1[0]) < 1e-12 and abs(d2[0]) < 1e-12 and abs(da[0]) < 1e-12
    assert abs(d1[1] - dA_l1) <= tol and abs(d1[2] - dB_l1) <= tol
    assert abs(d2[1]) <= tol and abs(d2[2] - dB_l2) <= tol
    # the chain is linear in the initial amount of A
    assert abs(da[1] - e1) <= tol and abs(da[2] - k1 / (k2 - k1) * (e1 - e2)) <= tol


def test_jacobian_directional_derivative():
    """jacobian_dir: df = J d, and dJ equals central differences of the analytical Jacobian."""
    mech, p, phi, _ = _small_cell(11)
    rng = np.random.default_rng(7)
    d = rng.normal(size=mech.N) * np.maximum(np.abs(phi), 1e-6)
    f, J, df, dJ = mech.jacobian_dir(p, phi, dphi=d)
    T, Y = phi[:1], np.concatenate([phi[1:], [1.0 - phi[1:].sum()]])[:, None]
    np.testing.assert_array_equal(J, mech.jacobian(p, T, Y)[0])
    np.testing.assert_allclose(df, J @ d, rtol=1e-10, atol=1e-10 * np.abs(J @ d).max())
    eps = 1e-5

    def jac(x):
        return mech.jacobian(p, x[:1], np.concatenate([x[1:], [1.0 - x[1:].sum()]])[:, None])[0]

    fd = (jac(phi + eps * d) - jac(phi - eps * d)) / (2 * eps)
    assert np.max(np.abs(fd - dJ)) <= 1e-6 * np.max(np.abs(dJ))
