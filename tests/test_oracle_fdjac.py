"""Pins of the oracle's forward-difference Jacobian (the alternative the paper measures the
analytical Jacobian against, Sec. 2.3) and of the Rosenbrock solve that uses it.

* the forward differences match the analytical (complex-step-pinned) Jacobian to the first-order
  truncation and rounding of the difference, 1e-4 row-normwise, on shear-layer states;
* the Rosenbrock solve with it stays within a few tolerance units of the analytical-Jacobian
  solve: with an inexact J the stages are those of a slightly different discrete method (the
  order conditions assume the exact J), so the step sequence and result move by O(tolerance).
"""
import numpy as np

import oracle as O
from paper_2105_12070_gb300 import synth


def _mech():
    w = synth.workload_shear_layer()
    return w, O.OracleMechanism(w["mech"].write_temp())


def test_fd_jacobian_matches_analytical():
    w, m = _mech()
    for c in (7, 20000, 40000, 65000):
        phi = np.concatenate([[w["T"][c]], w["Y"][:-1, c]])
        Jfd = m.jacobian_fd(w["p_Pa"], phi)
        Ja = m.jacobian(w["p_Pa"], phi[:1], np.concatenate([phi[1:], [1.0 - phi[1:].sum()]])[:, None])[0]
        rel = np.abs(Jfd - Ja).max(axis=1) / np.abs(Ja).max(axis=1)
        assert rel.max() <= 1e-4, (c, rel.max())


def test_integration_with_fd_jacobian_within_tolerance():
    w, m = _mech()
    idx = np.array([7, 40000])
    T, Y = w["T"][idx], w["Y"][:, idx]
    Ta, Ya, sta, _, _ = m.integrate(w["p_Pa"], T, Y, w["dt"])
    Tf, Yf, stf, _, _ = m.integrate(w["p_Pa"], T, Y, w["dt"], solver="rosenbrock_fdjac")
    assert np.all(sta == 0) and np.all(stf == 0)
    assert np.all(np.abs(Tf - Ta) <= 5 * (1e-6 * np.abs(Ta) + 1e-10))
    assert np.all(np.abs(Yf - Ya) <= 5 * (1e-6 * np.abs(Ya) + 1e-10))
