"""Pins of the oracle's zonal reference-cell mapping (Sec. 2.2, DLBFoam's mapping of ambient
cells): with no cell inside a zone it is the plain integration; a cell that is an exact copy of
a reference state gets exactly the reference's solution; and on the shear layer, cells within
1e-9 of an unmixed stream get a result within the integration tolerance of their own solve."""
import numpy as np

import oracle as O
from paper_2105_12070_gb300 import synth


def _shear(idx):
    w = synth.workload_shear_layer()
    (Tf, Yf), (To, Yo) = w["streams"]
    refs = np.array([np.concatenate([[Tf], Yf]), np.concatenate([[To], Yo])])
    return w, O.OracleMechanism(w["mech"].write_temp()), w["T"][idx], w["Y"][:, idx], refs


def test_no_zone_is_plain_integration():
    w = synth.workload_small()
    m = O.OracleMechanism(w["mech"].write_temp())
    idx = np.arange(0, 256, 32)
    T, Y = w["T"][idx], w["Y"][:, idx]
    ref = np.concatenate([[5000.0], np.full(m.K, 1.0 / m.K)])[None, :]
    Tn, Yn, st, zone = m.integrate_mapped(w["p_Pa"], T, Y, w["dt"], ref, 0.0, 0.0)
    Tp, Yp, stp, _, _ = m.integrate(w["p_Pa"], T, Y, w["dt"])
    assert np.all(zone == -1)
    np.testing.assert_array_equal(Tn, Tp)
    np.testing.assert_array_equal(Yn, Yp)


def test_exact_copies_get_the_reference_solution():
    w = synth.workload_small()
    m = O.OracleMechanism(w["mech"].write_temp())
    T = np.array([w["T"][3], w["T"][3], w["T"][9]])
    Y = np.stack([w["Y"][:, 3], w["Y"][:, 3], w["Y"][:, 9]], axis=1)
    ref = np.concatenate([[w["T"][3]], w["Y"][:, 3]])[None, :]
    Tn, Yn, st, zone = m.integrate_mapped(w["p_Pa"], T, Y, w["dt"], ref, 0.0, 0.0)
    Tp, Yp, _, _, _ = m.integrate(w["p_Pa"], T[:1], Y[:, :1], w["dt"])
    assert list(zone) == [0, 0, -1]
    np.testing.assert_allclose(Tn[:2], Tp[0], rtol=1e-15)
    np.testing.assert_allclose(Yn[:-1, :2], np.repeat(Yp[:-1], 2, axis=1), rtol=0, atol=1e-16)
    assert np.all(np.abs(Yn.sum(axis=0) - 1.0) <= 1e-14)


def test_ambient_cells_within_tolerance_of_their_own_solve():
    idx = np.array([5, 300, 65000, 65300])  # far from the layer on both sides
    w, m, T, Y, refs = _shear(idx)
    Tn, Yn, st, zone = m.integrate_mapped(w["p_Pa"], T, Y, w["dt"], refs, 1e-6, 1e-9)
    assert np.all(zone >= 0) and np.all(st == 0)
    Tp, Yp, _, _, _ = m.integrate(w["p_Pa"], T, Y, w["dt"])
    assert np.all(np.abs(Tn - Tp) <= 1e-6 * np.abs(Tp) + 1e-10)
    assert np.all(np.abs(Yn - Yp) <= 1e-6 * np.abs(Yp) + 1e-10)
