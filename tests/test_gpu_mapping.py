"""Zonal reference-cell mapping on the GPU (chem_integrate_mapped) against the oracle's mapping
(Sec. 2.2, DLBFoam's mapping of ambient cells), through the C ABI.

* the zone of every cell (an integer decision on the same doubles) is bit-exact;
* solved cells are bit-identical to chem_integrate on the same cells (the per-cell solve does
  not depend on where the cell sits in the launch);
* mapped cells match the oracle's mapping and their own full solve within the integrate
  tolerance 1e-6 |x| + 1e-10 (their state is within 1e-9 of the reference's).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def shear():
    w = synth.workload_shear_layer()
    path = w["mech"].write_temp()
    (Tf, Yf), (To, Yo) = w["streams"]
    refs = np.array([np.concatenate([[Tf], Yf]), np.concatenate([[To], Yo])])
    return w, chem.Mechanism(path), O.OracleMechanism(path), refs


def _mapped(mech, w, T, Y, refs, tT, tY):
    Td, Yd = _dev(T), _dev(Y)
    n = T.shape[0]
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    zone = torch.zeros(n, dtype=torch.int32, device="cuda")
    h = torch.zeros(n, dtype=torch.float64, device="cuda")
    nm, _ = chem.chem_integrate_mapped(mech, w["p_Pa"], Td, Yd, w["dt"], refs, tT, tY, h_inout=h, status=status,
                                       zone=zone)
    torch.cuda.synchronize()
    return Td.cpu().numpy(), Yd.cpu().numpy(), status.cpu().numpy(), zone.cpu().numpy(), nm


def test_mapping_parity(shear):
    w, mech, om, refs = shear
    idx = np.linspace(0, w["T"].shape[0] - 1, 192).astype(np.int64)
    T, Y = w["T"][idx], w["Y"][:, idx]
    Tg, Yg, st, zone, nm = _mapped(mech, w, T, Y, refs, 1e-6, 1e-9)
    To, Yo, sto, zo = om.integrate_mapped(w["p_Pa"], T, Y, w["dt"], refs, 1e-6, 1e-9, nthreads=8)
    np.testing.assert_array_equal(zone, zo)
    assert nm == int((zo >= 0).sum()) and 0 < nm < idx.shape[0]
    assert np.all(st == 0) and np.all(sto == 0)
    assert np.all(np.abs(Tg - To) <= 1e-6 * np.abs(To) + 1e-10)
    assert np.all(np.abs(Yg - Yo) <= 1e-6 * np.abs(Yo) + 1e-10)
    # solved cells: bit-identical to the plain solve of the same cells
    solved = np.nonzero(zone < 0)[0]
    Tp, Yp = _dev(T[solved]), _dev(Y[:, solved])
    chem.chem_integrate(mech, w["p_Pa"], Tp, Yp, w["dt"], w["rtol"], w["atol"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Tg[solved], Tp.cpu().numpy())
    np.testing.assert_array_equal(Yg[:, solved], Yp.cpu().numpy())
    # mapped cells: within tolerance of their own full solve
    mapped = np.nonzero(zone >= 0)[0]
    Tf, Yf = _dev(T[mapped]), _dev(Y[:, mapped])
    chem.chem_integrate(mech, w["p_Pa"], Tf, Yf, w["dt"], w["rtol"], w["atol"])
    torch.cuda.synchronize()
    Tf, Yf = Tf.cpu().numpy(), Yf.cpu().numpy()
    assert np.all(np.abs(Tg[mapped] - Tf) <= 1e-6 * np.abs(Tf) + 1e-10)
    assert np.all(np.abs(Yg[:, mapped] - Yf) <= 1e-6 * np.abs(Yf) + 1e-10)


def test_mapping_edge_cases(shear):
    w, mech, om, refs = shear
    idx = np.arange(0, 64)
    T, Y = w["T"][idx].copy(), w["Y"][:, idx].copy()
    # no references: the plain solve
    Tg, Yg, st, zone, nm = _mapped(mech, w, T, Y, np.zeros((0, mech.K + 1)), 0.0, 0.0)
    Tp, Yp = _dev(T), _dev(Y)
    chem.chem_integrate(mech, w["p_Pa"], Tp, Yp, w["dt"], w["rtol"], w["atol"])
    torch.cuda.synchronize()
    assert nm == 0 and np.all(zone == -1)
    np.testing.assert_array_equal(Tg, Tp.cpu().numpy())
    # a non-finite cell is never mapped and reports bad input; every cell mapped also works
    T[3] = np.nan
    Tg, Yg, st, zone, nm = _mapped(mech, w, T, Y, refs, 1e-6, 1e-9)
    assert zone[3] == -1 and st[3] == 3
    Tg, Yg, st, zone, nm = _mapped(mech, w, np.full(8, refs[1, 0]), np.repeat(refs[1, 1:, None], 8, axis=1),
                                   refs, 0.0, 0.0)
    assert nm == 8 and np.all(zone == 1) and np.all(st == 0)
    assert np.all(Tg == Tg[0])
