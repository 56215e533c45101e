"""Per-cell pressure (chem_integrate_varp) against the oracle run cell by cell at each cell's
pressure (Eq. 1 at constant pressure within a cell), and bit-identical to chem_integrate when
every cell has the same pressure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_varp_parity_and_uniform_case():
    w = synth.workload_small()
    path = w["mech"].write_temp()
    mech, om = chem.Mechanism(path), O.OracleMechanism(path)
    idx = np.arange(0, 256, 8)
    T, Y = w["T"][idx], w["Y"][:, idx]
    p = np.random.default_rng(9).uniform(0.5, 5.0, size=idx.shape[0]) * 101325.0
    Td, Yd = _dev(T), _dev(Y)
    st = torch.zeros(idx.shape[0], dtype=torch.int32, device="cuda")
    chem.chem_integrate_varp(mech, _dev(p), Td, Yd, w["dt"], status=st)
    torch.cuda.synchronize()
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for i in range(idx.shape[0]):
        To, Yo, sto, _, _ = om.integrate(p[i], T[i:i + 1], Y[:, i:i + 1], w["dt"])
        assert sto[0] == 0
        assert abs(Tg[i] - To[0]) <= 1e-6 * abs(To[0]) + 1e-10
        assert np.all(np.abs(Yg[:, i] - Yo[:, 0]) <= 1e-6 * np.abs(Yo[:, 0]) + 1e-10)
    # uniform pressure: the same result as the scalar entry point, bit for bit
    T1, Y1 = _dev(T), _dev(Y)
    chem.chem_integrate_varp(mech, _dev(np.full(idx.shape[0], w["p_Pa"])), T1, Y1, w["dt"])
    T2, Y2 = _dev(T), _dev(Y)
    chem.chem_integrate(mech, w["p_Pa"], T2, Y2, w["dt"])
    torch.cuda.synchronize()
    assert torch.equal(T1, T2) and torch.equal(Y1, Y2)


def test_varp_bad_pressure():
    w = synth.workload_small()
    mech = chem.Mechanism(w["mech"].write_temp())
    T, Y = w["T"][:4], w["Y"][:, :4]
    p = np.array([1e5, 0.0, np.nan, 2e5])
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    Td = _dev(T)
    chem.chem_integrate_varp(mech, _dev(p), Td, _dev(Y), w["dt"], status=st)
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 3, 3, 0]
    np.testing.assert_array_equal(Td.cpu().numpy()[[1, 2]], T[[1, 2]])
