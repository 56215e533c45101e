"""The library's CHEMKIN-II reader on the GPU: rates and integration from a CHEMKIN file against
the oracle reading the same file with its own reader (rates to 1e-11 of the gross flux, the
integrate tolerance 1e-6 |x| + 1e-10 for T and Y)."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import chem, synth

import test_chemkin as ck

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_chemkin_rates_toy_mechanism():
    path = ck._write(ck._toy_chemkin(), ".ck")
    mech, om = chem.Mechanism(path), O.OracleMechanism(path)
    rng = np.random.default_rng(4)
    T = rng.uniform(800.0, 2000.0, size=64)
    Y = rng.dirichlet(np.ones(4), size=64).T.copy()
    out = torch.empty((4, 64), dtype=torch.float64, device="cuda")
    chem.chem_rates(mech, 2e5, _dev(T), _dev(Y), out)
    torch.cuda.synchronize()
    f, g = om.rates(2e5, T, Y, gross=True)
    assert np.all(np.abs(out.cpu().numpy() - f) <= 1e-11 * g)


def test_chemkin_integrate_small_mechanism():
    m = synth.mechanism_small().rounded()
    path = m.write_chemkin(ck._write("", ".ck"))
    mech, om = chem.Mechanism(path), O.OracleMechanism(path)
    w = synth.workload_small()
    idx = np.arange(0, 256, 8)
    T, Y = w["T"][idx], w["Y"][:, idx]
    Td, Yd = _dev(T), _dev(Y)
    st = torch.zeros(idx.shape[0], dtype=torch.int32, device="cuda")
    chem.chem_integrate(mech, w["p_Pa"], Td, Yd, w["dt"], status=st)
    torch.cuda.synchronize()
    To, Yo, so, _, _ = om.integrate(w["p_Pa"], T, Y, w["dt"], nthreads=8)
    assert np.all(so == 0) and np.all(st.cpu().numpy() == 0)
    assert np.all(np.abs(Td.cpu().numpy() - To) <= 1e-6 * np.abs(To) + 1e-10)
    assert np.all(np.abs(Yd.cpu().numpy() - Yo) <= 1e-6 * np.abs(Yo) + 1e-10)
