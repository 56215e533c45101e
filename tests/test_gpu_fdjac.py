"""The forward-difference Jacobian mode of the GPU Rosenbrock solve (opts.jacobian =
CHEM_JAC_FD) against the oracle's forward-difference mode: the same differences (step
2^-26 max(|phi_j|, s_j)) and the same method.  The two sides' rate values differ by rounding
(summation order), and a forward difference divides that by the step: for a trace species
(step 2^-26 1e-6) the columns differ by up to ~1e-2 relative.  An inexact Jacobian moves the
result by O(tolerance) (the oracle's FD-vs-analytical pin), so the bound is 5 tolerance units:
|x_gpu - x_oracle| <= 5 (1e-6 |x_oracle| + 1e-10) for T and every Y."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("which", ["small", "shear"])
def test_fd_jacobian_parity(which):
    w = synth.workload_small() if which == "small" else synth.workload_shear_layer()
    path = w["mech"].write_temp()
    mech, om = chem.Mechanism(path), O.OracleMechanism(path)
    n = w["T"].shape[0]
    idx = np.arange(0, n, 16) if which == "small" else np.linspace(0, n - 1, 24).astype(np.int64)
    T, Y = w["T"][idx], w["Y"][:, idx]
    Td, Yd = _dev(T), _dev(Y)
    status = torch.zeros(idx.shape[0], dtype=torch.int32, device="cuda")
    opts = chem.default_opts(jacobian=chem.CHEM_JAC_FD)
    chem.chem_integrate(mech, w["p_Pa"], Td, Yd, w["dt"], 1e-6, 1e-10, status=status, opts=opts)
    torch.cuda.synchronize()
    To, Yo, sto, _, _ = om.integrate(w["p_Pa"], T, Y, w["dt"], solver="rosenbrock_fdjac", nthreads=8)
    assert np.all(sto == 0) and np.all(status.cpu().numpy() == 0)
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    assert np.all(np.abs(Tg - To) <= 5 * (1e-6 * np.abs(To) + 1e-10))
    assert np.all(np.abs(Yg - Yo) <= 5 * (1e-6 * np.abs(Yo) + 1e-10))


def test_fd_jacobian_rejected_where_unsupported():
    w = synth.workload_small()
    mech = chem.Mechanism(w["mech"].write_temp())
    Td, Yd = _dev(w["T"][:2]), _dev(w["Y"][:, :2])
    with pytest.raises(chem.ChemError):
        chem.chem_integrate(mech, w["p_Pa"], Td, Yd, w["dt"],
                            opts=chem.default_opts(jacobian=chem.CHEM_JAC_FD, solver=chem.CHEM_SOLVER_SEULEX))
    rec = torch.empty((2, 8, mech.N + 1), dtype=torch.float64, device="cuda")
    ns = torch.empty(2, dtype=torch.int32, device="cuda")
    st = torch.empty(2, dtype=torch.int32, device="cuda")
    with pytest.raises(chem.ChemError):
        chem.chem_integrate_record(mech, w["p_Pa"], Td, Yd, w["dt"], rec, ns, st,
                                   opts=chem.default_opts(jacobian=chem.CHEM_JAC_FD))
