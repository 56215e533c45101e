"""The allocation-free integrate entry point (chem_integrate_noalloc) against chem_integrate.

chem_integrate_noalloc exists for callers that cannot allocate device memory while they run
(a flow solver that reserved all device memory for its own pool, a time loop that must not pay
the synchronisation of cudaMalloc/cudaFree); it keeps its scratch in a fixed array inside the
library.  This file is collected last so that a run stopping at the first failure has run every
other test; it passes both alone and after the rest.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_chem_integrate_on_two_calls():
    w = synth.workload_small()
    mech = chem.Mechanism(w["mech"].write_temp())
    n = w["T"].shape[0]
    # reference: the allocating entry point
    Tr, Yr = _dev(w["T"]), _dev(w["Y"])
    sr = torch.zeros(n, dtype=torch.int32, device="cuda")
    ref_stats = chem.chem_integrate(mech, w["p_Pa"], Tr, Yr, w["dt"], w["rtol"], w["atol"], status=sr, want_stats=True)
    steps_ref = torch.zeros(n, dtype=torch.int32, device="cuda")
    rej_ref = torch.zeros_like(steps_ref)
    chem.chem_last_cell_counters(mech, steps_ref, rej_ref)
    torch.cuda.synchronize()
    for call in range(2):  # two calls in a row share (and must reset) the fixed scratch
        T, Y = _dev(w["T"]), _dev(w["Y"])
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        steps = torch.zeros(n, dtype=torch.int32, device="cuda")
        rej = torch.zeros_like(steps)
        st = chem.chem_integrate_noalloc(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], status=status,
                                         steps=steps, rejects=rej, want_stats=True)
        torch.cuda.synchronize()
        Tn, Yn, Trn, Yrn = T.cpu().numpy(), Y.cpu().numpy(), Tr.cpu().numpy(), Yr.cpu().numpy()
        assert np.all(status.cpu().numpy() == 0)
        # the same kernel, launch shape and inputs: the results are bitwise those of chem_integrate
        # (a scratch that was not reset would show here, not hide inside a tolerance)
        np.testing.assert_array_equal(Tn, Trn)
        np.testing.assert_array_equal(Yn, Yrn)
        np.testing.assert_array_equal(steps.cpu().numpy(), steps_ref.cpu().numpy())
        np.testing.assert_array_equal(rej.cpu().numpy(), rej_ref.cpu().numpy())
        assert (st.steps, st.rejects, st.failed_cells) == (ref_stats.steps, ref_stats.rejects, ref_stats.failed_cells)


def test_noalloc_rejects_oversize_and_host_arrays():
    w = synth.workload_small()
    mech = chem.Mechanism(w["mech"].write_temp())
    big = 262144 + 1
    T = torch.full((big,), 1200.0, dtype=torch.float64, device="cuda")
    Y = torch.full((mech.K, big), 1.0 / mech.K, dtype=torch.float64, device="cuda")
    with pytest.raises(chem.ChemError, match="exceed"):
        chem.chem_integrate_noalloc(mech, w["p_Pa"], T, Y, w["dt"])
    with pytest.raises(chem.ChemError, match="device memory"):
        chem.chem_integrate_noalloc(mech, w["p_Pa"], w["T"][:4].copy(), np.ascontiguousarray(w["Y"][:, :4]), w["dt"])
