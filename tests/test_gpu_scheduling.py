"""Scheduling options of chem_integrate (the GPU counterpart of the paper's load balancing,
Sec. 2.2): results do not depend on how cells are scheduled, and the graph and batch paths give
the same answer as the plain launch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import autotune, chem, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    w = synth.workload_small()
    return w, chem.Mechanism(w["mech"].write_temp())


def _run(mech, w, opts, T=None, Y=None):
    T = torch.from_numpy((w["T"] if T is None else T).copy()).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(w["Y"] if Y is None else Y)).cuda()
    st = chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], opts=opts, want_stats=True)
    torch.cuda.synchronize()
    return T.cpu().numpy(), Y.cpu().numpy(), st


def test_graph_replay_and_batches_are_bitwise_equal(small):
    w, mech = small
    ref = _run(mech, w, chem.default_opts())
    for opts in (chem.default_opts(use_graph=1), chem.default_opts(use_graph=1),  # capture, then replay
                 chem.default_opts(batch_cells=37), chem.default_opts(batch_cells=64, use_queue=0),
                 chem.default_opts(batch_cells=100, use_graph=1), chem.default_opts(warps_per_cell=8)):
        T, Y, st = _run(mech, w, opts)
        np.testing.assert_array_equal(T, ref[0])
        np.testing.assert_array_equal(Y, ref[1])
        assert (st.steps, st.rejects) == (ref[2].steps, ref[2].rejects)


def test_graph_recaptures_on_new_arguments(small):
    w, mech = small
    a = _run(mech, w, chem.default_opts(use_graph=1), T=w["T"][:100], Y=w["Y"][:, :100])
    b = _run(mech, w, chem.default_opts(use_graph=1), T=w["T"][:50], Y=w["Y"][:, :50])
    c = _run(mech, w, chem.default_opts(), T=w["T"][:50], Y=w["Y"][:, :50])
    np.testing.assert_array_equal(b[0], c[0])
    np.testing.assert_array_equal(a[0][:50], c[0])


def test_autotune_returns_a_valid_shape(small, tmp_path):
    w, mech = small
    opts = autotune.autotune(mech, w["p_Pa"], w["T"], w["Y"], w["dt"], cache_path=str(tmp_path / "c.json"))
    assert opts.warps_per_cell in (1, 2, 4, 8) and opts.cells_per_cta >= 1
    again = autotune.autotune(mech, w["p_Pa"], w["T"], w["Y"], w["dt"], cache_path=str(tmp_path / "c.json"))
    assert (again.warps_per_cell, again.cells_per_cta) == (opts.warps_per_cell, opts.cells_per_cta)
    T, Y, st = _run(mech, w, opts)
    ref = _run(mech, w, chem.default_opts())
    np.testing.assert_array_equal(T, ref[0])


def test_uneven_field_mech100_parity_and_order_independence():
    """100 species / 700 reactions: sampled igniting, cold and burnt cells match the oracle, and
    the blocked and shuffled orders give each cell the same result."""
    w = synth.workload_uneven(200, "blocked")
    path = w["mech"].write_temp()
    mech = chem.Mechanism(path)
    ora = O.OracleMechanism(path)
    cls = w["cls"]
    idx = np.concatenate([np.where(cls == c)[0][:3] for c in (0, 1, 2)])
    T, Y = w["T"][idx], w["Y"][:, idx]
    Tg, Yg, st = _run(mech, w, chem.default_opts(), T=T, Y=Y)
    To, Yo, so, _, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], nthreads=16)
    assert st.failed_cells == 0 and np.all(so == 0)
    assert np.all(np.abs(Tg - To) <= 1e-6 * np.abs(To) + 1e-10)
    assert np.all(np.abs(Yg - Yo) <= 1e-6 * np.abs(Yo) + 1e-10)
    # the same cells in another position of a larger, reordered field give the same result
    perm = np.random.default_rng(1).permutation(200)
    Tall, Yall, st2 = _run(mech, w, chem.default_opts(), T=w["T"][perm], Y=w["Y"][:, perm])
    inv = np.argsort(perm)
    np.testing.assert_array_equal(Tall[inv][idx], Tg)
