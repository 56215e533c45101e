"""GPU path vs the CPU oracle, through the C ABI (Sec. 2.1 Eq. 1; Sec. 2.3 Eq. 2).

Tolerances (stated from the arithmetic):
  * rates f: |f_gpu - f_oracle| <= 1e-11 * gross flux scale of the component (the sum of
    |forward| + |reverse| fluxes that enter it).  Both sides round exp() of arguments up to a
    few hundred and sum in different orders, so the error is a few 1e-14 of the gross flux;
    near partial equilibrium the net rate can be many orders below the gross scale.
  * Jacobian: |J_gpu - J_oracle| <= 1e-12 * max_j |J_oracle(i, j)| per row (row-normwise), the
    stated gate for Jacobian entries.
  Both tests print the measured maximum (and 99th percentile) of their error measure.
  * integrate: |x_gpu - x_oracle| <= 1e-6 |x_oracle| + 1e-10 for T and every Y (rtol/atol-shaped),
    the same adaptive method and controller on both sides.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-6, 1e-10


@pytest.fixture(scope="module")
def small():
    w = synth.workload_small()
    path = w["mech"].write_temp()
    return w, chem.Mechanism(path), O.OracleMechanism(path)


@pytest.fixture(scope="module")
def shear():
    w = synth.workload_shear_layer()
    path = w["mech"].write_temp()
    return w, chem.Mechanism(path), O.OracleMechanism(path)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_rates(mech, p, T, Y):
    out = torch.empty((mech.N, T.shape[0]), dtype=torch.float64, device="cuda")
    chem.chem_rates(mech, p, _dev(T), _dev(Y), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _gpu_jac(mech, p, T, Y):
    out = torch.empty((T.shape[0], mech.N, mech.N), dtype=torch.float64, device="cuda")
    chem.chem_jacobian(mech, p, _dev(T), _dev(Y), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _gpu_integrate(mech, w, T, Y, dt=None, opts=None, h=None):
    Td, Yd = _dev(T), _dev(Y)
    status = torch.zeros(T.shape[0], dtype=torch.int32, device="cuda")
    hd = _dev(h) if h is not None else None
    st = chem.chem_integrate(mech, w["p_Pa"], Td, Yd, dt or w["dt"], w["rtol"], w["atol"], h_inout=hd,
                             status=status, opts=opts, want_stats=True)
    torch.cuda.synchronize()
    steps = torch.zeros_like(status)
    rej = torch.zeros_like(status)
    chem.chem_last_cell_counters(mech, steps, rej)
    return (Td.cpu().numpy(), Yd.cpu().numpy(), status.cpu().numpy(), st, steps.cpu().numpy(),
            hd.cpu().numpy() if hd is not None else None)


def _sample_shear(n=64, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(65536, size=n, replace=False))


@pytest.mark.parametrize("which", ["small", "shear"])
def test_rates_parity(which, request):
    w, mech, ora = request.getfixturevalue(which)
    idx = np.arange(256) if which == "small" else _sample_shear(256)
    T, Y = w["T"][idx], w["Y"][:, idx]
    f = _gpu_rates(mech, w["p_Pa"], T, Y)
    fo, gross = ora.rates(w["p_Pa"], T, Y, gross=True)
    err = np.abs(f - fo)
    rel = err / np.maximum(gross, 1e-300)
    print(f"rates parity {which}: max |f_gpu - f_oracle| / gross {rel.max():.3e}, p99 {np.percentile(rel, 99):.3e}")
    assert np.all(err <= 1e-11 * gross + 1e-300), rel.max()


@pytest.mark.parametrize("which", ["small", "shear"])
def test_jacobian_parity(which, request):
    w, mech, ora = request.getfixturevalue(which)
    idx = np.arange(0, 256, 8) if which == "small" else _sample_shear(32, 1)
    T, Y = w["T"][idx], w["Y"][:, idx]
    J = _gpu_jac(mech, w["p_Pa"], T, Y)
    Jo = ora.jacobian(w["p_Pa"], T, Y)
    rowmax = np.abs(Jo).max(axis=2, keepdims=True)
    rel = np.abs(J - Jo) / rowmax
    worst = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"jacobian parity {which}: max row-normwise {rel.max():.3e} (cell {worst[0]}, row {worst[1]}), "
          f"p99 {np.percentile(rel, 99):.3e}")
    assert rel.max() <= 1e-12, rel.max()


def _assert_state_close(T, Y, To, Yo):
    assert np.all(np.abs(T - To) <= RTOL * np.abs(To) + ATOL), np.abs(T - To).max()
    err = np.abs(Y - Yo) - (RTOL * np.abs(Yo) + ATOL)
    assert np.all(err <= 0), err.max()


def test_integrate_parity_small(small):
    w, mech, ora = small
    T, Y = w["T"], w["Y"]
    Tg, Yg, sg, stats, steps, _ = _gpu_integrate(mech, w, T, Y)
    To, Yo, so, steps_o, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], nthreads=8)
    assert np.all(sg == 0) and np.all(so == 0)
    _assert_state_close(Tg, Yg, To, Yo)
    assert stats.steps == steps.sum() and stats.failed_cells == 0
    # the same controller takes the same decisions except within roundoff of err == 1
    assert np.mean(steps == steps_o) > 0.9


def test_integrate_parity_shear_sample(shear):
    w, mech, ora = shear
    idx = _sample_shear(24, 2)
    T, Y = w["T"][idx], w["Y"][:, idx]
    Tg, Yg, sg, stats, steps, _ = _gpu_integrate(mech, w, T, Y)
    To, Yo, so, steps_o, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], nthreads=16)
    assert np.all(sg == 0) and np.all(so == 0)
    _assert_state_close(Tg, Yg, To, Yo)


def test_ragged_and_empty(small):
    w, mech, ora = small
    for n in (1, 5, 37):
        T, Y = w["T"][:n], w["Y"][:, :n]
        Tg, Yg, sg, _, _, _ = _gpu_integrate(mech, w, T, Y)
        To, Yo, so, _, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"])
        _assert_state_close(Tg, Yg, To, Yo)
    T0 = torch.zeros(0, dtype=torch.float64, device="cuda")
    Y0 = torch.zeros((mech.K, 0), dtype=torch.float64, device="cuda")
    chem.chem_integrate(mech, w["p_Pa"], T0, Y0, w["dt"])


def test_bad_input_and_max_steps(small):
    w, mech, _ = small
    T, Y = w["T"][:8].copy(), w["Y"][:, :8].copy()
    T[1] = np.nan
    T[2] = -5.0
    Y[3, 4] = np.inf
    Tg, Yg, sg, stats, _, _ = _gpu_integrate(mech, w, T, Y)
    assert list(sg[[1, 2, 4]]) == [3, 3, 3]
    assert np.all(sg[[0, 3, 5, 6, 7]] == 0)
    assert Tg[2] == -5.0 and np.isinf(Yg[3, 4])
    assert stats.failed_cells == 3
    opts = chem.default_opts(max_steps=2)
    _, _, sg, _, _, _ = _gpu_integrate(mech, w, w["T"][:8], w["Y"][:, :8], opts=opts)
    assert np.all(sg == 1)
    # the context is still usable after the failed cells
    _gpu_rates(mech, w["p_Pa"], w["T"][:4], w["Y"][:, :4])


def test_host_pointers_match_device(small):
    w, mech, _ = small
    T, Y = w["T"][:64].copy(), w["Y"][:, :64].copy()
    Tg, Yg, _, _, _, _ = _gpu_integrate(mech, w, T, Y)
    status = np.zeros(64, np.int32)
    chem.chem_integrate(mech, w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], status=status)
    np.testing.assert_array_equal(T, Tg)
    np.testing.assert_array_equal(Y, Yg)
    f = np.zeros((mech.N, 64))
    chem.chem_rates(mech, w["p_Pa"], w["T"][:64].copy(), w["Y"][:, :64].copy(), f)
    np.testing.assert_array_equal(f, _gpu_rates(mech, w["p_Pa"], w["T"][:64], w["Y"][:, :64]))


def test_queue_static_and_determinism(small):
    w, mech, _ = small
    T, Y = w["T"], w["Y"]
    a = _gpu_integrate(mech, w, T, Y)
    b = _gpu_integrate(mech, w, T, Y, opts=chem.default_opts(use_queue=0))
    c = _gpu_integrate(mech, w, T, Y, opts=chem.default_opts(cells_per_cta=1, ctas_per_sm=2))
    for other in (b, c):
        np.testing.assert_array_equal(a[0], other[0])
        np.testing.assert_array_equal(a[1], other[1])
        np.testing.assert_array_equal(a[4], other[4])


def test_step_carry_over(small):
    """h_inout: the second call starts from the first call's proposed sub-step (Sec. 2.3)."""
    w, mech, ora = small
    T, Y = w["T"][:32], w["Y"][:, :32]
    h = np.zeros(32)
    Tg, Yg, _, _, _, hg = _gpu_integrate(mech, w, T, Y, h=h)
    ho = np.zeros(32)
    To, Yo, _, _, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"], h_inout=ho)
    assert np.all(hg > 0)
    # the proposal scales with err^-1/4 of a cancellation-prone error estimate: not a solution
    # quantity, so only its agreement to a loose relative tolerance is meaningful
    np.testing.assert_allclose(hg, ho, rtol=1e-3)
    Tg2, Yg2, _, st2, steps2, _ = _gpu_integrate(mech, w, Tg, Yg, h=hg)
    To2, Yo2, _, steps_o2, _ = ora.integrate(w["p_Pa"], To, Yo, w["dt"], h_inout=ho)
    _assert_state_close(Tg2, Yg2, To2, Yo2)


@pytest.mark.parametrize("which", ["small", "shear"])
def test_integrate_parity_mixed_precision(which, request):
    """FP32 LU + FP64-residual refinement matches the FP64 oracle to the same tolerance."""
    w, mech, ora = request.getfixturevalue(which)
    idx = np.arange(256) if which == "small" else _sample_shear(16, 3)
    T, Y = w["T"][idx], w["Y"][:, idx]
    opts = chem.default_opts(precision=chem.CHEM_PREC_MIXED)
    Tg, Yg, sg, stats, steps, _ = _gpu_integrate(mech, w, T, Y, opts=opts)
    To, Yo, so, steps_o, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], nthreads=16)
    assert np.all(sg == 0) and np.all(so == 0)
    _assert_state_close(Tg, Yg, To, Yo)
    # an attempt whose FP32 refinement does not converge is redone with FP64 factors, and the
    # cell then stays on FP64 factors for 16 attempts: fallbacks stay a small fraction
    assert stats.refine_fallbacks <= 0.1 * (stats.steps + stats.rejects)


@pytest.mark.parametrize("sweeps", [2, 0])
@pytest.mark.parametrize("which", ["small", "shear"])
def test_integrate_parity_fp32_pairs(which, sweeps, request):
    """LU and substitutions in FP32 pairs (about 48 significand bits) match the FP64 oracle to
    the integrate tolerance, with FP64-residual refinement (2 sweeps at most) and without it."""
    w, mech, ora = request.getfixturevalue(which)
    idx = np.arange(256) if which == "small" else _sample_shear(16, 3)
    T, Y = w["T"][idx], w["Y"][:, idx]
    opts = chem.default_opts(precision=chem.CHEM_PREC_MIXED_FF, refine_sweeps=sweeps)
    Tg, Yg, sg, stats, steps, _ = _gpu_integrate(mech, w, T, Y, opts=opts)
    To, Yo, so, steps_o, _ = ora.integrate(w["p_Pa"], T, Y, w["dt"], w["rtol"], w["atol"], nthreads=16)
    assert np.all(sg == 0) and np.all(so == 0)
    _assert_state_close(Tg, Yg, To, Yo)
    # pair factors solve to ~kappa 2^-48: one sweep converges, the FP64 fallback stays rare
    assert stats.refine_fallbacks <= 0.005 * (stats.steps + stats.rejects)
    # the same steps as the FP64 oracle, up to a few attempts decided by rounding in err ~ 1
    assert np.all(np.abs(steps.astype(np.int64) - steps_o) <= 0.01 * steps_o + 2)
