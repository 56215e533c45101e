"""Discrete adjoint on the GPU (chem_integrate_record + chem_adjoint) against the oracle's
tangent-linear model of the same accepted steps (Sec. 2.3, Eq. 2 with the step sizes frozen).

For the map Phi(dt) = M(Phi_0, ln A) of the recorded steps, the adjoint returns
g = (dM/dPhi_0)^T lambda and (dM/d ln A)^T lambda; the oracle's dual-number replay returns
dM . d along a direction d.  Both are the derivative of one map, so for every lambda and d
    <lambda, dM . d> = <g, d>
up to rounding (the GPU differentiates its transformed-form steps, the oracle its classical-form
steps; the two agree to rounding, and the derivatives agree to rounding amplified by the
conditioning of the step sequence).  Tolerance: 1e-8 of sum |lambda_i| |(dM . d)_i|, from
numpy prototypes of the same sweep (5e-10 on a stiff 53-species cell, 4e-14 on the 10-species
mechanism).  Central differences of the replay (step 1e-6 relative in the state, 1e-6 in ln A)
agree to 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2105_12070_gb300 import autograd as cad
from paper_2105_12070_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small():
    w = synth.workload_small()
    path = w["mech"].write_temp()
    return w, chem.Mechanism(path), O.OracleMechanism(path)


@pytest.fixture(scope="module")
def igniting():
    w = synth.workload_igniting(16)
    path = w["mech"].write_temp()
    return w, chem.Mechanism(path), O.OracleMechanism(path)


def _record(mech, w, cells, cap=4096, dt=None):
    T, Y = _dev(w["T"][cells]), _dev(w["Y"][:, cells])
    n = len(cells)
    rec = torch.empty((n, cap, mech.N + 1), dtype=torch.float64, device="cuda")
    nsteps = torch.empty(n, dtype=torch.int32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    chem.chem_integrate_record(mech, w["p_Pa"], T, Y, dt or w["dt"], rec, nsteps, status, rtol=w["rtol"],
                               atol=w["atol"])
    return T, Y, rec, nsteps, status


def _adjoint(mech, w, rec, nsteps, status, gT, gY, per_cell=True):
    n = gT.shape[0]
    gT0 = torch.empty(n, dtype=torch.float64, device="cuda")
    gY0 = torch.empty((mech.K, n), dtype=torch.float64, device="cuda")
    gA = torch.empty(mech.R, dtype=torch.float64, device="cuda")
    gC = torch.empty((n, mech.R), dtype=torch.float64, device="cuda") if per_cell else None
    chem.chem_adjoint(mech, w["p_Pa"], rec, nsteps, status, _dev(gT), _dev(gY), gT0, gY0, g_lnA=gA, g_lnA_cells=gC)
    torch.cuda.synchronize()
    return gT0.cpu().numpy(), gY0.cpu().numpy(), gA.cpu().numpy(), (gC.cpu().numpy() if per_cell else None)


def _phi0(w, c):
    return np.concatenate([[w["T"][c]], w["Y"][:-1, c]])


def _lambda_phi(gT, gY, c):
    return np.concatenate([[gT[c]], gY[:-1, c] - gY[-1, c]])


def test_record_mode_matches_plain_integrate(small):
    w, mech, _ = small
    cells = np.arange(48)
    T, Y, rec, nsteps, status = _record(mech, w, cells)
    T2, Y2 = _dev(w["T"][cells]), _dev(w["Y"][:, cells])
    chem.chem_integrate(mech, w["p_Pa"], T2, Y2, w["dt"], rtol=w["rtol"], atol=w["atol"])
    torch.cuda.synchronize()
    assert torch.all(status == 0)
    assert torch.equal(T, T2) and torch.equal(Y, Y2)
    ns = nsteps.cpu().numpy()
    r = rec.cpu().numpy()
    for i, c in enumerate(cells[:6]):
        assert np.array_equal(r[i, 0, :-1], _phi0(w, c))
        assert abs(r[i, :ns[i], -1].sum() - w["dt"]) <= 1e-12 * w["dt"]


def test_record_full_status_and_nan_gradients(small):
    w, mech, _ = small
    cells = np.arange(8)
    T, Y, rec, nsteps, status = _record(mech, w, cells, cap=5)
    st = status.cpu().numpy()
    assert np.all(st == chem.CHEM_CELL_RECORD_FULL)
    assert np.all(nsteps.cpu().numpy() == 5)
    rng = np.random.default_rng(0)
    gT0, gY0, gA, gC = _adjoint(mech, w, rec, nsteps, status, rng.normal(size=8), rng.normal(size=(mech.K, 8)))
    assert np.all(np.isnan(gT0)) and np.all(np.isnan(gY0)) and np.all(np.isnan(gA)) and np.all(np.isnan(gC))


def _dot_test(w, mech, om, cells, seed, tol=1e-8):
    T, Y, rec, nsteps, status = _record(mech, w, cells)
    assert torch.all(status == 0)
    n = len(cells)
    rng = np.random.default_rng(seed)
    gT = rng.normal(size=n) * 1e-3
    gY = rng.normal(size=(mech.K, n))
    gT0, gY0, gA, gC = _adjoint(mech, w, rec, nsteps, status, gT, gY)
    assert np.all(gY0[-1] == 0.0)
    np.testing.assert_allclose(gA, gC.sum(axis=0), rtol=1e-12, atol=1e-12 * np.abs(gC).sum(axis=0).max())
    r = rec.cpu().numpy()
    ns = nsteps.cpu().numpy()
    for i, c in enumerate(cells):
        phi0 = _phi0(w, c)
        hs = r[i, :ns[i], -1]
        lam = _lambda_phi(gT, gY, i)
        dphi = rng.normal(size=mech.N) * np.maximum(np.abs(phi0), 1e-8)
        dlnA = rng.normal(size=mech.R)
        _, tl = om.replay(w["p_Pa"], phi0, hs, dphi=dphi, dlnA=dlnA)
        lhs = lam @ tl
        rhs = gT0[i] * dphi[0] + gY0[:-1, i] @ dphi[1:] + gC[i] @ dlnA
        scale = np.abs(lam) @ np.abs(tl)
        assert abs(lhs - rhs) <= tol * scale, (c, lhs, rhs, scale)


def test_adjoint_dot_product_small(small):
    w, mech, om = small
    _dot_test(w, mech, om, np.arange(0, 256, 16), seed=1)


def test_adjoint_full_gradient_small(small):
    """Every component of the gradient, from N + R tangent-linear replays of one cell."""
    w, mech, om = small
    cells = np.array([3, 77])
    T, Y, rec, nsteps, status = _record(mech, w, cells)
    rng = np.random.default_rng(2)
    gT = rng.normal(size=2) * 1e-3
    gY = rng.normal(size=(mech.K, 2))
    gT0, gY0, gA, gC = _adjoint(mech, w, rec, nsteps, status, gT, gY)
    r = rec.cpu().numpy()
    ns = nsteps.cpu().numpy()
    for i, c in enumerate(cells):
        phi0 = _phi0(w, c)
        hs = r[i, :ns[i], -1]
        lam = _lambda_phi(gT, gY, i)
        g_phi = np.array([lam @ om.replay(w["p_Pa"], phi0, hs, dphi=np.eye(mech.N)[j])[1] for j in range(mech.N)])
        g_lnA = np.array([lam @ om.replay(w["p_Pa"], phi0, hs, dlnA=np.eye(mech.R)[j])[1] for j in range(mech.R)])
        got_phi = np.concatenate([[gT0[i]], gY0[:-1, i]])
        np.testing.assert_allclose(got_phi, g_phi, rtol=1e-8, atol=1e-8 * np.abs(g_phi).max())
        np.testing.assert_allclose(gC[i], g_lnA, rtol=1e-8, atol=1e-8 * np.abs(g_lnA).max())


def test_adjoint_central_differences_igniting(igniting):
    """The 53-species igniting band at 20 atm over dt = 1e-4 s: adjoint vs central differences
    (step 1e-6 relative) of the oracle's replay of the recorded steps, and vs the tangent-linear
    model by the dot-product test."""
    w, mech, om = igniting
    cells = np.array([0, 5])
    _dot_test(w, mech, om, cells, seed=3)
    T, Y, rec, nsteps, status = _record(mech, w, cells)
    rng = np.random.default_rng(4)
    gT = rng.normal(size=2) * 1e-3
    gY = rng.normal(size=(mech.K, 2))
    gT0, gY0, gA, gC = _adjoint(mech, w, rec, nsteps, status, gT, gY)
    r = rec.cpu().numpy()
    ns = nsteps.cpu().numpy()
    i, c = 0, cells[0]
    phi0 = _phi0(w, c)
    hs = r[i, :ns[i], -1]
    lam = _lambda_phi(gT, gY, i)
    d = rng.normal(size=mech.N) * np.abs(phi0)
    eps = 1e-6
    fd = lam @ (om.replay(w["p_Pa"], phi0 + eps * d, hs) - om.replay(w["p_Pa"], phi0 - eps * d, hs)) / (2 * eps)
    adj = gT0[i] * d[0] + gY0[:-1, i] @ d[1:]
    assert abs(fd - adj) <= 1e-5 * abs(adj) + 1e-12, (fd, adj)
    dl = rng.normal(size=mech.R)
    fd = lam @ (om.replay(w["p_Pa"], phi0, hs, lnA_shift=eps * dl) -
                om.replay(w["p_Pa"], phi0, hs, lnA_shift=-eps * dl)) / (2 * eps)
    adj = gC[i] @ dl
    assert abs(fd - adj) <= 1e-5 * abs(adj) + 1e-12, (fd, adj)


def test_lnA_get_set_roundtrip_and_use(small):
    w, mech, om = small
    lnA0 = chem.chem_get_lnA(mech)
    shift = np.random.default_rng(5).normal(size=mech.R) * 0.05
    try:
        chem.chem_set_lnA(mech, lnA0 + shift)
        np.testing.assert_array_equal(chem.chem_get_lnA(mech), lnA0 + shift)
        cells = np.arange(4)
        T, Y, rec, nsteps, status = _record(mech, w, cells)
        r = rec.cpu().numpy()
        ns = nsteps.cpu().numpy()
        for i, c in enumerate(cells):
            out = om.replay(w["p_Pa"], _phi0(w, c), r[i, :ns[i], -1], lnA_shift=shift)
            got = np.concatenate([[T[i].item()], Y[:-1, i].cpu().numpy()])
            np.testing.assert_allclose(got, out, rtol=1e-9, atol=1e-14)
    finally:
        chem.chem_set_lnA(mech, lnA0)
    np.testing.assert_array_equal(chem.chem_get_lnA(mech), lnA0)


def test_autograd_function(small):
    """loss = <a, T(dt)> + <B, Y(dt)> through the torch.autograd.Function equals the direct
    chem_adjoint call, and its ln A gradient is the sum of the per-cell terms."""
    w, mech, om = small
    cells = np.arange(32)
    T0 = _dev(w["T"][cells]).requires_grad_(True)
    Y0 = _dev(w["Y"][:, cells]).requires_grad_(True)
    lnA = torch.from_numpy(chem.chem_get_lnA(mech)).cuda().requires_grad_(True)
    T1, Y1, status = cad.integrate(mech, w["p_Pa"], T0, Y0, lnA, w["dt"], rtol=w["rtol"], atol=w["atol"])
    assert torch.all(status == 0)
    rng = np.random.default_rng(6)
    a = _dev(rng.normal(size=32) * 1e-3)
    B = _dev(rng.normal(size=(mech.K, 32)))
    loss = (a * T1).sum() + (B * Y1).sum()
    loss.backward()
    _, _, rec, nsteps, st = _record(mech, w, cells)
    gT0, gY0, gA, gC = _adjoint(mech, w, rec, nsteps, st, a.cpu().numpy(), B.cpu().numpy())
    np.testing.assert_array_equal(T0.grad.cpu().numpy(), gT0)
    np.testing.assert_array_equal(Y0.grad.cpu().numpy(), gY0)
    np.testing.assert_array_equal(lnA.grad.cpu().numpy(), gA)
