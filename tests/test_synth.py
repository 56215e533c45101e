"""The seeded input generator draws the workloads it states (CPU only).

* mechanisms: species / reaction / element counts and the third-body, Lindemann and Troe counts
  of the three named mechanisms; every reaction element-balanced, one or two molecules a side
  (the templates A+B=C+D, A+B=C, A=B+C), the pressure-dependent ones association or
  dissociation; distinct non-zero compositions with 0-3 atoms per element; the Arrhenius,
  efficiency, low-pressure and Troe parameters inside their stated ranges;
* thermo: cp, h and s continuous at T_mid = 1000 K (value continuity of the two NASA-7 fits),
  and cp/R close to the smooth model it was fitted to (3.5 for one atom at any T);
* fields: the shear layer's size, temperature bounds, mixing law and sum Y = 1; the igniting
  band; the uneven field's 10 / 60 / 30 % classes with their temperature ranges; the same seed
  gives the same arrays.
"""
import numpy as np
import pytest

from paper_2105_12070_gb300 import synth

MECHS = {
    "small": (synth.mechanism_small, 10, 30, 3, (3, 1, 0)),
    "53": (synth.mechanism_53, 53, 325, 4, (30, 0, 25)),
    "100": (synth.mechanism_100, 100, 700, 4, (60, 0, 40)),
}


@pytest.fixture(scope="module", params=sorted(MECHS))
def mech(request):
    make, K, R, E, counts = MECHS[request.param]
    return make(), K, R, E, counts


def test_mechanism_counts_and_templates(mech):
    m, K, R, E, (n_tb, n_lind, n_troe) = mech
    assert (m.K, m.R, len(m.elements)) == (K, R, E)
    assert np.sum(m.rtype == synth.TYPE_THIRD_BODY) == n_tb
    assert np.sum(m.rtype == synth.TYPE_LINDEMANN) == n_lind
    assert np.sum(m.rtype == synth.TYPE_TROE) == n_troe
    n_pd = n_tb + n_lind + n_troe
    for r in range(m.R):
        lhs = [k for k in m.reac[r] if k >= 0]
        rhs = [k for k in m.prod[r] if k >= 0]
        assert 1 <= len(lhs) <= 2 and 1 <= len(rhs) <= 2 and len(lhs) + len(rhs) >= 3, r
        # element balance
        assert np.array_equal(m.comp[lhs].sum(0), m.comp[rhs].sum(0)), r
        if r < n_pd:
            assert len(lhs) + len(rhs) == 3, r  # A+B=C or A=B+C
    # no reaction drawn twice (as written or reversed)
    keys = set()
    for r in range(m.R):
        lhs = tuple(sorted(int(k) for k in m.reac[r] if k >= 0))
        rhs = tuple(sorted(int(k) for k in m.prod[r] if k >= 0))
        key = (min(lhs, rhs), max(lhs, rhs))
        assert key not in keys, r
        keys.add(key)


def test_species_compositions(mech):
    m = mech[0]
    assert np.all(m.comp >= 0) and np.all(m.comp <= 3)
    assert np.all(m.comp.sum(1) > 0)
    assert len({tuple(c) for c in m.comp}) == m.K
    np.testing.assert_allclose(m.W, m.comp @ np.array([synth.ELEMENT_MASS[e] for e in m.elements]), rtol=1e-15)


def test_rate_parameter_ranges(mech):
    m = mech[0]
    assert np.all((np.log10(m.A) >= 8.0) & (np.log10(m.A) <= 14.0))
    assert np.all((m.b >= -1.0) & (m.b <= 2.0))
    assert np.all((m.Ea >= 0.0) & (m.Ea <= 50000.0))
    for r, e in m.eff.items():
        assert e.shape == (m.K,) and np.all((e >= 0.5) & (e <= 5.0))
    for r, (A0, b0, E0) in m.low.items():
        assert 14.0 <= np.log10(A0) <= 18.0 and -2.0 <= b0 <= 0.0 and 0.0 <= E0 <= 30000.0
    for r, (a, T3, T1, T2) in m.troe.items():
        assert 0.1 <= a <= 0.9 and 50.0 <= T3 <= 500.0 and 500.0 <= T1 <= 5000.0 and 2000.0 <= T2 <= 8000.0
    assert set(m.eff) == set(np.nonzero(m.rtype >= synth.TYPE_THIRD_BODY)[0])
    assert set(m.low) == set(np.nonzero(m.rtype >= synth.TYPE_LINDEMANN)[0])
    assert set(m.troe) == set(np.nonzero(m.rtype == synth.TYPE_TROE)[0])


def _nasa(a, T):
    cp = a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
    h = a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
    s = a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4 + a[6]
    return np.array([cp, h, s])


def test_thermo_continuity_and_model(mech):
    m = mech[0]
    for k in range(m.K):
        lo = _nasa(m.a_low[k], synth.T_MID)
        hi = _nasa(m.a_high[k], synth.T_MID)
        np.testing.assert_allclose(lo, hi, rtol=1e-10, atol=1e-10)
        atoms = int(m.comp[k].sum())
        for T in (400.0, 1500.0, 3000.0):
            a = m.a_low[k] if T <= synth.T_MID else m.a_high[k]
            cp = _nasa(a, T)[0]
            assert 3.5 - 0.05 <= cp <= 3.5 + 1.5 * (atoms - 1) + 0.05, (k, T, cp)
            if atoms == 1:
                assert abs(cp - 3.5) < 1e-6


def test_shear_layer_field():
    w = synth.workload_shear_layer()
    T, Y = w["T"], w["Y"]
    assert T.shape == (65536,) and Y.shape == (53, 65536)
    assert w["p_Pa"] == 40.0 * 101325.0 and w["dt"] == 1e-5 and (w["rtol"], w["atol"]) == (1e-6, 1e-10)
    assert T.min() >= 800.0 - 1e-9 and T.max() <= 1500.0 + 1e-9
    np.testing.assert_allclose(Y.sum(0), 1.0, atol=1e-14)
    # Y mixes linearly in Z between the two streams, with Z recovered from T
    (Tf, Yf), (To, Yo) = w["streams"]
    Z = (T - To) / (Tf - To)
    np.testing.assert_allclose(Y, Yf[:, None] * Z + Yo[:, None] * (1.0 - Z), atol=1e-14)
    # the tanh layer: both pure streams present, and a mixed band of a few dozen rows
    assert Z.min() < 1e-6 and Z.max() > 1 - 1e-6
    mixed = np.mean((Z > 0.01) & (Z < 0.99))
    assert 0.1 < mixed < 0.5, mixed
    again = synth.workload_shear_layer()
    assert np.array_equal(again["T"], T) and np.array_equal(again["Y"], Y)


def test_igniting_band():
    w = synth.workload_igniting()
    assert w["T"].shape == (16384,) and w["Y"].shape == (53, 16384)
    assert w["T"].min() >= 1000.0 and w["T"].max() <= 1300.0
    assert w["p_Pa"] == 20.0 * 101325.0 and w["dt"] == 1e-4
    np.testing.assert_allclose(w["Y"].sum(0), 1.0, atol=1e-14)


@pytest.mark.parametrize("order", ["shuffled", "blocked"])
def test_uneven_field(order):
    n = 4000
    w = synth.workload_uneven(n, order)
    T, Y, cls = w["T"], w["Y"], w["cls"]
    assert Y.shape == (100, n) and w["p_Pa"] == 60.0 * 101325.0 and w["dt"] == 5e-6
    counts = np.bincount(cls, minlength=3)
    assert tuple(counts) == (n // 10, n - n // 10 - (3 * n) // 10, (3 * n) // 10)
    assert np.all((T[cls == 0] >= 900.0) & (T[cls == 0] <= 1200.0))
    assert np.all((T[cls == 1] >= 300.0) & (T[cls == 1] <= 700.0))
    assert np.all((T[cls == 2] >= 2000.0) & (T[cls == 2] <= 2400.0))
    np.testing.assert_allclose(Y.sum(0), 1.0, atol=1e-12)
    if order == "blocked":
        assert np.all(np.diff(cls) >= 0)
    else:
        assert np.any(np.diff(cls) < 0)
