"""The oracle's pins catch plausible mistakes: each planted mistake fails the pin that guards it.

chem_oracle.cpp compiled with -DORACLE_PLANT=n carries one deliberate error (marked "plant n"
there).  Several are planted consistently in f and in the analytical Jacobian, so the
complex-step Jacobian check cannot see them and a physical pin has to.  A pin fails either at its
property or earlier, when the integration it runs no longer completes (plants 1, 3 and 5 end
that way: a cell status other than OK).

  1  sign of the delta-nu term of ln Kc (rates and d ln Kc/dT)   -> equilibrium, detailed balance
  2  W_k dropped from dY_k/dt (rates and the species rows of J)   -> element conservation
  3  sign of dT/dt (rates and the temperature row of J)           -> enthalpy conservation
  4  NASA h/RT coefficient of a3 T^2 taken as 1/2                 -> d(h/R)/dT = cp/R
  5  [M] missing on the reverse rate of third-body reactions       -> closed-form A=B with [M]
  6  sign of d ln rho/dY_i in the Jacobian                         -> complex-step Jacobian
  7  Troe c = -0.4 + 0.67 log10 Fcent (rates and J)                -> Troe F = Fcent at the centre
  8  Rosenbrock weight b_1 off by 1e-3                             -> order conditions
  9  third-body efficiencies ignored in [M]                        -> closed-form A=B with [M]
 10  the Jacobian returned transposed                              -> complex-step Jacobian
 11  Troe width n = 0.75 + 1.27 log10 Fcent (rates and J)          -> Troe broadening width
 12  Troe slope term n + 0.14 (log10 Pr + c) (rates and J)         -> Troe broadening width

The pins are the functions of test_oracle_chemistry.py and test_oracle_integrator.py, called on
oracle objects made from the planted build.  The unplanted oracle passes all of them (those
modules' own runs).
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle as O
import test_oracle_chemistry as C
import test_oracle_integrator as I
from paper_2105_12070_gb300 import synth

PLANTS = range(1, 13)


class _Fixtures:
    """Stands in for pytest's request object of the parametrised pins."""

    def __init__(self, values):
        self._values = values

    def getfixturevalue(self, name):
        return self._values[name]


def _fixtures():
    gs, g53 = synth.mechanism_small(), synth.mechanism_53()
    return (gs, O.OracleMechanism(gs.write_temp())), (g53, O.OracleMechanism(g53.write_temp()))


def _integrate_small(small):
    """The integration of test_oracle_chemistry.test_invariants_small (32 cells, rtol 1e-6)."""
    gen, ora = small
    w = synth.workload_small()
    T0, Y0 = w["T"][:32], w["Y"][:, :32]
    Tn, Yn, st, _, _ = ora.integrate(w["p_Pa"], T0, Y0, w["dt"], rtol=1e-6, atol=1e-10, nthreads=4)
    assert np.all(st == 0)
    return gen, ora, T0, Y0, Tn, Yn


def _elements(small):
    # the element-conservation assertion of test_invariants_small
    gen, _, _, Y0, _, Yn = _integrate_small(small)
    e0, e1 = C._element_totals(gen, Y0), C._element_totals(gen, Yn)
    assert np.abs(e1 - e0).max() / np.abs(e0).max() < 1e-12


def _enthalpy(small):
    # the enthalpy-conservation assertion of test_invariants_small
    gen, ora, T0, Y0, Tn, Yn = _integrate_small(small)
    h0, sc = C._mix_enthalpy(ora, gen, T0, Y0)
    h1, _ = C._mix_enthalpy(ora, gen, Tn, Yn)
    assert np.all(np.abs(h1 - h0) <= 2e-5 * sc)


# plant -> the pin that must fail, as a function of the (small, mech53) fixtures
GUARD = {
    1: ("equilibrium and detailed balance", lambda s, m: C.test_equilibrium_and_detailed_balance(s)),
    2: ("element conservation (invariants)", lambda s, m: _elements(s)),
    3: ("enthalpy conservation (invariants)", lambda s, m: _enthalpy(s)),
    4: ("thermo complex step", lambda s, m: C.test_thermo_complex_step(s, m)),
    5: ("closed-form A=B third body", lambda s, m: I.test_closed_form_isomer_third_body()),
    6: ("complex-step Jacobian", lambda s, m: C.test_jacobian_complex_step("small", _Fixtures({"small": s}))),
    7: ("Troe fall-off centre", lambda s, m: C.test_falloff_limits(True)),
    8: ("Rosenbrock order conditions", lambda s, m: I.test_order_conditions()),
    9: ("closed-form A=B third body", lambda s, m: I.test_closed_form_isomer_third_body()),
    10: ("complex-step Jacobian", lambda s, m: C.test_jacobian_complex_step("mech53", _Fixtures({"mech53": m}))),
    11: ("Troe broadening width", lambda s, m: C.test_troe_broadening_width()),
    12: ("Troe broadening width", lambda s, m: C.test_troe_broadening_width()),
}


@pytest.fixture(scope="module", autouse=True)
def planted_builds():
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        list(ex.map(lambda n: O.build(plant=n), PLANTS))


@pytest.mark.parametrize("plant", PLANTS)
def test_planted_mistake_fails_its_pin(plant):
    name, pin = GUARD[plant]
    with O.planted(plant):
        small, mech53 = _fixtures()
        with pytest.raises(Exception):
            pin(small, mech53)


def test_guards_pass_on_the_oracle():
    small, mech53 = _fixtures()
    for plant in PLANTS:
        GUARD[plant][1](small, mech53)
