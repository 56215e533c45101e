"""Mechanism files in CHEMKIN-II form (the common subset): the oracle's reader and the library's
reader (each its own code) against the generator's CHEMMECH format describing the same numbers.

* the synthetic 10- and 53-species mechanisms written in both formats (NASA coefficients carried
  with the 9 significant digits of the E15.8 thermo fields) give the same rates in the oracle, to
  rounding in the molar masses (computed from the element masses in the CHEMKIN case);
* a hand-written CHEMKIN file exercising KCAL/MOLE, a '2X' coefficient, '=' and '<=>', +M with a
  partial efficiency list (others 1), (+M) with LOW and a three-parameter TROE (no T2 term),
  DUPLICATE and '!' comments equals its CHEMMECH transcription;
* a named third body '(+D)' equals the transcription with efficiency 1 for D and 0 elsewhere;
* unsupported forms (irreversible '=>', three molecules on a side, PLOG, efficiencies after a
  named third body, unknown species) are refused by both readers with a message;
* the library's reader (CPU: chem_load_mechanism parses before it touches the GPU) accepts the
  valid files and refuses the invalid ones with CHEM_EFILE.  GPU rates and integration from
  CHEMKIN files are compared with the oracle in tests/test_gpu_chemkin.py.
"""
import ctypes
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2105_12070_gb300 import chem, synth

RU = 8.314462618e7


def _write(text, suffix):
    fd, path = tempfile.mkstemp(suffix=suffix)
    os.close(fd)
    with open(path, "w") as fh:
        fh.write(text)
    return path


@pytest.mark.parametrize("which", ["small", "53"])
def test_synthetic_mechanism_both_formats(which):
    m = (synth.mechanism_small() if which == "small" else synth.mechanism_53()).rounded()
    ck = m.write_chemkin(_write("", ".ck"))
    cm = m.write(_write("", ".txt"))
    oc, om = O.OracleMechanism(ck), O.OracleMechanism(cm)
    assert (oc.K, oc.R) == (om.K, om.R) == (m.K, m.R)
    w = synth.workload_small() if which == "small" else synth.workload_shear_layer()
    idx = np.arange(0, 256, 8)
    fc, gc = oc.rates(w["p_Pa"], w["T"][idx], w["Y"][:, idx], gross=True)
    fm, gm = om.rates(w["p_Pa"], w["T"][idx], w["Y"][:, idx], gross=True)
    assert np.max(np.abs(fc - fm) / gm) <= 1e-13


def _nasa_card(name, elems, lo, hi, tmid=1000.0):
    f = lambda x: f"{x:15.8E}"
    el = "".join(f"{e:<2s}{n:3d}" for e, n in elems).ljust(20)
    head = f"{name:<18s}{'TOY':6s}{el}G{300.0:10.3f}{5000.0:10.3f}{tmid:8.2f}"
    co = list(hi) + list(lo)
    return [head.ljust(79) + "1", "".join(f(x) for x in co[0:5]).ljust(79) + "2",
            "".join(f(x) for x in co[5:10]).ljust(79) + "3", "".join(f(x) for x in co[10:14]).ljust(79) + "4"]


# a toy mechanism: elements X (20 g/mol) and Z (10 g/mol); species A = X, B = X, C = X2, D = XZ
_TOY_THERMO = {
    "A": ([("X", 1)], [3.5, 1e-4, 0, 0, 0, -1000.0, 10.0], [3.6, 5e-5, 0, 0, 0, -1050.0, 9.0]),
    "B": ([("X", 1)], [3.5, 2e-4, 0, 0, 0, 2000.0, 12.0], [3.7, 4e-5, 0, 0, 0, 1900.0, 11.0]),
    "C": ([("X", 2)], [4.5, 3e-4, 0, 0, 0, -5000.0, 15.0], [4.8, 1e-4, 0, 0, 0, -5200.0, 13.0]),
    "D": ([("X", 1), ("Z", 1)], [4.0, 1e-4, 0, 0, 0, 500.0, 14.0], [4.2, 6e-5, 0, 0, 0, 400.0, 13.0]),
}
_NAMES = ["A", "B", "C", "D"]


def _toy_chemkin(extra=""):
    lines = ["! toy mechanism", "ELEMENTS X /20.0/ Z/10.0/ END", "SPECIES A B", "C D", "END", "THERMO ALL",
             f"{300.0:10.3f}{1000.0:10.3f}{5000.0:10.3f}"]
    for n in _NAMES:
        el, lo, hi = _TOY_THERMO[n]
        lines += _nasa_card(n, el, lo, hi)
    lines += ["END", "REACTIONS KCAL/MOLE",
              "A + B <=> C      1.0E12  0.5  10.0   ! spaces inside the equation",
              "2A=C             3.0E11  0.0   5.0",
              "DUPLICATE",
              "2A=C             1.0E10  1.0   2.0",
              "DUPLICATE",
              "A+M<=>B+M        2.0E13 -1.0  20.0",
              "C/2.5/ D/0.5/",
              "A+D(+M)<=>C+B(+M)  4.0E12  0.0  3.0",
              "LOW / 1.0E16 -0.5 1.0 /",
              "TROE / 0.6 200.0 2000.0 /",
              "C/3.0/"]
    lines += extra.splitlines()
    lines += ["END"]
    return "\n".join(lines) + "\n"


def _toy_chemmech():
    wx, wz = 20.0, 10.0
    W = {"A": wx, "B": wx, "C": 2 * wx, "D": wx + wz}
    comp = {"A": (1, 0), "B": (1, 0), "C": (2, 0), "D": (1, 1)}
    r = lambda x: repr(float(f"{x:15.8E}"))
    L = ["CHEMMECH 1", "elements 2", "X 20.0", "Z 10.0", "species 4"]
    for n in _NAMES:
        _, lo, hi = _TOY_THERMO[n]
        L.append(" ".join([n, repr(W[n]), "300.0", "1000.0", "5000.0", *map(str, comp[n])] +
                          [r(x) for x in lo] + [r(x) for x in hi]))
    i = {n: k for k, n in enumerate(_NAMES)}
    L += ["reactions 5",
          f"0 2 {i['A']} {i['B']} 1 {i['C']} -1 1e12 0.5 10000.0",
          f"0 2 {i['A']} {i['A']} 1 {i['C']} -1 3e11 0.0 5000.0",
          f"0 2 {i['A']} {i['A']} 1 {i['C']} -1 1e10 1.0 2000.0",
          f"1 1 {i['A']} -1 1 {i['B']} -1 2e13 -1.0 20000.0", "eff 1.0 1.0 2.5 0.5",
          f"3 2 {i['A']} {i['D']} 2 {i['C']} {i['B']} 4e12 0.0 3000.0", "eff 1.0 1.0 3.0 1.0",
          "low 1e16 -0.5 1000.0", "troe 0.6 200.0 2000.0 1e30", "end"]
    return "\n".join(L) + "\n"


def test_hand_written_chemkin_equals_its_transcription():
    oc = O.OracleMechanism(_write(_toy_chemkin(), ".ck"))
    om = O.OracleMechanism(_write(_toy_chemmech(), ".txt"))
    rng = np.random.default_rng(3)
    T = rng.uniform(800.0, 2000.0, size=16)
    Y = rng.dirichlet(np.ones(4), size=16).T.copy()
    for p in (1e5, 4e6):
        fc, gc = oc.rates(p, T, Y, gross=True)
        fm, gm = om.rates(p, T, Y, gross=True)
        assert np.max(np.abs(fc - fm) / gm) <= 1e-13
    assert np.max(np.abs(oc.jacobian(1e5, T, Y) - om.jacobian(1e5, T, Y))) <= 1e-9 * np.max(
        np.abs(om.jacobian(1e5, T, Y)))


def test_named_third_body_equals_one_hot_efficiencies():
    # (+D): a Lindemann fall-off whose third body is D alone
    ck = _toy_chemkin("A+B(+D)<=>C(+D)  5.0E11  0.2  4.0\nLOW / 2.0E15 -0.3 1.5 /")
    cm = _toy_chemmech().replace("reactions 5", "reactions 6").replace(
        "end", "2 2 0 1 1 2 -1 5e11 0.2 4000.0\neff 0.0 0.0 0.0 1.0\nlow 2e15 -0.3 1500.0\nend")
    oc = O.OracleMechanism(_write(ck, ".ck"))
    om = O.OracleMechanism(_write(cm, ".txt"))
    rng = np.random.default_rng(4)
    T = rng.uniform(800.0, 2000.0, size=16)
    Y = rng.dirichlet(np.ones(4), size=16).T.copy()
    for p in (1e5, 4e6):
        fc, gc = oc.rates(p, T, Y, gross=True)
        fm, gm = om.rates(p, T, Y, gross=True)
        assert np.max(np.abs(fc - fm) / gm) <= 1e-13
    # the library reads the same tables (checked in full by tests/test_chemkin_readers.py)
    lines = chem.chem_describe_mechanism(_write(ck, ".ck")).splitlines()
    assert lines[-1].startswith("rx 2 2 0 1 1 2 ") and " eff 0 0 0 1 low " in lines[-1]


BAD = {
    "irreversible": "A+B=>C 1.0E12 0.0 1.0",
    "three molecules": "A+A+B<=>C+B 1.0E12 0.0 1.0",
    "plog": "A<=>B 1.0E12 0.0 1.0\nPLOG / 1.0 1.0E12 0.0 1.0 /",
    "efficiencies after a named third body": "A+B(+D)<=>C(+D) 1.0E12 0.0 1.0\nLOW / 1.0E16 0.0 1.0 /\nC/2.0/",
    "two different named third bodies": "A+B(+D)<=>C(+A) 1.0E12 0.0 1.0\nLOW / 1.0E16 0.0 1.0 /",
    "unknown species": "A+Q<=>C 1.0E12 0.0 1.0",
}


@pytest.mark.parametrize("case", sorted(BAD))
def test_unsupported_forms_are_refused(case):
    path = _write(_toy_chemkin(BAD[case]), ".ck")
    with pytest.raises(RuntimeError):
        O.OracleMechanism(path)
    lib = chem.load_library()
    h = ctypes.c_void_p()
    rc = lib.chem_load_mechanism(path.encode(), ctypes.byref(h))
    assert rc == -2, (case, rc, lib.chem_last_error())  # CHEM_EFILE
    assert lib.chem_last_error()


def test_library_reader_accepts_valid_files():
    lib = chem.load_library()
    for path in (_write(_toy_chemkin(), ".ck"), synth.mechanism_small().rounded().write_chemkin(_write("", ".ck"))):
        h = ctypes.c_void_p()
        rc = lib.chem_load_mechanism(path.encode(), ctypes.byref(h))
        # 0 with a GPU; without one the parse succeeds and the device query fails (CHEM_ECUDA)
        assert rc in (0, -3), (rc, lib.chem_last_error())
        if rc == 0:
            lib.chem_free_mechanism(h)
