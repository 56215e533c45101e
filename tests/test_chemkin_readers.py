"""The library's mechanism reader against the oracle's (CPU only; each is its own code).

Both print the tables they read in one text form (chem_describe_mechanism, and the oracle's
describe): species molar mass, T_mid and NASA coefficients; per reaction the kind, the species
of each side, A, b, Ea/R, efficiencies, the low-pressure limit and the Troe parameters.  For the
generator's CHEMMECH files and for CHEMKIN-II files in the syntax variants real files use (unit
keywords, lower case and four-letter keywords, species names with parentheses, Troe with and
without T2, a named third body, per-species T_mid, efficiency lists over two lines, comments and
blank lines) the
two readings must agree to rounding, or both readers must refuse the file.
"""
import os
import re
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2105_12070_gb300 import chem, synth
from test_chemkin import _NAMES, _TOY_THERMO, _nasa_card


def _write(text, suffix=".ck"):
    fd, path = tempfile.mkstemp(suffix=suffix)
    os.close(fd)
    with open(path, "w") as fh:
        fh.write(text)
    return path


def _parse(text):
    lines = text.splitlines()
    K = int(lines[0].split()[1])
    sp = np.array([[float(x) for x in l.split()[1:]] for l in lines[1:1 + K]])
    R = int(lines[1 + K].split()[1])
    rx = []
    for l in lines[2 + K:2 + K + R]:
        t = l.split()[1:]
        kind = int(t[0])
        i = 1
        sides = []
        for _ in range(2):
            n = int(t[i])
            sides.append(tuple(int(x) for x in t[i + 1:i + 1 + n]))
            i += 1 + n
        rest = t[i:]
        arr = {"arr": [], "eff": [], "low": [], "troe": []}
        key = "arr"
        for tok in rest:
            if tok in arr:
                key = tok
            else:
                arr[key].append(float(tok))
        rx.append((kind, sides[0], sides[1], {k: np.array(v) for k, v in arr.items()}))
    assert len(lines) == 2 + K + R
    return sp, rx


def _compare(lib_text, ora_text):
    sp_l, rx_l = _parse(lib_text)
    sp_o, rx_o = _parse(ora_text)
    assert sp_l.shape == sp_o.shape
    np.testing.assert_allclose(sp_l, sp_o, rtol=1e-14, atol=0)
    assert len(rx_l) == len(rx_o)
    for r, (a, b) in enumerate(zip(rx_l, rx_o)):
        assert a[:3] == b[:3], (r, a[:3], b[:3])
        for key in ("arr", "eff", "low", "troe"):
            assert a[3][key].shape == b[3][key].shape, (r, key)
            # A and A0 pass through ln on the library side: a few ulp of |ln A|
            np.testing.assert_allclose(a[3][key], b[3][key], rtol=1e-13, atol=0, err_msg=f"reaction {r} {key}")


def _both(path):
    """(library text or None, oracle text or None), None for a refused file."""
    try:
        lib = chem.chem_describe_mechanism(path)
    except chem.ChemError:
        lib = None
    try:
        ora = O.OracleMechanism(path).describe()
    except RuntimeError:
        ora = None
    return lib, ora


@pytest.mark.parametrize("which", ["small", "53", "100"])
@pytest.mark.parametrize("fmt", ["chemmech", "chemkin"])
def test_synthetic_mechanisms(which, fmt):
    m = {"small": synth.mechanism_small, "53": synth.mechanism_53, "100": synth.mechanism_100}[which]()
    if fmt == "chemkin":
        m = m.rounded()
        path = m.write_chemkin(_write(""))
    else:
        path = m.write(_write("", ".txt"))
    lib, ora = _both(path)
    assert lib is not None and ora is not None
    _compare(lib, ora)
    assert len(_parse(lib)[1]) == m.R


# --- CHEMKIN syntax variants -------------------------------------------------------------------

_REACTIONS = [
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
    "C/3.0/",
    "C(+M)<=>A+B(+M)  1.0E10  0.3  15.0",
    "LOW / 3.0E14 0.0 9.0 /",
    "TROE / 0.45 100.0 1500.0 5000.0 /",
    "B+D(+M)<=>C+D(+M)  2.0E11  0.0  7.0",
    "LOW / 5.0E15 -1.0 0.0 /",
    "A+B(+D)<=>C(+D)  5.0E11  0.2  4.0   ! D alone is the third body",
    "LOW / 2.0E15 -0.3 1.5 /",
]


# the toy species as whole tokens (one pass, so that new names are not renamed again)
_rename = re.compile(r"(?<![A-Za-z])([ABCD])(?![A-Za-z])")


def _variant(units="KCAL/MOLE", names=None, keyword_case=str.upper, abbrev=False, tmid=None, split_eff=False,
             blank_comments=False):
    names = names or {n: n for n in _NAMES}
    kw = lambda k: keyword_case(k[:4] if abbrev else k)
    lines = ["! toy mechanism", f"{kw('ELEMENTS')} X /20.0/ Z/10.0/", kw("END"),
             f"{kw('SPECIES')} {names['A']} {names['B']}", f"{names['C']} {names['D']}", kw("END"),
             f"{keyword_case('THERMO')} {keyword_case('ALL')}", f"{300.0:10.3f}{1000.0:10.3f}{5000.0:10.3f}"]
    for n in _NAMES:
        el, lo, hi = _TOY_THERMO[n]
        lines += _nasa_card(names[n], el, lo, hi, tmid=(tmid or {}).get(n, 1000.0))
    lines += [kw("END"), (f"{kw('REACTIONS')} {units}" if units else kw("REACTIONS"))]
    conv = {"KCAL/MOLE": 1.0, "CAL/MOLE": 1e3, "JOULES/MOLE": 4184.0, "KJOULES/MOLE": 4.184,
            "KELVINS": 1e3 / (8.314462618 / 4.184), None: 1e3}[units]
    for l in _REACTIONS:
        m = re.match(r"^(\S.*?)\s+([0-9.E+-]+)\s+([0-9.E+-]+)\s+([0-9.E+-]+)(\s*!.*)?$", l)
        if m and "/" not in l.split("!")[0]:
            eq, A, b, E = m.group(1), m.group(2), m.group(3), float(m.group(4))
            eq = _rename.sub(lambda x: names[x.group(1)], eq)
            l = f"{eq}  {A}  {b}  {E * conv!r}{m.group(5) or ''}"
        elif l.startswith(("LOW", "TROE", "DUPLICATE")):
            head = l.split("/")[0].strip() if "/" in l else l.strip()
            l = l.replace(head, keyword_case(head), 1)
            if head == "LOW":
                vals = l.split("/")[1].split()
                l = f"{keyword_case('LOW')} / {vals[0]} {vals[1]} {float(vals[2]) * conv!r} /"
        else:  # efficiency list
            l = _rename.sub(lambda x: names[x.group(1)], l)
            if split_eff and l.count("/") >= 4:
                parts = l.split()
                lines.append(parts[0])
                l = " ".join(parts[1:])
        lines.append(l)
        if blank_comments:
            lines += ["", "   ! a comment line", ""]
    lines.append(kw("END"))
    return "\n".join(lines) + "\n"


VARIANTS = {
    "kcal": dict(),
    "cal": dict(units="CAL/MOLE"),
    "default units": dict(units=None),
    "joules": dict(units="JOULES/MOLE"),
    "kjoules": dict(units="KJOULES/MOLE"),
    "kelvins": dict(units="KELVINS"),
    "lower case keywords": dict(keyword_case=str.lower),
    "four-letter keywords": dict(abbrev=True),
    "names with parentheses and digits": dict(names={"A": "CH2(S)", "B": "C2H4", "C": "N-C3H7", "D": "AR2"}),
    "per-species Tmid": dict(tmid={"A": 1200.0, "C": 800.0}),
    "efficiencies over two lines": dict(split_eff=True),
    "blank lines and comments": dict(blank_comments=True),
}


@pytest.mark.parametrize("case", sorted(VARIANTS))
def test_chemkin_variants_read_alike(case):
    path = _write(_variant(**VARIANTS[case]))
    lib, ora = _both(path)
    assert (lib is None) == (ora is None), (case, lib is None, ora is None)
    assert lib is not None, case  # every variant above is valid CHEMKIN-II
    _compare(lib, ora)


def test_units_give_the_same_activation_energies():
    base = _parse(chem.chem_describe_mechanism(_write(_variant())))[1]
    for units in ("CAL/MOLE", "JOULES/MOLE", "KJOULES/MOLE", "KELVINS", None):
        other = _parse(chem.chem_describe_mechanism(_write(_variant(units=units))))[1]
        for a, b in zip(base, other):
            np.testing.assert_allclose(a[3]["arr"], b[3]["arr"], rtol=1e-13)
            np.testing.assert_allclose(a[3]["low"], b[3]["low"], rtol=1e-13)


def test_describe_refuses_bad_files():
    lib = chem.load_library()
    need = np.zeros(1, np.int64)
    import ctypes
    n = ctypes.c_int64()
    assert lib.chem_describe_mechanism(b"/nonexistent/mech.ck", None, 0, ctypes.byref(n)) == -2
    path = _write(_variant())
    assert lib.chem_describe_mechanism(path.encode(), None, 0, ctypes.byref(n)) == 0 and n.value > 100
    buf = ctypes.create_string_buffer(8)
    assert lib.chem_describe_mechanism(path.encode(), buf, 8, ctypes.byref(n)) == -4


def _thermo_variants():
    base = _variant()
    el, lo, hi = _TOY_THERMO["A"]
    extra = "\n".join(_nasa_card("EXTRA", el, lo, hi))
    i = base.index("\nEND\nREACTIONS")
    j = base.index("   300.000  1000.000  5000.000")
    k = base.index("D                 TOY")
    return {
        "THERMO without ALL": (base.replace("THERMO ALL", "THERMO"), True),
        "a thermo card for a species not in SPECIES": (base[:i] + "\n" + extra + base[i:], True),
        "a comment line in THERMO": (base[:j] + "! thermo comment\n" + base[j:], True),
        "a species without thermo": (base[:k] + base[k:].split("\n", 4)[4], False),
    }


@pytest.mark.parametrize("case", sorted(_thermo_variants()))
def test_thermo_section_variants(case):
    text, valid = _thermo_variants()[case]
    lib, ora = _both(_write(text))
    assert (lib is not None) == valid and (ora is not None) == valid, case
    if valid:
        _compare(lib, ora)
