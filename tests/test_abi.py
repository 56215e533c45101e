"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/chemgpu.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

from paper_2105_12070_gb300 import chem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chemgpu.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(chem_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("chem_load_mechanism", "chem_rates", "chem_jacobian", "chem_integrate", "chem_integrate_record",
                     "chem_adjoint", "chem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = chem.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_last_error_is_empty_string_initially():
    lib = chem.load_library()
    assert isinstance(lib.chem_last_error(), bytes)
