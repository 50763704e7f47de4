"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ssa.h declares (no compute call: no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ssa.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ssa_status|const char\*)\s+(ssa_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_1605_07990_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("ssa_load_graph", "ssa_solve", "ssa_max_coverage", "ssa_coverage", "ssa_estimate_inf",
                 "ssa_pool_grow", "ssa_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    import ctypes
    lib = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(built):
    import paper_1605_07990_gb300 as P
    assert set(_declared()) <= set(P.EXPORTS)
    assert P.ssa_version().startswith("ssa-gb300")


def test_status_strings(built):
    import paper_1605_07990_gb300 as P
    L = P.lib()
    assert L.ssa_status_str(0) == b"ok"
    assert L.ssa_status_str(3) == b"RR pool full"

