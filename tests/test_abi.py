"""The C ABI library builds here and exports every entry point include/lattice.h declares (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lattice.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:lat_status|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ["lattice_setup", "assemble_residual_tangent", "select_principal_cells",
                 "apply_reduced_tangent", "newton_step", "adjoint_gradient"]:
        assert must in names


def test_library_builds_and_exports_everything():
    import __graft_entry__ as g
    g.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2603_10741_gb300", "liblattice.so"))
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2603_10741_gb300 import lattice as L
    assert sorted(L.EXPORTS) == _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2603_10741_gb300 import lattice as L
    with pytest.raises(ImportError):
        L.load_library(str(tmp_path / "missing.so"))
