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


def test_binding_structures_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and field offsets (a C
    probe compiled with gcc against include/lattice.h), so a field added on one side only fails
    here instead of shifting the other fields."""
    import shutil
    import subprocess
    from paper_2603_10741_gb300 import lattice as L
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    pairs = {"lat_mesh_desc": L.MeshDesc, "lat_sizes": L.Sizes, "lat_newton_opts": L.NewtonOpts,
             "lat_newton_report": L.NewtonReport}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lattice.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
