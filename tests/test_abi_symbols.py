"""The C-ABI library builds for sm_103a, loads, and exports every function the
header declares; the binding refuses to run without it.  No GPU needed."""
import ctypes
import os

import pytest

from paper_2402_13171_gb300 import build as B
from paper_2402_13171_gb300 import lbm


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_core_calls():
    names = lbm.header_functions()
    for n in ("lbm_create", "lbm_set_inflow", "alm_add_turbine", "lbm_step", "lbm_get_moments", "lbm_destroy"):
        assert n in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in lbm.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_loads_library(libpath):
    L = lbm.load()
    assert L.lbm_status_string(0) == b"ok"
    assert L.lbm_status_string(4) == b"non-finite state"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(lbm.LbmError):
        lbm.load()


def test_config_struct_matches_header_layout():
    # the ctypes mirror must have the same field order as lbm_config
    hdr = open(os.path.join(os.path.dirname(lbm.HERE), "include", "lbm_gb300.h")).read()
    body = hdr[hdr.index("typedef struct {\n    int nx, ny, nz;"):]
    body = body[:body.index("} lbm_config;")]
    order = ["nx", "collision", "nu", "smag_c", "storage", "bc", "body_force", "seed", "diag_every", "cuda_stream",
             "dev_alloc", "dev_free", "alloc_user", "tile_x", "tile_z", "staged"]
    pos = [body.index(k) for k in order]
    assert pos == sorted(pos)
    fields = [f[0] for f in lbm.LbmConfig._fields_]
    assert [f for f in fields if f in order] == order


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every struct the binding mirrors (lbm_config, lbm_inflow,
    alm_turbine_desc) has the size and field offsets the C compiler gives the
    header's definition."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"lbm_config": lbm.LbmConfig, "lbm_inflow": lbm.LbmInflow, "alm_turbine_desc": lbm.AlmTurbineDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm_gb300.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(lbm.HERE), "include")
    subprocess.run([gcc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, fname, v = line.split()
        got[(cname, fname)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
