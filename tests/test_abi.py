"""CPU checks of the C ABI: the library builds, loads without a GPU and
exports every function include/dhfwi.h declares; host-side validation."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|const\s+char\s*\*)\s*\**\s*(\w+)\s*\(", txt, re.M)
    return names


def test_library_exports_every_declared_symbol():
    from paper_2403_17518_gb300 import _lib, build

    build()
    L = _lib.load()
    names = _declared()
    assert {"dhfwi_create", "model_shots", "fwi_gradient", "born_demig", "rtm_mig"} <= set(names)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_create_rejects_bad_grid_without_gpu():
    import ctypes

    from paper_2403_17518_gb300 import _lib

    L = _lib.load()
    h = ctypes.c_void_p()
    g = _lib.Grid(0, 10, 20, 10.0, 1e-3)
    assert L.dhfwi_create(ctypes.byref(h), ctypes.byref(g), 0) == -1
    assert b"bad grid" in L.dhfwi_last_error(None)
    g = _lib.Grid(10, 10, 20, -1.0, 1e-3)
    assert L.dhfwi_create(ctypes.byref(h), ctypes.byref(g), 0) == -1
    assert h.value is None


def test_null_context_is_rejected():
    from paper_2403_17518_gb300 import _lib

    L = _lib.load()
    assert L.model_shots(None, None, None, None, None) == -1
    assert L.image_laplacian(None, None, None, None) == -1
    assert L.dhfwi_selftest_timeout(None, None) == -1
    L.dhfwi_destroy(None)  # accepted


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2403_17518_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "liboracle" not in txt, f


def test_ctypes_structs_match_the_header(tmp_path):
    """Every field offset and struct size of the binding's ctypes mirrors
    equals the C compiler's layout of include/dhfwi.h (a mismatch would pass
    garbage through the ABI without any error)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2403_17518_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"dhfwi_grid": _lib.Grid, "dhfwi_geom": _lib.Geom, "dhfwi_stats_t": _lib.Stats,
               "dhfwi_train_cfg": _lib.TrainCfg}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dhfwi.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
