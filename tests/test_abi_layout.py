"""The Python binding's ctypes structs against the C header: every struct the
binding passes through the C ABI has the header's size, and each of its
fields the header's name and offset.  Compiles a small C program against
include/ecris.h with the host compiler (no GPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("Geometry", "ecris_geometry"), ("BField", "ecris_bfield"), ("Grid", "ecris_grid"),
         ("Species", "ecris_species"), ("Mcc", "ecris_mcc"), ("DiagOut", "ecris_diag_out"),
         ("Tuning", "ecris_tuning"), ("Request", "ecris_request"), ("Result", "ecris_result"),
         ("CalibRequest", "ecris_calib_request"), ("CalibResult", "ecris_calib_result"),
         ("ProbeSpec", "ecris_probe_spec"), ("Profile", "ecris_profile")]


@pytest.fixture(scope="module")
def layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_1507_03392_gb300 import ecris as E
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ecris.h"', "int main(void) {"]
    for py, c in PAIRS:
        lines.append(f'    printf("{c} %zu\\n", sizeof({c}));')
        for name, _ in getattr(E, py)._fields_:
            lines.append(f'    printf("{c}.{name} %zu\\n", offsetof({c}, {name}));')
    lines += ["    return 0;", "}"]
    d = os.path.join(ROOT, "paper_1507_03392_gb300", "_build", "abi")   # the package's build folder
    os.makedirs(d, exist_ok=True)
    src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr   # a field the header does not have fails here
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return E, dict(line.rsplit(" ", 1) for line in out.splitlines())


@pytest.mark.parametrize("py,c", PAIRS)
def test_struct_matches_header(layout, py, c):
    E, got = layout
    S = getattr(E, py)
    assert ctypes.sizeof(S) == int(got[c])
    for name, _ in S._fields_:
        assert getattr(S, name).offset == int(got[f"{c}.{name}"]), name
