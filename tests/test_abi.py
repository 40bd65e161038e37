"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports
every entry point include/ecris.h declares; calls that need no device reject
NULL arguments."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "ecris.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ecris_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_03392_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_library_exports_every_declared_entry_point(lib):
    _, path = lib
    names = declared_entry_points()
    assert "ecris_step" in names and "ecris_init_fields" in names
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ecris_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_null_arguments_are_rejected_without_a_device(lib):
    L, _ = lib
    L.ecris_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert L.ecris_create(None, 0, None) == 1          # ECRIS_EINVAL
    L.ecris_last_error.restype = ctypes.c_char_p
    assert b"NULL" in L.ecris_last_error(None)
    for name in ("ecris_step", "ecris_diag", "ecris_get_state", "ecris_load_ions", "ecris_init_fields"):
        f = getattr(L, name)
        f.restype = ctypes.c_int
    L.ecris_step.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_double]
    assert L.ecris_step(None, 1, 1e-9) == 1
    L.ecris_diag.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert L.ecris_diag(None, None) == 1


def test_binding_loads_and_names_match(lib):
    from paper_1507_03392_gb300 import ecris as E
    for n in declared_entry_points():
        assert callable(getattr(E, n))
