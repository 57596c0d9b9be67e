"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point that include/pcloth.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^PC_API[^;(]*?\b(pc_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2008_00409_gb300 import build
    return build.build()


def test_header_declares_the_four_hot_path_calls():
    names = declared_symbols()
    for n in ("pc_assemble_pattern", "pc_assemble_values", "pc_pcg_solve", "pc_step"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pc_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.pc_status_string.restype = ctypes.c_char_p
    assert lib.pc_status_string(0) == b"ok"
    assert b"converge" in lib.pc_status_string(3)


def test_binding_loads_and_names_match(libpath):
    from paper_2008_00409_gb300 import pcloth
    for name in declared_symbols():
        assert callable(getattr(pcloth.lib(), name))
    for name in ("pc_create", "pc_destroy", "pc_assemble_pattern", "pc_assemble_values", "pc_bsr_spmv",
                 "pc_pcg_solve", "pc_step", "pc_step_host"):
        assert callable(getattr(pcloth, name))
