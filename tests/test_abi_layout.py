"""The Python binding agrees with include/pcloth.h without a GPU: every #define that the
binding mirrors has the header's value, and every structure that the binding declares with
ctypes has the size and field offsets that the C compiler gives the header's struct (a
field added to one side only, or in another order, fails here instead of corrupting a call)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcloth.h")

# structures passed by pointer or by value through the C ABI, and the module declaring each
STRUCTS = [("pcloth", "pc_material"), ("pcloth", "pc_contacts"), ("pcloth", "pc_bsr"),
           ("pcloth", "pc_solve_opts"), ("pcloth", "pc_solve_info"), ("pcloth", "pc_step_opts"),
           ("pcloth", "pc_step_info"), ("pcloth", "pc_adam_opts"), ("dist", "pc_comm")]


def header_defines():
    text = open(HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (PC_\w+)\s+(-?\d+)\b", text, flags=re.M)}


def binding_struct(module, name):
    import importlib
    return getattr(importlib.import_module(f"paper_2008_00409_gb300.{module}"), name)


def test_binding_constants_match_the_header():
    from paper_2008_00409_gb300 import pcloth
    defs = header_defines()
    mirrored = [n for n in defs if hasattr(pcloth, n)]
    for n in ("PC_OK", "PC_ERR_TIMEOUT", "PC_ERR_MESH", "PC_PREC_MIXED", "PC_SCHED_AUTO", "PC_SCHED_GRID",
              "PC_SCHED_CLUSTER", "PC_WARM_MLP", "PC_WARM_COMBINED"):
        assert n in mirrored, n
    for n in mirrored:
        assert getattr(pcloth, n) == defs[n], n


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pcloth.h"', "int main(void) {"]
    for module, name in STRUCTS:
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in binding_struct(module, name)._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("    return 0;\n}")
    d = tmp_path_factory.mktemp("abi_layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


@pytest.mark.parametrize("module,name", STRUCTS)
def test_binding_structure_matches_the_c_layout(c_layout, module, name):
    cls = binding_struct(module, name)
    assert ctypes.sizeof(cls) == c_layout[(name, "size")]
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(name, field)], field
