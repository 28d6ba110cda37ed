"""The ctypes binding's structures match the C declarations of include/crhyb.h.

A small C program, compiled here with the host compiler against the header,
prints sizeof and every field's offset; each ctypes Structure of the binding
must agree field by field (a field added on one side only, or in another
order, shifts every later option the library reads).  No GPU is needed.
"""

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2101_03777_gb300 import crhyb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [crhyb.cr_mesh_opts, crhyb.cr_params, crhyb.cr_hyb_opts, crhyb.cr_solve_opts, crhyb.cr_solve_stats,
           crhyb.cr_batch_opts, crhyb.cr_newton_stats]


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "crhyb.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "abi_probe.c"
    exe = tmp_path / "abi_probe"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        struct, field, value = line.split()
        layout[(struct, field)] = int(value)
    return layout


def test_structures_match_the_header(tmp_path):
    layout = c_layout(tmp_path)
    for st in STRUCTS:
        name = st.__name__
        assert layout[(name, "sizeof")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert layout[(name, field)] == getattr(st, field).offset, (name, field)
