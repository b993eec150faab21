"""The ctypes structures of the Python binding have the layout of the C header's structures: a
small C program that includes include/chns.h prints sizeof and offsetof of every field (host
compiler, no GPU), and the binding's ctypes.sizeof / field offsets must agree. A field added on
one side only (or in a different order) shifts every later field and fails here."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2107_05123_gb300 import _lib as capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["chns_mesh_info", "chns_params", "chns_coef", "chns_solver_params", "chns_solve_stats",
           "chns_state", "chns_step_params", "chns_step_stats", "chns_mg_params"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chns.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in getattr(capi, name)._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        parts = line.split()
        table[tuple(parts[:-1])] = int(parts[-1])
    return table


def test_binding_structs_match_the_header(tmp_path):
    table = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(capi, name)
        assert ctypes.sizeof(cls) == table[(name, "size")], name
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == table[(name, fname)], (name, fname)
