"""The Python binding's ctypes structures against the C header: a small C program built with the
host compiler prints sizeof and offsetof of every member of every struct the boundary takes, and
each must equal what ctypes lays out (a member added on one side only shifts every later one)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2501_18781_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = {"OpParams": "mf_op_params", "SolverParams": "mf_solver_params", "SolveInfo": "mf_solve_info",
         "Evaporation": "mf_evaporation", "Laser": "mf_laser", "MeltPoolParams": "mf_meltpool_params",
         "MeltPoolInfo": "mf_meltpool_info", "MeltPoolTrace": "mf_meltpool_trace"}


def test_ctypes_structures_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mfgb.h"', "int main(void) {"]
    expected = {}
    for py, c in PAIRS.items():
        cls = getattr(_lib, py)
        lines.append(f'printf("{py} %zu\\n", sizeof({c}));')
        expected[py] = ctypes.sizeof(cls)
        for name, *_ in cls._fields_:
            lines.append(f'printf("{py}.{name} %zu\\n", offsetof({c}, {name}));')
            expected[f"{py}.{name}"] = getattr(cls, name).offset
    lines.append("return 0; }")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    subprocess.run([cc, "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {k: int(v) for k, v in (line.split() for line in out if line)}
    assert got == expected

