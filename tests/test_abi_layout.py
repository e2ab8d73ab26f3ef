"""The ctypes structures of the binding against the C header's layout: gcc
compiles include/hirep_gb300.h and prints sizeof and every field's offsetof;
each must match the ctypes structure of paper_2411_18511_gb300/hr.py (a
mismatch would pass wrong values silently)."""

import os
import shutil
import subprocess

import pytest

from paper_2411_18511_gb300 import hr

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")

STRUCTS = [hr.hr_lattice, hr.hr_solver_opts, hr.hr_hmc_params, hr.hr_hmc_info, hr.hr_tune_result,
           hr.hr_solve_info]


def _program():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hirep_gb300.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    return "\n".join(lines)


def test_ctypes_structures_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(_program())
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for st in STRUCTS:
        name = st.__name__
        assert got[(name, "sizeof")] == __import__("ctypes").sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
