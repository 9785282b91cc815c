"""The C ABI seen from plain C and from the Python binding agree: include/qeq.h compiles as pedantic
C99 with warnings as errors, and a C program compiled against it prints the size and every field
offset of qeq_plan_desc, qeq_info and qeq_plan_info and the value of every QEQ_ constant the binding
defines; the ctypes structures and constants of paper_2607_17978_b300/qeq.py must match them."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2607_17978_b300 import qeq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"qeq_plan_desc": qeq.PlanDesc, "qeq_info": qeq.Info, "qeq_plan_info": qeq.PlanInfo}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_ctypes_layouts_and_constants_match_the_header(tmp_path):
    consts = sorted(k for k, v in vars(qeq).items() if k.startswith("QEQ_") and isinstance(v, int))
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "qeq.h"', "int main(void) {"]
    for cname, S in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in S._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    for k in consts:
        lines.append(f'  printf("const {k} %lld\\n", (long long)({k}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, S in STRUCTS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(S), cname
        for f in S._fields_:
            assert got[(cname, f[0])] == getattr(S, f[0]).offset, (cname, f[0])
    for k in consts:
        assert got[("const", k)] == getattr(qeq, k), k
