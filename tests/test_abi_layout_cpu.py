"""The C ABI seen from plain C and from the Python binding agree: include/qeq.h compiles as pedantic
C99 with warnings as errors, and a C program compiled against it prints the size and every field
offset of qeq_plan_desc, qeq_info and qeq_plan_info and the value of every QEQ_ constant the binding
defines; the ctypes structures and constants of paper_2607_17978_b300/qeq.py must match them.  Every
declared function's ctypes prototype has the header's parameter count, and each parameter and the
return value the same kind (pointer or handle, integer or floating point of the same size)."""
import ctypes
import os
import re
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


_C_SCALARS = {"int32_t": ("int", 4), "int64_t": ("int", 8), "qeq_status": ("int", 4), "double": ("float", 8),
              "float": ("float", 4)}
_HANDLES = ("qeq_plan", "qeq_dense", "qeq_mlp")


def _c_kind(decl):
    decl = " ".join(decl.replace("const ", "").split())
    if "*" in decl:
        return ("ptr",)
    typ = decl.split()[0]
    if typ in _HANDLES:
        return ("ptr",)
    return _C_SCALARS[typ]


def _ct_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return ("ptr",)
    if t in (ctypes.c_float, ctypes.c_double):
        return ("float", ctypes.sizeof(t))
    return ("int", ctypes.sizeof(t))


def test_ctypes_prototypes_match_the_header():
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "qeq.h")).read(), flags=re.S)
    decls = re.findall(r"([A-Za-z_][A-Za-z_0-9 *]*?)\b(qeq_[a-z_]+)\s*\(([^)]*)\)\s*;", src)
    assert len(decls) == len(qeq.EXPORTED)
    from paper_2607_17978_b300 import build
    build.build()
    lib = qeq.load_library()
    for ret, name, args in decls:
        fn = getattr(lib, name)
        params = [a for a in args.split(",") if a.strip() and a.strip() != "void"]
        assert fn.argtypes is not None and len(fn.argtypes) == len(params), name
        for c, t in zip(params, fn.argtypes):
            assert _c_kind(c) == _ct_kind(t), (name, c, t)
        ret = ret.strip()
        if ret == "void":
            assert fn.restype is None, name
        else:
            assert _c_kind(ret) == _ct_kind(fn.restype), (name, ret, fn.restype)

