"""The Python binding mirrors include/fe.h exactly (no GPU needed): every constant the header defines has the same
value in the binding, and the ctypes structures have the C structures' size and field offsets.  A C program
generated from the binding's own field and constant names is compiled against the header, so a renamed, reordered
or retyped field fails here instead of corrupting arguments at run time."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fe.h")


def header_constants():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^#define\s+(FE_[A-Z0-9_]+)\s+\S", src, flags=re.M)) - {"FE_GB300_H"})


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    import paper_2104_08012_gb300 as fe
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fe.h"', "int main(void) {"]
    for cname, py in (("fe_solver_opts", fe.SolverOpts), ("fe_solve_stats", fe.SolveStats)):
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("field {cname} {field} %zu %zu\\n", offsetof({cname}, {field}), '
                         f'sizeof((({cname}*)0)->{field}));')
    for name in header_constants():
        lines.append(f'  printf("const {name} %d\\n", (int)({name}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi_layout")
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(d / "layout")
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    return [line.split() for line in out if line]


def test_structures_match(c_layout):
    import paper_2104_08012_gb300 as fe
    py = {"fe_solver_opts": fe.SolverOpts, "fe_solve_stats": fe.SolveStats}
    import ctypes
    for rec in c_layout:
        if rec[0] == "size":
            assert int(rec[2]) == ctypes.sizeof(py[rec[1]]), rec
        elif rec[0] == "field":
            f = getattr(py[rec[1]], rec[2])
            assert (int(rec[3]), int(rec[4])) == (f.offset, f.size), rec


def test_constants_match(c_layout):
    import paper_2104_08012_gb300 as fe
    consts = [rec for rec in c_layout if rec[0] == "const"]
    assert len(consts) == len(header_constants()) > 20
    for _, name, value in consts:
        assert hasattr(fe, name), f"{name} missing from the binding"
        assert getattr(fe, name) == int(value), name


def header_prototypes():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"^\s*((?:const\s+)?[a-z_ ]+?\**)\s*\b(fe_[a-z0-9_]+)\s*\(([^;]*?)\)\s*;",
                                        src, flags=re.M | re.S):
        ps = [p.strip() for p in params.split(",")] if params.strip() not in ("", "void") else []
        protos[name] = (ret.strip(), ps)
    return protos


def _kind_c(decl):
    decl = " ".join(decl.split())
    if "*" in decl:
        return "ptr"
    if "long long" in decl:
        return "ll"
    if "double" in decl:
        return "d"
    if decl.startswith("int") or decl.startswith("const int") or decl == "int":
        return "i"
    if decl.startswith("void"):
        return "void"
    raise AssertionError(decl)


def _kind_py(t):
    import ctypes
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    return {ctypes.c_int: "i", ctypes.c_double: "d", ctypes.c_longlong: "ll"}[t]


def test_function_signatures_match(c_layout):
    import paper_2104_08012_gb300 as fe
    lib = fe.load()
    protos = header_prototypes()
    assert set(protos) == set(fe.EXPORTED)
    for name, (ret, params) in protos.items():
        f = getattr(lib, name)
        assert _kind_py(f.restype) == _kind_c(ret), (name, ret, f.restype)
        assert [_kind_py(a) for a in f.argtypes] == [_kind_c(p) for p in params], (name, params, f.argtypes)
