"""The ctypes structures of the binding lay out memory exactly like the C structs of include/mgmlmc.h: a small C
program compiled here with the system C compiler prints sizeof and every field's offsetof, and each must equal
the ctypes figure (a mismatch would make the library read or write the wrong bytes of a parameter block)."""
import os
import shutil
import subprocess

import pytest

from paper_2303_11512_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [("mg_params", _lib.MgParams), ("solve_params", _lib.SolveParams), ("solve_stats", _lib.SolveStats),
           ("est_params", _lib.EstParams), ("est_result", _lib.EstResult), ("hutch_params", _lib.HutchParams),
           ("hutch_result", _lib.HutchResult)]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mgmlmc.h"', "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for field in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field[0], cname, field[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        struct, field, value = line.split()
        got[struct, field] = int(value)
    import ctypes
    for cname, cls in STRUCTS:
        assert got[cname, "sizeof"] == ctypes.sizeof(cls), cname
        for field in cls._fields_:
            assert got[cname, field[0]] == getattr(cls, field[0]).offset, (cname, field[0])


def _prototypes():
    """name -> (return type, [argument types]) of every function the header declares (comments removed)."""
    import re
    src = open(os.path.join(ROOT, "include", "mgmlmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for m in re.finditer(r"^\s*((?:const\s+)?[A-Za-z_]\w*\s*\**)\s*([A-Za-z_]\w*)\s*\(([^)]*)\)\s*;", src, re.M):
        ret, name, args = m.group(1), m.group(2), m.group(3).strip()
        params = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
        out[name] = (ret.strip(), params)
    return out


def _kind_of_c(decl: str) -> str:
    """Calling-convention class of a C parameter or return type: pointer, double, int64, uint64, int, void."""
    if "*" in decl:
        return "pointer"
    words = decl.replace("const", "").split()
    base = words[0] if words else ""
    return {"double": "double", "int64_t": "int64", "uint64_t": "uint64", "int": "int", "void": "void"}[base]


def _kind_of_ctypes(t) -> str:
    import ctypes as C
    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or hasattr(t, "contents") or t.__name__.startswith("LP_"):
        return "pointer"
    return {C.c_double: "double", C.c_int64: "int64", C.c_uint64: "uint64", C.c_int: "int"}[t]


def test_ctypes_signatures_match_the_prototypes():
    """Every entry point's ctypes argument and return types have the C prototype's calling-convention classes
    (pointer, double, 64-bit or 32-bit integer), in the same number and order."""
    protos = _prototypes()
    assert set(protos) == set(_lib.SIGNATURES)
    for name, (res, args) in _lib.SIGNATURES.items():
        cret, cargs = protos[name]
        assert _kind_of_ctypes(res) == _kind_of_c(cret), name
        assert len(args) == len(cargs), (name, len(args), len(cargs))
        for i, (a, c) in enumerate(zip(args, cargs)):
            assert _kind_of_ctypes(a) == _kind_of_c(c.rsplit(" ", 1)[0] if "*" not in c else c), (name, i, c)


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, precisions, forms, policies, noise kinds, trace weights, stream phases and the level limit
    of the binding have the header's values (printed by a C program compiled on the host)."""
    import re
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    hdr = open(os.path.join(ROOT, "include", "mgmlmc.h")).read()
    names = sorted(set(re.findall(r"\bMGMLMC_([A-Z0-9_]+)\s*=", hdr)))
    assert len(names) > 20
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "mgmlmc.h"\nint main(void) {\n'
                   + "".join('printf("%s %%d\\n", (int)MGMLMC_%s);\n' % (n, n) for n in names + ["MAX_LEVELS"])
                   + "return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    values = dict((a, int(b)) for a, b in (line.split() for line in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()))
    checked = 0
    for name, value in values.items():
        if hasattr(_lib, name):
            assert getattr(_lib, name) == value, name
            checked += 1
    assert checked >= 25
