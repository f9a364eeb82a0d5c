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
