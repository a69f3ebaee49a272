"""The Python binding's ctypes structures match the C header byte for byte: a small C
program compiled against include/nsp.h prints the size of each structure and the offset of
each field, which must equal what ctypes computes (a field added on one side only would
shift every field after it)."""

import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = ["nsp_csr", "nsp_partition", "nsp_params", "nsp_info"]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structures_match_the_header(tmp_path):
    import paper_2101_12164_gb300 as N
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nsp.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(N, name)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for name in STRUCTS:
        cls = getattr(N, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
