"""The oracle's C interface and its Python wrapper agree: oracle/oracle.h
compiles as C99 alone, and every ctypes mirror in oracle/__init__.py has the C
struct's size, field names and offsets (a mismatch would feed the oracle
shifted fields and every pin and parity test would read garbage)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "oracle", "oracle.h")
STRUCTS = {"orc_material": "Material", "orc_params": "Params", "orc_state": "State", "orc_derivs": "Derivs"}


def _c_fields(struct):
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    body = dict((n, b) for b, n in re.findall(r"typedef struct \{([^{}]*)\}\s*(\w+);", text))[struct]
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*(\[[^\]]*\])?\s*$", part.strip())
            names.append(m.group(1))
    return names


def test_oracle_header_and_wrapper_layouts_agree(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import oracle
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "oracle.h"', "int main(void) {"]
    for cs in STRUCTS:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cs, cs))
        for f in _c_fields(cs):
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cs, f, cs, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cs, py in STRUCTS.items():
        cls = getattr(oracle, py)
        assert C.sizeof(cls) == got[(cs, "size")], cs
        cfields = _c_fields(cs)
        assert [f[0] for f in cls._fields_] == cfields, (cs, [f[0] for f in cls._fields_], cfields)
        for f in cfields:
            assert getattr(cls, f).offset == got[(cs, f)], (cs, f)
