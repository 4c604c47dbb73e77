"""The C ABI without a device: libsph.so cross-compiles for sm_103a, loads,
and exports every function that include/sph.h declares; the calls that fail
on their arguments alone do so before touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = re.sub(r"#[^\n]*", " ", text)
    return sorted(set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libsph():
    from paper_1604_03290_gb300 import build
    return C.CDLL(build.build())


def test_header_declares_the_entry_points():
    names = declared_functions()
    for f in ("sph_create", "sph_destroy", "sph_build_tree", "sph_neighbours", "sph_rhs", "sph_gravity",
              "sph_step", "sph_rhs_adjoint", "sph_pc_update", "sph_pc_update_adjoint", "sph_sync_status"):
        assert f in names


def test_library_exports_every_declared_function(libsph):
    missing = [f for f in declared_functions() if not hasattr(libsph, f)]
    assert not missing, missing


def test_argument_errors_need_no_device(libsph):
    SPH_ERR_INVALID = 1
    libsph.sph_create.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
    libsph.sph_create.restype = C.c_int
    assert libsph.sph_create(None, 3, 1000, 1, 64, 16, None) == SPH_ERR_INVALID
    h = C.c_void_p()
    assert libsph.sph_create(C.byref(h), 4, 1000, 1, 64, 16, None) == SPH_ERR_INVALID  # dim 4
    assert libsph.sph_create(C.byref(h), 3, 1000, 1, 64, 33, None) == SPH_ERR_INVALID  # leaf > 32
    assert h.value is None
    libsph.sph_last_error.argtypes = [C.c_void_p]
    libsph.sph_last_error.restype = C.c_char_p
    assert libsph.sph_last_error(None) == b"no context"
    for f in ("sph_rhs", "sph_step", "sph_neighbours", "sph_gravity"):
        getattr(libsph, f).restype = C.c_int
    assert libsph.sph_rhs(None, None, None, 0, None, None, None) == SPH_ERR_INVALID
    assert libsph.sph_neighbours(None, None, 16, 21, None, None, C.c_int64(0), None) == SPH_ERR_INVALID


STRUCTS = {"sph_material": "Material", "sph_params": "Params", "sph_state": "State", "sph_derivs": "Derivs",
           "sph_tuning": "Tuning"}


def _c_fields(struct):
    """Field names of a typedef'd struct in the header, in order."""
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


def test_header_is_plain_c_and_the_binding_matches_its_layout(tmp_path):
    # the header compiles as C99 on its own, and every ctypes mirror in the
    # binding has the C struct's size and field offsets
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1604_03290_gb300 import sph
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sph.h"', "int main(void) {"]
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
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cs, py in STRUCTS.items():
        cls = getattr(sph, py)
        assert C.sizeof(cls) == got[(cs, "size")], cs
        cfields = _c_fields(cs)
        assert [f[0] for f in cls._fields_] == cfields, cs
        for f in cfields:
            assert getattr(cls, f).offset == got[(cs, f)], (cs, f)


def test_static_entry_rejects_huge_instance_counts_on_the_host(libsph):
    # ninst = INT32_MAX needs 31 instance bits, more than a 3D key at depth 21
    # leaves: SPH_ERR_INVALID from argument checks, before any device call
    from paper_1604_03290_gb300 import sph
    SPH_ERR_INVALID = 1
    st = sph.State()
    st.dim, st.ninst, st.n = 3, 2 ** 31 - 1, 10
    dummy = C.c_double(0.0)
    for ax in range(3):
        st.x[ax] = st.v[ax] = C.cast(C.byref(dummy), C.c_void_p)
    st.rho = st.u = st.m = st.h = st.inst_off = C.cast(C.byref(dummy), C.c_void_p)
    f = libsph.sph_neighbours_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_char_p,
                  C.c_int32, C.c_void_p]
    msg = C.create_string_buffer(256)
    out = C.c_int64(0)
    r = f(C.byref(st), 16, 21, 64, C.byref(out), C.byref(out), 0, msg, 256, None)
    assert r == SPH_ERR_INVALID
    assert b"max_depth" in msg.value
