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
