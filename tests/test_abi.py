"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sbp_\w+)\s*\(",
                                text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2601_00551_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_symbols()
    for fn in ("sbp_create_array", "sbp_set_sampling_level", "sbp_forward", "sbp_residual",
               "sbp_adjoint", "sbp_filter_grow", "sbp_destroy_array"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(lib):
    lib.sbp_version.restype = ctypes.c_char_p
    lib.sbp_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sbp_version()
    assert isinstance(lib.sbp_last_error(), bytes)


def test_create_array_rejects_bad_arguments_on_the_host(lib):
    """Argument checks run before any CUDA call, so they work without a GPU."""
    out = ctypes.c_void_p()
    pos = (ctypes.c_float * 3)(0, 0, 0)
    nrm = (ctypes.c_float * 3)(0, 0, 1)
    fac = (ctypes.c_int * 1)(1)
    f = lib.sbp_create_array
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                  ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert f(pos, nrm, 0, 1.5, 40.0, 128, fac, 1, 10, None, ctypes.byref(out)) == -1   # M = 0
    assert f(pos, nrm, 1, -1.0, 40.0, 128, fac, 1, 10, None, ctypes.byref(out)) == -1  # c < 0
    bad = (ctypes.c_int * 1)(0)
    assert f(pos, nrm, 1, 1.5, 40.0, 128, bad, 1, 10, None, ctypes.byref(out)) == -1   # f = 0
    zero = (ctypes.c_float * 3)(0, 0, 0)
    assert f(pos, zero, 1, 1.5, 40.0, 128, fac, 1, 10, None, ctypes.byref(out)) == -6  # |n| = 0
    assert out.value is None
