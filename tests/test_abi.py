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


def declared_parameter_counts():
    counts = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, params in re.findall(r"\b(sbp_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
            p = params.strip()
            counts[name] = 0 if p in ("", "void") else len(p.split(","))
    return counts


def test_python_binding_covers_every_entry_point_with_its_arity():
    """The binding is argument marshalling only: one ctypes signature per
    declared entry point, with the header's number of parameters."""
    from paper_2601_00551_gb300 import slingbag

    counts = declared_parameter_counts()
    assert set(counts) == declared_symbols()
    missing = sorted(set(counts) - set(slingbag._SIGS))
    assert not missing, missing
    wrong = {n: (counts[n], len(slingbag._SIGS[n][1])) for n in counts
             if len(slingbag._SIGS[n][1]) != counts[n]}
    assert not wrong, wrong


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


def test_new_entry_points_reject_bad_arguments_on_the_host(lib):
    """The envelope, voxel grid, convolution and CNN entry points check their
    arguments (and build the hull) on the host before any CUDA call."""
    P = ctypes.c_void_p
    out = ctypes.c_void_p()
    f = lib.sbp_envelope_create
    f.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    pts = (ctypes.c_float * 30)(*([0.0] * 30))
    assert f(pts, 3, ctypes.byref(out)) == -1  # fewer than 4 sensors
    # ten sensors in the plane z = 1.5: no closed envelope
    flat = (ctypes.c_float * 30)(*[v for i in range(10) for v in (float(i % 4), float(i // 4), 1.5)])
    assert f(flat, 10, ctypes.byref(out)) == -1
    nan = (ctypes.c_float * 12)(*([0.0] * 11 + [float("nan")]))
    assert f(nan, 4, ctypes.byref(out)) == -6  # SBP_ERR_NUMERIC
    g = lib.sbp_conv3d_bf16
    g.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P,
                  ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P]
    assert g(None, 4, 4, 4, 16, None, 448, None, 32, 1, None, 0, None) == -1
    buf = (ctypes.c_char * 64)()
    addr = (ctypes.addressof(buf) + 15) // 16 * 16
    assert g(addr, 4, 4, 4, 16, addr, 430, None, 32, 1, addr, 0, None) == -1  # kp % 64
    assert g(addr, 4, 4, 4, 16, addr, 448, None, 48, 1, addr, 0, None) == -1  # unsupported cout
    c = lib.sbp_cnn_create
    c.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                  ctypes.POINTER(ctypes.c_void_p)]
    assert c(0, 4, 4, 1, ctypes.byref(out)) == -1
    v = lib.sbp_voxelize
    v.restype = ctypes.c_int
    assert lib.sbp_cnn_num_params() == 16 * 27 + 16 + 32 * 27 * 16 + 32 + 64 * 27 * 32 + 64 + 128 + 2


def test_tile_entry_points_reject_a_null_array_on_the_host(lib):
    """The per-level tile calls check their array before any CUDA call."""
    P = ctypes.c_void_p
    lib.sbp_set_tiles.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.sbp_get_tiles.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    assert lib.sbp_set_tiles(None, 0, 256, 2) == -1
    c, s = ctypes.c_int(7), ctypes.c_int(7)
    assert lib.sbp_get_tiles(None, 0, ctypes.byref(c), ctypes.byref(s)) == -1
    assert (c.value, s.value) == (7, 7)  # untouched
    lib.sbp_last_error.restype = ctypes.c_char_p
    assert b"null array" in lib.sbp_last_error()


def test_forward_static_binding_checks_its_arguments_on_the_host():
    """Shapes, dtypes and devices are checked before the library is called."""
    import torch

    from paper_2601_00551_gb300 import slingbag

    balls = torch.zeros((5, 4))
    on_host = torch.zeros((6, 4))
    three_rows = torch.zeros((3, 4))
    doubles = torch.zeros((6, 4), dtype=torch.float64)
    for sensors in (on_host, three_rows, doubles):
        with pytest.raises(ValueError):
            slingbag.forward_static(sensors, 1.5, 0.025, 16, balls)


def test_pointers_must_be_device_memory():
    """The binding refuses host tensors for every device pointer, before any
    call into the library (a host pointer would reach a kernel)."""
    import torch

    from paper_2601_00551_gb300 import slingbag as sb

    with pytest.raises(ValueError):
        sb._dptr(torch.zeros(4))
    with pytest.raises(ValueError):
        sb._rows(torch.zeros((5, 4)))
    assert sb._dptr(None) is None
