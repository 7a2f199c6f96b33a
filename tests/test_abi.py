"""The C ABI library builds, loads and exports every entry point include/tds.h declares;
host-side argument checks return their status before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2411_13532_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tds.h")).read()
    return re.findall(r"TDS_API\s+[\w\s\*]+?\**\s*(tds_\w+)\s*\(", text)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("tds_plan_create", "tds_plan_destroy", "tds_workspace_bytes", "tds_deriv",
                     "tds_deriv_adjoint", "tds_reorder", "tds_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    from paper_2411_13532_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    # the binding covers exactly the declared entry points
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == sorted(names)


def test_status_strings(L):
    for code in range(8):
        s = L.tds_status_string(code)
        assert s and s != b"unknown status"
    assert L.tds_status_string(99) == b"unknown status"


def test_plan_argument_errors_need_no_gpu(L):
    from paper_2411_13532_gb300 import _lib
    h = ctypes.c_void_p()
    cases = [
        # (nx, ny, nz, dir, order, bc, P, h, dtype, sz, mode) -> status
        ((64, 64, 64, 0, 3, 0, 1, 0.1, 0, 32, 0), _lib.ERR_ARG),      # order
        ((64, 64, 64, 5, 1, 0, 1, 0.1, 0, 32, 0), _lib.ERR_ARG),      # dir
        ((64, 64, 64, 0, 1, 2, 1, 0.1, 0, 32, 0), _lib.ERR_ARG),      # bc
        ((64, 64, 64, 0, 1, 0, 1, -1.0, 0, 32, 0), _lib.ERR_ARG),     # h
        ((64, 64, 64, 0, 1, 0, 1, 0.1, 2, 32, 0), _lib.ERR_ARG),      # dtype
        ((64, 64, 64, 0, 1, 0, 1, 0.1, 0, 16, 0), _lib.ERR_ARG),      # SZ
        ((64, 64, 64, 0, 1, 0, 0, 0.1, 0, 32, 0), _lib.ERR_ARG),      # P
        ((64, 64, 64, 0, 1, 0, 3, 0.1, 0, 32, 0), _lib.ERR_SHAPE),    # n % P
        ((64, 64, 64, 0, 1, 0, 32, 0.1, 0, 32, 0), _lib.ERR_SHAPE),   # m < 4
        ((4, 64, 64, 0, 1, 0, 1, 0.1, 0, 32, 0), _lib.ERR_SHAPE),     # n < 8
        ((64, 5, 3, 0, 1, 0, 1, 0.1, 0, 32, 0), _lib.ERR_SHAPE),      # lines % 32
    ]
    for args, want in cases:
        assert L.tds_plan_create(ctypes.byref(h), *args) == want, args
        assert not h.value


def test_null_pointer_errors_need_no_gpu(L):
    from paper_2411_13532_gb300 import _lib
    assert L.tds_plan_create(None, 64, 64, 64, 0, 1, 0, 1, 0.1, 0, 32, 0) == _lib.ERR_ARG
    assert L.tds_deriv(None, None, None, None, 0, None) == _lib.ERR_ARG
    assert L.tds_deriv_adjoint(None, None, None, None, 0, None) == _lib.ERR_ARG
    assert L.tds_solve(None, None, None, None, 0, None) == _lib.ERR_ARG
    assert L.tds_deriv_thomas(None, None, None, None) == _lib.ERR_ARG
    h = ctypes.c_void_p()
    assert L.tds_plan_create_band(ctypes.byref(h), 64, 64, 64, 0, None, None, None, 0, 1, 0, 32, 0) == _lib.ERR_ARG
    assert L.tds_plan_create_band(None, 64, 64, 64, 0, None, None, None, 0, 1, 0, 32, 0) == _lib.ERR_ARG
    assert L.tds_deriv_host(None, None, None, None, None, None, 0, None) == _lib.ERR_ARG
    assert L.tds_deriv_multi(0, None, None, None, None, None, 0, None) == _lib.ERR_ARG
    assert L.tds_deriv_multi(5, None, None, None, None, None, 0, None) == _lib.ERR_ARG
    assert L.tds_deriv_adjoint_host(None, None, None, None, None, None, 0, None) == _lib.ERR_ARG
    sz = ctypes.c_size_t()
    assert L.tds_workspace_bytes(None, ctypes.byref(sz)) == _lib.ERR_ARG
    assert L.tds_reorder(None, None, 32, 32, 1, 0, 1, 0, 32, None) == _lib.ERR_ARG
    assert L.tds_reorder_add(None, None, 32, 32, 1, 0, 1, 0, 32, None) == _lib.ERR_ARG
    assert L.tds_transport(None, None, None, None, 0.1, None, None) == _lib.ERR_ARG
    assert L.tds_plan_create_filter(None, 64, 64, 64, 0, 0.4, 0, 1, 0, 32, 0) == _lib.ERR_ARG
    assert L.tds_plan_create_interp(None, 64, 64, 64, 0, 0, 1, 0, 32, 0) == _lib.ERR_ARG
    # argument and shape rules of the filter and interpolation plans, checked before the device
    for af, want in ((0.5, _lib.ERR_ARG), (-0.5, _lib.ERR_ARG), (float("nan"), _lib.ERR_ARG)):
        assert L.tds_plan_create_filter(ctypes.byref(h), 64, 64, 64, 0, af, 0, 1, 0, 32, 0) == want
        assert not h.value
    assert L.tds_plan_create_filter(ctypes.byref(h), 64, 64, 64, 0, 0.4, 0, 3, 0, 32, 0) == _lib.ERR_SHAPE
    assert L.tds_plan_create_interp(ctypes.byref(h), 64, 64, 64, 3, 0, 1, 0, 32, 0) == _lib.ERR_ARG
    assert L.tds_plan_create_interp(ctypes.byref(h), 64, 64, 64, 0, 2, 1, 0, 32, 0) == _lib.ERR_ARG
    assert L.tds_plan_create_interp(ctypes.byref(h), 64, 64, 64, 0, 1, 32, 0, 32, 0) == _lib.ERR_SHAPE
    assert not h.value
    assert L.tds_plan_set_width(None, 32) == _lib.ERR_ARG
    assert L.tds_plan_set_arith(None, 1) == _lib.ERR_ARG
    assert L.tds_fanout_copy(None, None, 1, 16, None) == _lib.ERR_ARG
    w = ctypes.c_int()
    assert L.tds_plan_width(None, ctypes.byref(w)) == _lib.ERR_ARG
    assert L.tds_plan_run_chunks(None, ctypes.byref(w)) == _lib.ERR_ARG
    L.tds_plan_destroy(None)


def test_reorder_shape_errors_need_no_gpu(L):
    from paper_2411_13532_gb300 import _lib
    buf = (ctypes.c_double * 2)()
    a = ctypes.addressof(buf)
    a16 = (a + 15) & ~15
    # nx not a multiple of 32 -> shape error before any launch (pointers never dereferenced)
    assert L.tds_reorder(ctypes.c_void_p(a16), ctypes.c_void_p(a16 + 4096), 48, 32, 2, 0, 1, 0,
                         32, None) == _lib.ERR_SHAPE
    assert L.tds_reorder(ctypes.c_void_p(a16), ctypes.c_void_p(a16 + 8), 32, 32, 1, 0, 1, 0,
                         32, None) == _lib.ERR_ARG  # misaligned out
    # the accumulating form follows the same rules
    assert L.tds_reorder_add(ctypes.c_void_p(a16), ctypes.c_void_p(a16 + 4096), 48, 32, 2, 0, 1, 0,
                             32, None) == _lib.ERR_SHAPE
    assert L.tds_reorder_add(ctypes.c_void_p(a16), ctypes.c_void_p(a16 + 8), 32, 32, 1, 0, 1, 0,
                             32, None) == _lib.ERR_ARG
    assert L.tds_reorder_add(ctypes.c_void_p(a16), ctypes.c_void_p(a16), 32, 32, 1, 1, 1, 0,
                             32, None) == _lib.ERR_ALIAS
