"""ctypes binding of libtds.so (C ABI in include/tds.h): argument marshalling only.

The library must have been built (``paper_2411_13532_gb300.build.build()``); loading fails
loudly otherwise -- there is no CPU fallback.
"""
import ctypes
import os

from . import build as _build

OK, ERR_ARG, ERR_SHAPE, ERR_ALIAS, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM = range(8)
DIRS = {"x": 0, "y": 1, "z": 2}
LAYOUTS = {"cart": 0, "x": 1, "y": 2, "z": 3}
BCS = {"periodic": 0, "closed": 1}
DTYPES = {"f64": 0, "f32": 1}
MODES = {"exact": 0, "paper_drop": 1}
VARIANTS = {"auto": 0, "resident": 1, "streaming": 2, "pipelined": 3, "segmented": 4}
ARITHS = {"native": 0, "split": 1}

# (name, restype, argtypes) of every entry point declared in include/tds.h
_vp, _i, _sz, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
_ip = ctypes.POINTER(ctypes.c_int)
SIGNATURES = [
    ("tds_plan_create", _i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i, _i, _i, _d, _i, _i, _i]),
    ("tds_plan_create_filter", _i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _d, _i, _i, _i, _i, _i]),
    ("tds_plan_create_interp", _i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i, _i, _i, _i, _i]),
    ("tds_plan_create_band", _i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i]),
    ("tds_plan_set_variant", _i, [_vp, _i]),
    ("tds_plan_set_width", _i, [_vp, _i]),
    ("tds_plan_set_arith", _i, [_vp, _i]),
    ("tds_plan_info", _i, [_vp, _ip, _ip, _ip, _ip, _ip]),
    ("tds_plan_width", _i, [_vp, _ip]),
    ("tds_plan_run_chunks", _i, [_vp, _ip]),
    ("tds_workspace_bytes", _i, [_vp, ctypes.POINTER(_sz)]),
    ("tds_deriv", _i, [_vp, _vp, _vp, _vp, _sz, _vp]),
    ("tds_deriv_adjoint", _i, [_vp, _vp, _vp, _vp, _sz, _vp]),
    ("tds_solve", _i, [_vp, _vp, _vp, _vp, _sz, _vp]),
    ("tds_deriv_thomas", _i, [_vp, _vp, _vp, _vp]),
    ("tds_deriv_multi", _i, [_i, ctypes.POINTER(_vp), _ip, _vp, ctypes.POINTER(_vp), _vp, _sz, _vp]),
    ("tds_transport", _i, [_vp, _vp, _vp, _vp, _d, _vp, _vp]),
    ("tds_deriv_host", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    ("tds_deriv_adjoint_host", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    ("tds_reorder", _i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    ("tds_reorder_add", _i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    ("tds_fanout_copy", _i, [_vp, ctypes.POINTER(_vp), _i, _sz, _vp]),
    ("tds_plan_destroy", None, [_vp]),
    ("tds_status_string", ctypes.c_char_p, [_i]),
    ("tds_device_status", _i, []),
    ("tds_selftest_timeout", _i, [_d, _vp]),
    ("tds_plan_reduced_coeffs", _i, [_vp, _vp, _vp]),
    ("tds_reduced_solve", _i, [_vp, _vp, _vp, _vp]),
    ("tds_deriv_noalloc", _i, [_vp, _vp, _vp, _vp]),
]

_lib = None


class TdsError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (what, status_string(status), status))


def lib():
    """The loaded libtds.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libtds.so is missing (%s); build it with "
                               "paper_2411_13532_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(status):
    return lib().tds_status_string(int(status)).decode()


def check(status, what):
    if status != OK:
        raise TdsError(status, what)
