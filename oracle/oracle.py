"""Python side of the FP64 oracle (ctypes wrapper over ``tds_oracle.c`` + layouts).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Layouts (the interleaved group data structure of Sec. 4.1): for a Cartesian field
``cart[z][y][x]`` and a derivative direction, each line of n points along that direction
gets a line number l; lines are packed in groups of SZ so that element (s, j, g) sits at
flat offset ``s + SZ*(j + n*g)`` with ``l = g*SZ + s`` (shape (SZ, n, N_lines/SZ) in the
column-major notation of Sec. 4.1).  Line numbering used throughout:
    x lines: l = y + ny*z      (n = nx)
    y lines: l = x + nx*z      (n = ny)
    z lines: l = x + nx*y      (n = nz)
These maps are written here with numpy transposes/reshapes, independently of any GPU
reorder code.  Parity "unpinned": none -- every function here is pinned by tests in
``tests/test_oracle_pins.py`` (dense LU brute force, closed-form modified wavenumbers,
polynomial exactness, adjoint identities, a hand-enumerated layout example).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tds_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libtds_oracle.so")
_lib = None

DIRS = {"x": 0, "y": 1, "z": 2}


def build(force=False):
    """Compile the oracle's C file into a shared library (gcc, FP contraction off)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.tdso_bands.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   dp, dp, dp, dp]
        for name in ("tdso_deriv_lines", "tdso_deriv_adjoint_lines", "tdso_rhs_lines"):
            getattr(lib, name).argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, dp, dp]
        lib.tdso_tridiag_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
        _lib = lib
    return _lib


def _ptr(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def grid_spacing(n, bc):
    """h for a line of n nodes on [0, 2*pi]: 2*pi/n periodic, 2*pi/(n-1) closed (both
    end nodes on the boundary)."""
    return 2.0 * np.pi / n if bc == "periodic" else 2.0 * np.pi / (n - 1)


def bands(n, order, bc, h):
    """Return (a, b, c, B7): the tridiagonal band of A and the 7-tap rows of B."""
    a = np.empty(n); b = np.empty(n); c = np.empty(n); B7 = np.empty((n, 7))
    _check(_load().tdso_bands(n, order, int(bc == "periodic"), h, _ptr(a), _ptr(b), _ptr(c),
                              _ptr(B7)), "bands")
    return a, b, c, B7


def _lines_call(fn, lines, order, bc, h):
    lines = np.ascontiguousarray(lines, dtype=np.float64)
    nl, n = lines.shape
    out = np.empty_like(lines)
    _check(fn(n, nl, order, int(bc == "periodic"), h, _ptr(lines), _ptr(out)), fn.__name__)
    return out


def rhs_lines(lines, order, bc, h):
    """d = B f for every row of ``lines`` (shape (N_lines, n))."""
    return _lines_call(_load().tdso_rhs_lines, lines, order, bc, h)


def deriv_lines(lines, order, bc, h):
    """D f = A^{-1} B f for every row of ``lines``."""
    return _lines_call(_load().tdso_deriv_lines, lines, order, bc, h)


def deriv_adjoint_lines(lines, order, bc, h):
    """D^T g = B^T A^{-T} g for every row of ``lines``."""
    return _lines_call(_load().tdso_deriv_adjoint_lines, lines, order, bc, h)


def tridiag_solve(a, b, c, d, periodic):
    """Solve one (cyclic if periodic) tridiagonal system with the oracle's solver."""
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    x = np.empty_like(d)
    _check(_load().tdso_tridiag_solve(len(d), int(bool(periodic)), _ptr(a), _ptr(b), _ptr(c),
                                      _ptr(d), _ptr(x)), "tridiag_solve")
    return x


def lines_view(cart, direction):
    """(N_lines, n) array of the lines of ``cart[z][y][x]`` along ``direction``,
    in the line numbering of the module docstring."""
    nz, ny, nx = cart.shape
    if direction == "x":
        return cart.reshape(nz * ny, nx)
    if direction == "y":
        return cart.transpose(0, 2, 1).reshape(nz * nx, ny)
    if direction == "z":
        return cart.transpose(1, 2, 0).reshape(ny * nx, nz)
    raise ValueError(direction)


def from_lines_view(lines, direction, shape):
    """Inverse of ``lines_view``: back to a Cartesian (nz, ny, nx) array."""
    nz, ny, nx = shape
    if direction == "x":
        return lines.reshape(nz, ny, nx)
    if direction == "y":
        return lines.reshape(nz, nx, ny).transpose(0, 2, 1)
    if direction == "z":
        return lines.reshape(ny, nx, nz).transpose(2, 0, 1)
    raise ValueError(direction)


def layout_lines_count(shape, direction):
    nz, ny, nx = shape
    return {"x": ny * nz, "y": nx * nz, "z": nx * ny}[direction]


def to_layout(cart, direction, sz):
    """Flat array of the SZ-interleaved direction layout: offset s + SZ*(j + n*g)."""
    L = lines_view(np.asarray(cart), direction)
    nl, n = L.shape
    if nl % sz:
        raise ValueError("number of lines %d is not a multiple of SZ=%d" % (nl, sz))
    return np.ascontiguousarray(L.reshape(nl // sz, sz, n).transpose(0, 2, 1)).reshape(-1)


def from_layout(flat, direction, shape, sz):
    """Inverse of ``to_layout``."""
    nz, ny, nx = shape
    n = {"x": nx, "y": ny, "z": nz}[direction]
    nl = layout_lines_count(shape, direction)
    L = np.asarray(flat).reshape(nl // sz, n, sz).transpose(0, 2, 1).reshape(nl, n)
    return np.ascontiguousarray(from_lines_view(L, direction, shape))


def deriv(cart, direction, order, bc, h=None):
    """Derivative of a Cartesian field along one direction (Cartesian in and out)."""
    cart = np.ascontiguousarray(cart, dtype=np.float64)
    n = {"x": cart.shape[2], "y": cart.shape[1], "z": cart.shape[0]}[direction]
    h = grid_spacing(n, bc) if h is None else h
    out = deriv_lines(lines_view(cart, direction), order, bc, h)
    return np.ascontiguousarray(from_lines_view(out, direction, cart.shape))


def deriv_adjoint(cart, direction, order, bc, h=None):
    """Adjoint (transpose) of ``deriv`` applied to a Cartesian field."""
    cart = np.ascontiguousarray(cart, dtype=np.float64)
    n = {"x": cart.shape[2], "y": cart.shape[1], "z": cart.shape[0]}[direction]
    h = grid_spacing(n, bc) if h is None else h
    out = deriv_adjoint_lines(lines_view(cart, direction), order, bc, h)
    return np.ascontiguousarray(from_lines_view(out, direction, cart.shape))


def transport_term_lines(ui, uj, nu, bc, h):
    """One term group of the skew-symmetric momentum transport equation (Sec. 5, Eq. mom-comps)
    on lines (L, n) along the derivative direction j:
        -1/2 (u_j du_i/dx_j + d(u_j u_i)/dx_j) + nu d2u_i/dx_j2,
    each derivative the compact scheme of ``deriv_lines`` (first: Eq. cfds; second: its order-2
    counterpart), the products pointwise, all in FP64."""
    ui = np.ascontiguousarray(ui, dtype=np.float64)
    uj = np.ascontiguousarray(uj, dtype=np.float64)
    conv = uj * deriv_lines(ui, 1, bc, h)
    cons = deriv_lines(uj * ui, 1, bc, h)
    visc = deriv_lines(ui, 2, bc, h)
    return -0.5 * (conv + cons) + nu * visc


def transport_term(ui, uj, direction, nu, bc, h=None):
    """``transport_term_lines`` along one direction of Cartesian fields (Cartesian in and out)."""
    ui = np.ascontiguousarray(ui, dtype=np.float64)
    uj = np.ascontiguousarray(uj, dtype=np.float64)
    n = {"x": ui.shape[2], "y": ui.shape[1], "z": ui.shape[0]}[direction]
    h = grid_spacing(n, bc) if h is None else h
    out = transport_term_lines(lines_view(ui, direction), lines_view(uj, direction), nu, bc, h)
    return np.ascontiguousarray(from_lines_view(out, direction, ui.shape))


def transport_rhs(u, nu, bc, h=None):
    """Eq. mom-comps: the right-hand sides of the three momentum components, u = (u_x, u_y, u_z)
    Cartesian; component i sums the term groups of the three directions j."""
    dirs = ("x", "y", "z")
    return [sum(transport_term(u[i], u[j], dirs[j], nu, bc, h) for j in range(3)) for i in range(3)]


FILTER, INTERP = 3, 4   # operator codes of the oracle's band builder (see tds_oracle.c)


def filter_lines(lines, alpha_f, bc):
    """The fourth-order tridiagonal compact filter (Lele 1992, App. C.2) of every line."""
    return _lines_call(_load().tdso_deriv_lines, lines, FILTER, bc, alpha_f)


def filter_adjoint_lines(lines, alpha_f, bc):
    """Transpose of ``filter_lines``."""
    return _lines_call(_load().tdso_deriv_adjoint_lines, lines, FILTER, bc, alpha_f)


def interp_lines(lines, bc="periodic"):
    """Sixth-order compact interpolation from the nodes to the mid-points x_i + h/2 (Lele 1992,
    App. C.1); closed lines give n - 1 mid-points and a zero in the last slot."""
    return _lines_call(_load().tdso_deriv_lines, lines, INTERP, bc, 1.0)


def interp_adjoint_lines(lines, bc="periodic"):
    """Transpose of ``interp_lines``: the interpolation from the mid-points back to the nodes
    (closed lines: the last slot of the input is not used)."""
    return _lines_call(_load().tdso_deriv_adjoint_lines, lines, INTERP, bc, 1.0)


def apply_op(cart, direction, op, bc, param=None, adjoint=False):
    """One of the line operators along a direction of a Cartesian field: op 1 / 2 (derivatives,
    param = h or None for the default spacing), 3 (filter, param = alpha_f) or 4 (mid-point
    interpolation)."""
    cart = np.ascontiguousarray(cart, dtype=np.float64)
    n = {"x": cart.shape[2], "y": cart.shape[1], "z": cart.shape[0]}[direction]
    if op in (1, 2) and param is None:
        param = grid_spacing(n, bc)
    if op == INTERP:
        param = 1.0
    fn = _load().tdso_deriv_adjoint_lines if adjoint else _load().tdso_deriv_lines
    out = _lines_call(fn, lines_view(cart, direction), op, bc, param)
    return np.ascontiguousarray(from_lines_view(out, direction, cart.shape))

