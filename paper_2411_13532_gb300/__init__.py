"""GB300-native batched compact finite-difference derivatives (DistD2, arXiv 2411.13532).

Python layer over the C ABI of libtds.so (``include/tds.h``): PyTorch supplies device memory
and streams, every step of the computation runs in the library's CUDA kernels.

Shapes are Cartesian ``(nz, ny, nx)`` (a field ``cart[z][y][x]``).  A field handed to a plan
is in the plan direction's interleaved layout (Sec. 4.1), as a contiguous tensor of
nx*ny*nz elements; ``reorder`` converts between layouts.
"""
import ctypes
import math

import torch

from . import _lib
from ._lib import TdsError  # noqa: F401

__all__ = ["Plan", "deriv", "deriv_adjoint", "deriv_multi", "reorder", "reorder_add", "fanout_copy", "transport_term",
           "TransportRHS", "CompactDeriv", "compact_deriv", "device_status", "grid_spacing", "TdsError"]

_TORCH_DTYPES = {torch.float64: "f64", torch.float32: "f32"}


def grid_spacing(n, bc):
    """2*pi/n on periodic lines, 2*pi/(n-1) on closed lines (nodes on both ends)."""
    return 2.0 * math.pi / n if bc == "periodic" else 2.0 * math.pi / (n - 1)


def _stream_ptr(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _check_tensor(t, dtype, numel, what):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise ValueError("%s has dtype %s, expected %s" % (what, t.dtype, dtype))
    if not t.is_contiguous() or t.numel() != numel:
        raise ValueError("%s must be contiguous with %d elements" % (what, numel))


class Plan:
    """One derivative operator: direction, order (1 or 2), boundary condition, P chunks.

    Creation runs the operator preprocessing (Algorithm 4) on the host and uploads it to the
    current (or given) CUDA device.  With ``band=(a, b, c)`` (n values each) the plan is the
    batched tridiagonal solve of that band instead (``tds_plan_create_band``; ``order`` and ``h``
    are ignored and only ``solve`` is available).  ``order="filter"`` (with ``alpha_f``) makes the
    fourth-order compact filter and ``order="interp"`` the sixth-order interpolation to the
    mid-points (closed lines: n - 1 of them, the last slot zero) (``tds_plan_create_filter`` /
    ``tds_plan_create_interp``;
    ``deriv`` applies them, ``adjoint`` their transposes).  ``arith="split"`` (FP64 plans) runs
    the resident sweeps of forward-form operators in float-pair arithmetic
    (``tds_plan_set_arith``).
    """

    def __init__(self, shape, direction, order, bc, P=1, h=None, dtype=torch.float64,
                 mode="exact", variant="auto", width=None, device=None, band=None, alpha_f=None,
                 arith="native"):
        nz, ny, nx = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        kind = {"filter": 3, "interp": 4}.get(order, order)
        self.direction, self.order, self.bc, self.P = direction, int(kind), bc, int(P)
        self.n = {"x": nx, "y": ny, "z": nz}[direction]
        self.h = float(grid_spacing(self.n, bc) if h is None else h)
        self.dtype = dtype
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._handle = None
        L = _lib.lib()
        h_ = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if self.order == 3:
                if alpha_f is None:
                    raise ValueError("a filter plan needs alpha_f")
                self.alpha_f = float(alpha_f)
                _lib.check(L.tds_plan_create_filter(ctypes.byref(h_), nx, ny, nz, _lib.DIRS[direction],
                                                    self.alpha_f, _lib.BCS[bc], self.P,
                                                    _lib.DTYPES[_TORCH_DTYPES[dtype]], 32,
                                                    _lib.MODES[mode]), "tds_plan_create_filter")
            elif self.order == 4:
                _lib.check(L.tds_plan_create_interp(ctypes.byref(h_), nx, ny, nz, _lib.DIRS[direction],
                                                    _lib.BCS[bc], self.P, _lib.DTYPES[_TORCH_DTYPES[dtype]],
                                                    32, _lib.MODES[mode]), "tds_plan_create_interp")
            elif band is None:
                _lib.check(L.tds_plan_create(ctypes.byref(h_), nx, ny, nz, _lib.DIRS[direction],
                                             self.order, _lib.BCS[bc], self.P, self.h,
                                             _lib.DTYPES[_TORCH_DTYPES[dtype]], 32,
                                             _lib.MODES[mode]), "tds_plan_create")
            else:
                arrs = [torch.as_tensor(v, dtype=torch.float64).contiguous().cpu() for v in band]
                if any(a.numel() != self.n for a in arrs):
                    raise ValueError("band arrays must have %d entries each" % self.n)
                self.order = 0
                _lib.check(L.tds_plan_create_band(ctypes.byref(h_), nx, ny, nz, _lib.DIRS[direction],
                                                  *[ctypes.c_void_p(a.data_ptr()) for a in arrs],
                                                  _lib.BCS[bc], self.P, _lib.DTYPES[_TORCH_DTYPES[dtype]],
                                                  32, _lib.MODES[mode]), "tds_plan_create_band")
        self._handle = h_
        if arith != "native":   # first: it re-picks the width and the AUTO variant
            _lib.check(L.tds_plan_set_arith(h_, _lib.ARITHS[arith]), "tds_plan_set_arith")
        self.arith = arith
        if width is not None:
            _lib.check(L.tds_plan_set_width(h_, int(width)), "tds_plan_set_width")
        if variant != "auto":
            _lib.check(L.tds_plan_set_variant(h_, _lib.VARIANTS[variant]), "tds_plan_set_variant")
        nbytes = ctypes.c_size_t()
        _lib.check(L.tds_workspace_bytes(h_, ctypes.byref(nbytes)), "tds_workspace_bytes")
        self.ws_bytes = nbytes.value
        n_, nl, p_, var, smem = (ctypes.c_int() for _ in range(5))
        _lib.check(L.tds_plan_info(h_, ctypes.byref(n_), ctypes.byref(nl), ctypes.byref(p_),
                                   ctypes.byref(var), ctypes.byref(smem)), "tds_plan_info")
        self.nlines = nl.value
        self.variant = {1: "resident", 2: "streaming", 3: "pipelined", 4: "segmented"}[var.value]
        self.smem_bytes = smem.value
        w_ = ctypes.c_int()
        _lib.check(L.tds_plan_width(h_, ctypes.byref(w_)), "tds_plan_width")
        self.width = w_.value   # lines per resident CTA (0: cannot run resident)
        _lib.check(L.tds_plan_run_chunks(h_, ctypes.byref(w_)), "tds_plan_run_chunks")
        self.run_chunks = w_.value   # chunks per line the kernels run with (P, or finer under AUTO)
        self.numel = nx * ny * nz

    def __del__(self):
        if getattr(self, "_handle", None) is not None and _lib._lib is not None:
            _lib._lib.tds_plan_destroy(self._handle)
            self._handle = None

    def workspace(self):
        """A fresh workspace tensor for this plan (None if it needs none)."""
        if not self.ws_bytes:
            return None
        return torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def _run(self, fn, x, out, ws, stream, what):
        _check_tensor(x, self.dtype, self.numel, "input")
        if out is None:
            out = torch.empty_like(x)
        _check_tensor(out, self.dtype, self.numel, "out")
        if ws is None:
            ws = self.workspace()
        wp = ctypes.c_void_p(ws.data_ptr()) if ws is not None else None
        wb = ws.numel() if ws is not None else 0
        with torch.cuda.device(self.device):
            _lib.check(fn(self._handle, ctypes.c_void_p(x.data_ptr()),
                          ctypes.c_void_p(out.data_ptr()), wp, wb,
                          _stream_ptr(stream, self.device)), what)
        return out

    def deriv(self, x, out=None, ws=None, stream=None):
        """out = A^{-1} B x (x and out in this plan's direction layout)."""
        return self._run(_lib.lib().tds_deriv, x, out, ws, stream, "tds_deriv")

    def adjoint(self, g, out=None, ws=None, stream=None):
        """out = B^T A^{-T} g, the transpose of ``deriv``."""
        return self._run(_lib.lib().tds_deriv_adjoint, g, out, ws, stream, "tds_deriv_adjoint")

    def _run_host(self, fn, host_in, host_out, d_in, d_out, ws, stream, what):
        for t, nm in ((host_in, "host_in"), (host_out, "host_out")):
            if t is None and nm == "host_in":
                continue
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.numel:
                raise ValueError("%s must be a contiguous host tensor of %d %s" % (nm, self.numel, self.dtype))
        _check_tensor(d_in, self.dtype, self.numel, "d_in")
        _check_tensor(d_out, self.dtype, self.numel, "d_out")
        if ws is None:
            ws = self.workspace()
        wp = ctypes.c_void_p(ws.data_ptr()) if ws is not None else None
        wb = ws.numel() if ws is not None else 0
        hin = ctypes.c_void_p(host_in.data_ptr()) if host_in is not None else None
        with torch.cuda.device(self.device):
            _lib.check(fn(self._handle, hin, ctypes.c_void_p(host_out.data_ptr()),
                          ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), wp, wb,
                          _stream_ptr(stream, self.device)), what)
        return host_out

    def solve(self, d, out=None, ws=None, stream=None):
        """x = A^{-1} d: the tridiagonal solve of this plan's compact scheme alone (``tds_solve``)."""
        return self._run(_lib.lib().tds_solve, d, out, ws, stream, "tds_solve")

    def thomas(self, x, out=None, stream=None):
        """``tds_deriv_thomas``: this plan's operator by the plain Thomas algorithm on whole lines
        (cyclic lines: Sherman-Morrison), the single-rank baseline of the DistD2 kernels."""
        _check_tensor(x, self.dtype, self.numel, "input")
        if out is None:
            out = torch.empty_like(x)
        _check_tensor(out, self.dtype, self.numel, "out")
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().tds_deriv_thomas(self._handle, ctypes.c_void_p(x.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()),
                                                   _stream_ptr(stream, self.device)),
                       "tds_deriv_thomas")
        return out

    def deriv_host(self, host_in, host_out, d_in, d_out, ws=None, stream=None):
        """``tds_deriv_host``: host_in (a host tensor, or None when d_in already holds the input)
        through d_in / d_out to host_out, copies pipelined with the compute inside the call."""
        return self._run_host(_lib.lib().tds_deriv_host, host_in, host_out, d_in, d_out, ws, stream,
                              "tds_deriv_host")

    def adjoint_host(self, host_g, host_out, d_in, d_out, ws=None, stream=None):
        """``tds_deriv_adjoint_host``: the adjoint with host buffers (see ``deriv_host``)."""
        return self._run_host(_lib.lib().tds_deriv_adjoint_host, host_g, host_out, d_in, d_out, ws,
                              stream, "tds_deriv_adjoint_host")

    def deriv_noalloc(self, x, out, stream=None):
        """``tds_deriv_noalloc``: like ``deriv`` but with the library's built-in scratch instead
        of a caller workspace (for callers that cannot allocate; ``out`` must be given)."""
        _check_tensor(x, self.dtype, self.numel, "input")
        _check_tensor(out, self.dtype, self.numel, "out")
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().tds_deriv_noalloc(self._handle, ctypes.c_void_p(x.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    _stream_ptr(stream, self.device)),
                       "tds_deriv_noalloc")
        return out

    def reduced_coeffs(self):
        """(sub, sup) of the reduced chunk-end system, 2P doubles each."""
        R = 2 * self.P
        sub = (ctypes.c_double * R)()
        sup = (ctypes.c_double * R)()
        _lib.check(_lib.lib().tds_plan_reduced_coeffs(self._handle, sub, sup),
                   "tds_plan_reduced_coeffs")
        return list(sub), list(sup)

    def reduced_solve(self, rhs, out=None, stream=None):
        """Solve the reduced system for every line: rhs is (N, 2P) float64 on the device."""
        numel = self.nlines * 2 * self.P
        _check_tensor(rhs, torch.float64, numel, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().tds_reduced_solve(
                self._handle, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                _stream_ptr(stream, self.device)), "tds_reduced_solve")
        return out


_PLANS = {}


def _plan(shape, direction, order, bc, P, h, dtype, mode, device):
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (tuple(shape), direction, order, bc, P, h, dtype, mode, dev)
    p = _PLANS.get(key)
    if p is None:
        p = _PLANS[key] = Plan(shape, direction, order, bc, P, h, dtype, mode, device=dev)
    return p


def deriv_multi(ops, x, outs=None, ws=None, stream=None):
    """Several operators of one input through ``tds_deriv_multi``: ``ops`` is a list of
    ``(plan, adjoint)`` pairs (up to 4) over the same field; returns the list of results.
    Resident plans of one geometry with forward-form operators run as one fused pass."""
    if not 1 <= len(ops) <= 4:
        raise ValueError("deriv_multi takes 1 to 4 operators")
    plans = [p for p, _ in ops]
    p0 = plans[0]
    _check_tensor(x, p0.dtype, p0.numel, "input")
    if outs is None:
        outs = [torch.empty_like(x) for _ in ops]
    for o in outs:
        _check_tensor(o, p0.dtype, p0.numel, "out")
    if ws is None:
        need = max(p.ws_bytes for p in plans)
        ws = torch.empty(need, dtype=torch.uint8, device=x.device) if need else None
    n = len(ops)
    hp = (ctypes.c_void_p * n)(*[p._handle.value for p in plans])
    ad = (ctypes.c_int * n)(*[1 if a else 0 for _, a in ops])
    op_ = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    wp = ctypes.c_void_p(ws.data_ptr()) if ws is not None else None
    wb = ws.numel() if ws is not None else 0
    with torch.cuda.device(p0.device):
        _lib.check(_lib.lib().tds_deriv_multi(n, hp, ad, ctypes.c_void_p(x.data_ptr()), op_, wp, wb,
                                              _stream_ptr(stream, p0.device)), "tds_deriv_multi")
    return outs


def deriv(field, shape, direction, order, bc, P=1, h=None, mode="exact", out=None):
    """Derivative of ``field`` (in ``direction``'s layout) along ``direction``."""
    return _plan(shape, direction, order, bc, P, h, field.dtype, mode, field.device).deriv(field, out)


def deriv_adjoint(g, shape, direction, order, bc, P=1, h=None, mode="exact", out=None):
    """Transpose of ``deriv`` applied to ``g``."""
    return _plan(shape, direction, order, bc, P, h, g.dtype, mode, g.device).adjoint(g, out)


def reorder(x, shape, src, dst, out=None, stream=None):
    """Permute a field between layouts 'cart', 'x', 'y', 'z' (bit-exact)."""
    nz, ny, nx = (int(v) for v in shape)
    if x.dtype not in _TORCH_DTYPES:
        raise ValueError("reorder supports float64 and float32")
    _check_tensor(x, x.dtype, nx * ny * nz, "input")
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, x.dtype, nx * ny * nz, "out")
    with torch.cuda.device(x.device):
        _lib.check(_lib.lib().tds_reorder(
            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), nx, ny, nz,
            _lib.LAYOUTS[src], _lib.LAYOUTS[dst], _lib.DTYPES[_TORCH_DTYPES[x.dtype]], 32,
            _stream_ptr(stream, x.device)), "tds_reorder")
    return out


def reorder_add(x, shape, src, dst, out, stream=None):
    """out += x permuted from layout ``src`` to ``dst`` (one pass; bit-exact against a reorder
    followed by an add)."""
    nz, ny, nx = (int(v) for v in shape)
    if x.dtype not in _TORCH_DTYPES:
        raise ValueError("reorder_add supports float64 and float32")
    _check_tensor(x, x.dtype, nx * ny * nz, "input")
    _check_tensor(out, x.dtype, nx * ny * nz, "out")
    with torch.cuda.device(x.device):
        _lib.check(_lib.lib().tds_reorder_add(
            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), nx, ny, nz,
            _lib.LAYOUTS[src], _lib.LAYOUTS[dst], _lib.DTYPES[_TORCH_DTYPES[x.dtype]], 32,
            _stream_ptr(stream, x.device)), "tds_reorder_add")
    return out


def fanout_copy(x, outs, stream=None):
    """Copy ``x`` into each tensor of ``outs`` (1 to 4) reading it once (``tds_fanout_copy``):
    the traffic of the fused multi-operator pass, as a measured ceiling for it."""
    if not 1 <= len(outs) <= 4:
        raise ValueError("fanout_copy takes 1 to 4 outputs")
    for o in outs:
        if o.dtype != x.dtype or o.numel() != x.numel() or not o.is_contiguous():
            raise ValueError("outputs must match the input")
    n = len(outs)
    op_ = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    with torch.cuda.device(x.device):
        _lib.check(_lib.lib().tds_fanout_copy(ctypes.c_void_p(x.data_ptr()), op_, n,
                                              x.numel() * x.element_size(), _stream_ptr(stream, x.device)),
                   "tds_fanout_copy")
    return outs


def transport_term(d1, d2, ui, uj, nu, out=None, stream=None):
    """out = -1/2 (uj * D1 ui + D1 (uj ui)) + nu * D2 ui along the plans' direction, one fused
    kernel (``tds_transport``); d1 / d2 are order-1 / order-2 plans of one geometry, the fields
    are in their direction layout (``ui`` may be ``uj``)."""
    _check_tensor(ui, d1.dtype, d1.numel, "ui")
    _check_tensor(uj, d1.dtype, d1.numel, "uj")
    if out is None:
        out = torch.empty_like(ui)
    _check_tensor(out, d1.dtype, d1.numel, "out")
    with torch.cuda.device(d1.device):
        _lib.check(_lib.lib().tds_transport(d1._handle, d2._handle, ctypes.c_void_p(ui.data_ptr()),
                                            ctypes.c_void_p(uj.data_ptr()), float(nu),
                                            ctypes.c_void_p(out.data_ptr()),
                                            _stream_ptr(stream, d1.device)), "tds_transport")
    return out


class TransportRHS:
    """Right-hand side of the skew-symmetric momentum transport equation (Sec. 5, Eq. mom-comps)
    on a periodic (or closed) box, every field in the x-direction layout:

        rhs_i = sum_j [ -1/2 (u_j du_i/dx_j + d(u_j u_i)/dx_j) + nu d2u_i/dx_j2 ]

    One call runs the nine term groups as fused kernels (``transport_term``), reorders the three
    velocity components x -> y -> z once each (six reorders), and accumulates each y and z result
    into the x-layout output with ``reorder_add`` (six accumulations): 21 launches.  ``P`` is
    the chunk count per line (an int, or one per direction x, y, z); ``width`` optionally fixes
    the lines per resident CTA.  The plans must be able to hold their lines in a CTA.
    ``arith="split"`` (FP64) runs the term groups' sweeps in float-pair arithmetic
    (``tds_plan_set_arith``).  Six temporary fields are allocated with the object.
    """

    DIRS = ("x", "y", "z")

    def __init__(self, shape, P=1, bc="periodic", dtype=torch.float64, width=None, device=None,
                 arith="native"):
        self.shape = tuple(int(v) for v in shape)
        Ps = (P, P, P) if isinstance(P, int) else tuple(int(p) for p in P)
        self.d1, self.d2 = {}, {}
        for d, p in zip(self.DIRS, Ps):
            self.d1[d] = Plan(self.shape, d, 1, bc, P=p, dtype=dtype, width=width, device=device, arith=arith)
            self.d2[d] = Plan(self.shape, d, 2, bc, P=p, dtype=dtype, width=width, device=device, arith=arith)
            for pl in (self.d1[d], self.d2[d]):
                if not pl.width:
                    raise ValueError("the %s lines do not fit a resident CTA" % d)
        self.dtype, self.device = dtype, self.d1["x"].device
        numel = self.d1["x"].numel
        self._a = [torch.empty(numel, dtype=dtype, device=self.device) for _ in range(3)]
        self._b = [torch.empty(numel, dtype=dtype, device=self.device) for _ in range(3)]

    def launch_list(self, u, nu, out, stream=None):
        """The 21 launches of one evaluation, in order, as (label, callable) pairs."""
        if len(u) != 3 or len(out) != 3:
            raise ValueError("u and out hold the three velocity components")
        a, b, sh, d1, d2 = self._a, self._b, self.shape, self.d1, self.d2
        L = []
        # x: the terms land in the output directly
        for i in range(3):
            L.append(("term/x", lambda i=i: transport_term(d1["x"], d2["x"], u[i], u[0], nu, out[i], stream)))
        # y: reorder the components, the terms into b, accumulate into the output
        for i in range(3):
            L.append(("reorder/x-y", lambda i=i: reorder(u[i], sh, "x", "y", a[i], stream)))
        for i in range(3):
            L.append(("term/y", lambda i=i: transport_term(d1["y"], d2["y"], a[i], a[1], nu, b[i], stream)))
            L.append(("reorder_add/y-x", lambda i=i: reorder_add(b[i], sh, "y", "x", out[i], stream)))
        # z: the components from their y copies (a row permutation) into b, the terms into a
        for i in range(3):
            L.append(("reorder/y-z", lambda i=i: reorder(a[i], sh, "y", "z", b[i], stream)))
        for i in range(3):
            L.append(("term/z", lambda i=i: transport_term(d1["z"], d2["z"], b[i], b[2], nu, a[i], stream)))
            L.append(("reorder_add/z-x", lambda i=i: reorder_add(a[i], sh, "z", "x", out[i], stream)))
        return L

    def __call__(self, u, nu, out=None, stream=None):
        if out is None:
            out = [torch.empty_like(u[0]) for _ in range(3)]
        for _, fn in self.launch_list(u, nu, out, stream):
            fn()
        return out

    def graph(self, u, nu, out):
        """One evaluation captured as a CUDA graph on the fixed device buffers ``u`` / ``out``
        (x layout): ``g.replay()`` reruns the 21 launches with a single submission.  The buffers
        must stay alive, and keep their addresses, for as long as the graph is replayed."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self(u, nu, out, stream=side)          # warm-up outside the capture (kernel attributes)
        torch.cuda.current_stream(self.device).wait_stream(side)
        with torch.cuda.graph(g):
            self(u, nu, out)
        return g

    def call_host(self, host_u, host_out, nu, u, out, stream=None):
        """One evaluation from pinned host memory to pinned host memory, the copies overlapped
        with the kernels: component i is copied in on an input stream and its x term group starts
        as soon as it has landed (i = 0, 1, 2 in turn); each result is copied out on an output
        stream as soon as its last accumulation (the z group) is done.  ``u`` / ``out`` are the
        device buffers (x layout).  Ordered on ``stream`` (default: the current stream): the call
        returns at once, and the host results are complete once that stream has reached the end
        of the call."""
        if len(host_u) != 3 or len(host_out) != 3 or len(u) != 3 or len(out) != 3:
            raise ValueError("three velocity components in and three results out")
        for h in list(host_u) + list(host_out):
            if h.is_cuda or not h.is_pinned() or h.dtype != self.dtype or h.numel() != self.d1["x"].numel:
                raise ValueError("host buffers must be pinned CPU tensors of the field's dtype and size")
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        if not hasattr(self, "_copy_in"):
            self._copy_in = torch.cuda.Stream(self.device)
            self._copy_out = torch.cuda.Stream(self.device)
        cin, cout = self._copy_in, self._copy_out
        start = torch.cuda.Event()
        start.record(st)
        landed = []
        with torch.cuda.stream(cin):
            cin.wait_event(start)              # the device inputs are free to overwrite
            for h, d in zip(host_u, u):
                d.copy_(h, non_blocking=True)
                d.record_stream(cin)
                e = torch.cuda.Event()
                e.record(cin)
                landed.append(e)
        steps = self.launch_list(u, nu, out, st)
        done = 0
        for idx, (label, fn) in enumerate(steps):
            if label == "term/x":              # x group i needs components i and 0
                st.wait_event(landed[idx])
            fn()
            if label == "reorder_add/z-x":     # result `done` is final
                e = torch.cuda.Event()
                e.record(st)
                with torch.cuda.stream(cout):
                    cout.wait_event(e)
                    host_out[done].copy_(out[done], non_blocking=True)
                    out[done].record_stream(cout)
                done += 1
        fin = torch.cuda.Event()
        fin.record(cout)
        st.wait_event(fin)                     # the call is ordered on `stream`
        return host_out


def device_status():
    """Read and clear the device-side status word (0 = no bounded wait gave up)."""
    return _lib.lib().tds_device_status()


class CompactDeriv(torch.autograd.Function):
    """y = D x with D = A^{-1} B; the backward pass applies D^T = B^T A^{-T} with the
    library's adjoint kernels."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.deriv(x.contiguous())

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.adjoint(grad.contiguous()), None


def compact_deriv(x, plan):
    return CompactDeriv.apply(x, plan)
