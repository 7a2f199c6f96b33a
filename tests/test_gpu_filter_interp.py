"""GPU parity of the compact filter and mid-point interpolation plans (periodic and closed lines)
against the FP64 oracle.

Every point on small grids over dtype x variant x direction x boundary x P x (operator,
transpose) x CTA width; the segmented variant on long lines; sampled whole lines at 512^3, P = 8;
the fused multi-operator pass with a derivative, the filter and the interpolation.  Bars as for
the derivatives: max|d| / max|ref| <= 1e-12 (FP64), <= 1e-5 (FP32, against the oracle on the
FP32-rounded input)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_13532_gb300 import inputs
from tests.gpu_util import (TOL, TORCH, from_device_layout, gather_lines, rel_errors, report,
                            sample_lines, to_device_layout)

pytestmark = pytest.mark.gpu

tds = pytest.importorskip("paper_2411_13532_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_13532_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert tds.device_status() == 0


AF = 0.45
SMALL = (12, 40, 32)
PS = {"x": [1, 2, 8], "y": [1, 2, 5], "z": [1, 3]}
OPS = [("filter", "periodic"), ("filter", "closed"), ("interp", "periodic"), ("interp", "closed")]


def make_plan(shape, direction, kind, bc, P, dtype, **kw):
    if kind == "filter":
        return tds.Plan(shape, direction, "filter", bc, P=P, dtype=TORCH[dtype], alpha_f=AF, **kw)
    return tds.Plan(shape, direction, "interp", bc, P=P, dtype=TORCH[dtype], **kw)


def reference(cart, direction, kind, bc, adjoint):
    if kind == "filter":
        return oracle.apply_op(cart, direction, oracle.FILTER, bc, AF, adjoint=adjoint)
    return oracle.apply_op(cart, direction, oracle.INTERP, bc, adjoint=adjoint)


def rand_cart(shape, dtype, seed):
    cart = np.random.default_rng(seed).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    return cart


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["resident", "pipelined", "streaming"])
@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_small_grid_every_point(dtype, variant, direction, op, adjoint):
    kind, bc = op
    for i, P in enumerate(PS[direction]):
        cart = rand_cart(SMALL, dtype, seed=31 + i)
        plan = make_plan(SMALL, direction, kind, bc, P, dtype, variant=variant)
        x = to_device_layout(cart, direction, dtype)
        y = plan.adjoint(x) if adjoint else plan.deriv(x)
        torch.cuda.synchronize()
        mx, rms = rel_errors(from_device_layout(y, direction, SMALL), reference(cart, direction, kind, bc, adjoint))
        report("%s %s" % (kind, "T" if adjoint else ""), dtype=dtype, variant=variant, direction=direction,
               bc=bc, P=P, max_rel=mx, rms_rel=rms)
        assert mx <= TOL[dtype], (P, mx, rms)


WSHAPE = (32, 48, 64)
WIDTH_P = {16: {"x": 4, "y": 4, "z": 4}, 8: {"x": 8, "y": 12, "z": 8}}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("width", [16, 8])
@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_resident_width_every_point(dtype, width, direction, op, adjoint):
    kind, bc = op
    P = WIDTH_P[width][direction]
    cart = rand_cart(WSHAPE, dtype, seed=7)
    plan = make_plan(WSHAPE, direction, kind, bc, P, dtype, width=width, variant="resident")
    assert plan.width == width
    x = to_device_layout(cart, direction, dtype)
    y = plan.adjoint(x) if adjoint else plan.deriv(x)
    mx, rms = rel_errors(from_device_layout(y, direction, WSHAPE), reference(cart, direction, kind, bc, adjoint))
    assert mx <= TOL[dtype], (mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("op", OPS)
def test_segmented_long_lines(dtype, op):
    kind, bc = op
    shape = (1, 32, 2048)
    cart = rand_cart(shape, dtype, seed=5)
    for P in (1, 4, 16):
        plan = make_plan(shape, "x", kind, bc, P, dtype, variant="segmented")
        assert plan.variant == "segmented"
        for adjoint in (False, True):
            x = to_device_layout(cart, "x", dtype)
            y = plan.adjoint(x) if adjoint else plan.deriv(x)
            mx, rms = rel_errors(from_device_layout(y, "x", shape), reference(cart, "x", kind, bc, adjoint))
            assert mx <= TOL[dtype], (P, adjoint, mx, rms)


def test_plan_rules():
    with pytest.raises(ValueError):
        tds.Plan(SMALL, "x", "filter", "periodic")         # alpha_f missing
    with pytest.raises(tds.TdsError):
        tds.Plan(SMALL, "x", "filter", "periodic", alpha_f=0.5)
    with pytest.raises(tds.TdsError):
        tds.Plan(SMALL, "x", "filter", "periodic", alpha_f=-0.6)
    # the transport kernel takes derivative plans only
    p1 = tds.Plan(SMALL, "x", "filter", "periodic", P=2, alpha_f=AF)
    p2 = tds.Plan(SMALL, "x", 2, "periodic", P=2)
    u = torch.rand(p1.numel, dtype=torch.float64, device="cuda")
    with pytest.raises(tds.TdsError):
        tds.transport_term(p1, p2, u, u, 0.1)


def test_filter_and_interp_identities_on_device():
    """The filter keeps constants and removes the odd-even mode; the interpolation followed by its
    transpose on a Fourier mode gives the squared symbol (a property of the operators, checked on
    the device output alone)."""
    shape = (4, 32, 64)
    n = 64
    plan_f = tds.Plan(shape, "x", "filter", "periodic", P=4, alpha_f=AF)
    ones = torch.ones(plan_f.numel, dtype=torch.float64, device="cuda")
    assert torch.max(torch.abs(plan_f.deriv(ones) - 1.0)).item() <= 1e-14
    j = np.arange(n)
    cart = np.broadcast_to(((-1.0) ** j)[None, None, :], shape).copy()
    y = plan_f.deriv(to_device_layout(cart, "x", "f64"))
    assert torch.max(torch.abs(y)).item() <= 1e-14


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_closed_interp_last_slot(dtype):
    """Closed lines have n - 1 mid-points: the interpolation writes exactly zero to the last slot
    of every line, and its transpose does not read that slot of its input."""
    shape = (8, 32, 64)
    cart = rand_cart(shape, dtype, seed=19)
    for P in (1, 4):
        plan = make_plan(shape, "x", "interp", "closed", P, dtype)
        x = to_device_layout(cart, "x", dtype)
        y = from_device_layout(plan.deriv(x), "x", shape)
        assert not np.any(y[:, :, -1])
        cart2 = cart.copy()
        cart2[:, :, -1] = 3.0
        a = plan.adjoint(x)
        b = plan.adjoint(to_device_layout(cart2, "x", dtype))
        assert torch.equal(a, b)


FULL = (512, 512, 512)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("direction", ["x", "z"])
def test_full_size_sampled_lines(dtype, direction):
    shape = FULL
    f, _ = inputs.fourier_field(shape, seed=4, kmax=100, noise=0.1, noise_kind="normal", device="cuda")
    fx = tds.reorder(f.to(TORCH[dtype]).reshape(-1), shape, "cart", direction)
    del f
    n = 512
    lines = sample_lines(fx.numel() // n, 32, seed=11)
    src = gather_lines(fx, direction, shape, lines).double().cpu().numpy()
    for kind, bc in OPS:
        plan = make_plan(shape, direction, kind, bc, 8, dtype)
        for adjoint in (False, True):
            y = plan.adjoint(fx) if adjoint else plan.deriv(fx)
            got = gather_lines(y, direction, shape, lines).double().cpu().numpy()
            if kind == "filter":
                ref = (oracle.filter_adjoint_lines if adjoint else oracle.filter_lines)(src, AF, bc)
            else:
                ref = (oracle.interp_adjoint_lines if adjoint else oracle.interp_lines)(src, bc)
            mx, rms = rel_errors(got, ref)
            report("512^3 %s%s %s P=8" % (kind, "T" if adjoint else "", direction), dtype=dtype,
                   variant=plan.variant, width=plan.width, max_rel=mx, rms_rel=rms)
            assert mx <= TOL[dtype], (kind, adjoint, mx, rms)
            del y


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multi_operator_pass_with_filter_and_interp(dtype):
    """D1, the filter and the interpolation of one input in one fused pass: bitwise the single
    calls."""
    shape = (16, 64, 128)
    cart = rand_cart(shape, dtype, seed=3)
    x = to_device_layout(cart, "y", dtype)
    d1 = tds.Plan(shape, "y", 1, "periodic", P=2, dtype=TORCH[dtype])
    fl = make_plan(shape, "y", "filter", "periodic", 2, dtype)
    ip = make_plan(shape, "y", "interp", "periodic", 2, dtype)
    assert d1.variant == fl.variant == ip.variant == "resident" and d1.width == fl.width == ip.width
    outs = tds.deriv_multi([(d1, False), (fl, False), (ip, False), (ip, True)], x)
    singles = [d1.deriv(x), fl.deriv(x), ip.deriv(x), ip.adjoint(x)]
    for a, b in zip(outs, singles):
        assert torch.equal(a, b)
