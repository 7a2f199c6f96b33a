"""GPU parity of the plain Thomas kernel (``tds_deriv_thomas``: Algorithm 1 on whole lines, cyclic
lines by Sherman-Morrison) against the FP64 oracle: every point on small grids over dtype x
direction x boundary x operator, sampled whole lines at 512^3, argument rules.  Bars as for the
DistD2 kernels: max|d| / max|ref| <= 1e-12 (FP64), <= 1e-5 (FP32, against the oracle on the
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


SMALL = (12, 40, 32)
AF = 0.45
OPS = [(1, "periodic"), (1, "closed"), (2, "periodic"), (2, "closed"),
       ("filter", "periodic"), ("filter", "closed"), ("interp", "periodic"), ("interp", "closed")]


def make_plan(shape, direction, op, bc, dtype, P=1):
    if op == "filter":
        return tds.Plan(shape, direction, "filter", bc, P=P, dtype=TORCH[dtype], alpha_f=AF)
    if op == "interp":
        return tds.Plan(shape, direction, "interp", bc, P=P, dtype=TORCH[dtype])
    n = {"x": shape[2], "y": shape[1], "z": shape[0]}[direction]
    return tds.Plan(shape, direction, op, bc, P=P, h=oracle.grid_spacing(n, bc), dtype=TORCH[dtype])


def reference(cart, direction, op, bc):
    if op == "filter":
        return oracle.apply_op(cart, direction, oracle.FILTER, bc, AF)
    if op == "interp":
        return oracle.apply_op(cart, direction, oracle.INTERP, bc)
    return oracle.deriv(cart, direction, op, bc)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("op", OPS, ids=["%s-%s" % o for o in OPS])
def test_small_grid_every_point(dtype, direction, op):
    kind, bc = op
    cart = np.random.default_rng(17).uniform(-1, 1, SMALL)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    for P in (1, 2):   # the plan's chunking is ignored
        plan = make_plan(SMALL, direction, kind, bc, dtype, P=P)
        x = to_device_layout(cart, direction, dtype)
        y = plan.thomas(x)
        mx, rms = rel_errors(from_device_layout(y, direction, SMALL), reference(cart, direction, kind, bc))
        report("thomas %s" % (kind,), dtype=dtype, direction=direction, bc=bc, P=P, max_rel=mx, rms_rel=rms)
        assert mx <= TOL[dtype], (P, mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_long_and_short_lines(dtype, bc):
    """n = 8 (the smallest line: on closed lines the FP64 end rows of FP32 second derivatives
    meet), 9 and 12 (one and four rows between them) and 2048, both orders."""
    for shape in ((2, 32, 8), (2, 32, 9), (2, 32, 12), (1, 32, 2048)):
        cart = np.random.default_rng(3).uniform(-1, 1, shape)
        if dtype == "f32":
            cart = cart.astype(np.float32).astype(np.float64)
        for order in (1, 2):
            plan = make_plan(shape, "x", order, bc, dtype)
            y = plan.thomas(to_device_layout(cart, "x", dtype))
            mx, rms = rel_errors(from_device_layout(y, "x", shape), reference(cart, "x", order, bc))
            assert mx <= TOL[dtype], (shape, order, mx, rms)


def test_argument_rules():
    x = torch.rand(SMALL[0] * SMALL[1] * SMALL[2], dtype=torch.float64, device="cuda")
    n = SMALL[2]
    a = np.full(n, 0.25); b = np.ones(n); c = np.full(n, 0.25)
    band = tds.Plan(SMALL, "x", 0, "periodic", band=(a, b, c))
    with pytest.raises(tds.TdsError):
        band.thomas(x)
    p = make_plan(SMALL, "x", 1, "periodic", "f64")
    with pytest.raises(tds.TdsError):
        p.thomas(x, out=x)                       # in and out overlap
    with pytest.raises(ValueError):
        p.thomas(x.float())                      # dtype of the plan


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_full_size_sampled_lines(dtype, bc):
    shape = (512, 512, 512)
    f, _ = inputs.fourier_field(shape, seed=4, kmax=100, noise=0.1, noise_kind="normal", device="cuda")
    fx = tds.reorder(f.to(TORCH[dtype]).reshape(-1), shape, "cart", "x")
    del f
    lines = sample_lines(fx.numel() // 512, 32, seed=12)
    src = gather_lines(fx, "x", shape, lines).double().cpu().numpy()
    h = oracle.grid_spacing(512, bc)
    for order in (1, 2):
        plan = make_plan(shape, "x", order, bc, dtype)
        y = plan.thomas(fx)
        got = gather_lines(y, "x", shape, lines).double().cpu().numpy()
        mx, rms = rel_errors(got, oracle.deriv_lines(src, order, bc, h))
        report("512^3 thomas D%d x %s" % (order, bc), dtype=dtype, max_rel=mx, rms_rel=rms)
        assert mx <= TOL[dtype], (order, mx, rms)
        del y


@pytest.mark.parametrize("direction", ["x", "z"])
@pytest.mark.parametrize("order", [1, 2])
def test_fp32_closed_smooth_every_point(order, direction):
    """FP32 on closed lines of a smooth field (Fourier modes, kmax 20).  The second derivative's
    closure f''_0 + 11 f''_1 = ... magnifies an FP32 rounding at row 1 or n-2 about 100-fold at
    the end row, so FP32 plans with such a closure run the four rows at each end of the line in
    FP64; the closure and interior taps of the FP32 rows act on differences of nearby values.
    Every point of 512-point lines against the oracle on the FP32-rounded field."""
    shape = (512, 32, 32) if direction == "z" else (4, 32, 512)
    f, _ = inputs.fourier_field(shape, seed=9, kmax=20, noise=1e-3)
    cart = f.numpy().astype(np.float32).astype(np.float64)
    plan = make_plan(shape, direction, order, "closed", "f32")
    y = plan.thomas(to_device_layout(cart, direction, "f32"))
    mx, rms = rel_errors(from_device_layout(y, direction, shape), reference(cart, direction, order, "closed"))
    report("thomas smooth D%d %s closed" % (order, direction), dtype="f32", max_rel=mx, rms_rel=rms)
    assert mx <= TOL["f32"], (mx, rms)


@pytest.mark.parametrize("direction", ["x", "z"])
@pytest.mark.parametrize("order", [1, 2])
def test_fp32_closed_smooth_512_sampled_lines(order, direction):
    """The same at 512^3: sampled whole lines (both ends included) of a smooth field, FP32,
    closed, against the oracle on the FP32-rounded lines."""
    shape = (512, 512, 512)
    f, _ = inputs.fourier_field(shape, seed=6, kmax=20, noise=1e-3, device="cuda")
    fd = tds.reorder(f.to(torch.float32).reshape(-1), shape, "cart", direction)
    del f
    lines = sample_lines(fd.numel() // 512, 32, seed=13)
    src = gather_lines(fd, direction, shape, lines).double().cpu().numpy()
    plan = make_plan(shape, direction, order, "closed", "f32")
    y = plan.thomas(fd)
    got = gather_lines(y, direction, shape, lines).double().cpu().numpy()
    mx, rms = rel_errors(got, oracle.deriv_lines(src, order, "closed", oracle.grid_spacing(512, "closed")))
    report("512^3 thomas smooth D%d %s closed" % (order, direction), dtype="f32", max_rel=mx, rms_rel=rms)
    assert mx <= TOL["f32"], (mx, rms)
