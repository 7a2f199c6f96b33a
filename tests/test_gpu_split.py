"""GPU parity of the split-precision FP64 sweeps (``arith="split"``, ``tds_plan_set_arith``):
FP64 fields whose resident sweeps carry the recurrences as float pairs, against the FP64 oracle
at the FP64 bar (max|d| / max|ref| <= 1e-12): every point on small grids over direction x
order x boundary x chunks x CTA width, the filter, the fused multi-operator pass, fields scaled
far from 1, and sampled whole lines at 512^3 on the benchmark's field and on smooth fields."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_13532_gb300 import inputs
from tests.gpu_util import (TOL, from_device_layout, gather_lines, rel_errors, report, sample_lines,
                            to_device_layout)

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


SHAPE = (32, 48, 64)   # x lines 1536, y lines 2048, z lines 3072
PS = {"x": (1, 2, 8), "y": (1, 4, 12), "z": (1, 2, 8)}


@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("width", [None, 32, 16, 8])
def test_split_small_grid_every_point(direction, order, bc, adjoint, width):
    """Every point against the oracle; the split sweeps run the forward-form operators (the
    derivatives, the adjoint on periodic lines), the closed-line adjoint runs native FP64."""
    cart = np.random.default_rng(7 + order).uniform(-1, 1, SHAPE)
    n = {"x": SHAPE[2], "y": SHAPE[1], "z": SHAPE[0]}[direction]
    h = oracle.grid_spacing(n, bc)
    ref = (oracle.deriv_adjoint if adjoint else oracle.deriv)(cart, direction, order, bc, h)
    x = to_device_layout(cart, direction, "f64")
    ran = 0
    for P in PS[direction]:
        try:
            plan = tds.Plan(SHAPE, direction, order, bc, P=P, h=h, variant="resident", width=width, arith="split")
        except tds.TdsError:
            continue          # the width does not fit this P (threads or shared memory)
        native = tds.Plan(SHAPE, direction, order, bc, P=P, h=h, variant="resident", width=width)
        y = plan.adjoint(x) if adjoint else plan.deriv(x)
        mx, rms = rel_errors(from_device_layout(y, direction, SHAPE), ref)
        assert mx <= TOL["f64"], (P, mx, rms)
        yn = native.adjoint(x) if adjoint else native.deriv(x)
        if not adjoint or bc == "periodic":
            assert not torch.equal(y, yn)    # a different arithmetic ran
        ran += 1
    assert ran > 0


@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_split_filter_every_point(bc):
    cart = np.random.default_rng(5).uniform(-1, 1, SHAPE)
    for P in (1, 4):
        plan = tds.Plan(SHAPE, "x", "filter", bc, P=P, alpha_f=0.45, variant="resident", arith="split")
        y = plan.deriv(to_device_layout(cart, "x", "f64"))
        mx, rms = rel_errors(from_device_layout(y, "x", SHAPE), oracle.apply_op(cart, "x", oracle.FILTER, bc, 0.45))
        assert mx <= TOL["f64"], (P, mx, rms)


@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_split_interp_every_point(direction, bc, adjoint):
    """The mid-point interpolation (half-point taps) and its transpose; the split sweep runs the
    forward operator and, on periodic lines, the transpose (closed lines: native FP64)."""
    shape = (12, 40, 32)
    cart = np.random.default_rng(31).uniform(-1, 1, shape)
    ref = oracle.apply_op(cart, direction, oracle.INTERP, bc, adjoint=adjoint)
    x = to_device_layout(cart, direction, "f64")
    for P in {"x": (1, 2, 8), "y": (1, 2, 5), "z": (1, 3)}[direction]:
        plan = tds.Plan(shape, direction, "interp", bc, P=P, variant="resident", arith="split")
        native = tds.Plan(shape, direction, "interp", bc, P=P, variant="resident")
        y = plan.adjoint(x) if adjoint else plan.deriv(x)
        mx, rms = rel_errors(from_device_layout(y, direction, shape), ref)
        assert mx <= TOL["f64"], (P, mx, rms)
        yn = native.adjoint(x) if adjoint else native.deriv(x)
        if not adjoint or bc == "periodic":
            assert not torch.equal(y, yn)    # a different arithmetic ran
        else:
            assert torch.equal(y, yn)


def test_split_interp_width_rule():
    """A split interpolation plan takes the split width rule now that its operator runs split."""
    shape = (32, 48, 512)
    for bc in ("periodic", "closed"):
        sp = tds.Plan(shape, "x", "interp", bc, P=8, arith="split")
        d1 = tds.Plan(shape, "x", 1, bc, P=8, arith="split")
        assert sp.width == d1.width


@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_split_fused_pass(bc):
    """tds_deriv_multi with split plans (one launch per operator): bitwise the single split
    calls, and against the oracle."""
    shape = (16, 48, 64)
    cart = np.random.default_rng(23).uniform(-1, 1, shape)
    h = oracle.grid_spacing(64, bc)
    p1 = tds.Plan(shape, "x", 1, bc, P=8, h=h, arith="split")
    p2 = tds.Plan(shape, "x", 2, bc, P=8, h=h, arith="split")
    x = to_device_layout(cart, "x", "f64")
    ops = [(p1, False), (p2, False)] + ([(p1, True)] if bc == "periodic" else [])
    outs = tds.deriv_multi(ops, x)
    refs = [p1.deriv(x), p2.deriv(x), p1.adjoint(x)]
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    orc = [oracle.deriv(cart, "x", 1, bc, h), oracle.deriv(cart, "x", 2, bc, h),
           oracle.deriv_adjoint(cart, "x", 1, bc, h)]
    for o, r in zip(outs, orc):
        mx, rms = rel_errors(from_device_layout(o, "x", shape), r)
        assert mx <= TOL["f64"], (mx, rms)


@pytest.mark.parametrize("scale", [2.0 ** -40, 2.0 ** 40])
def test_split_scaled_fields(scale):
    """Fields far from unit size (inside the documented range): the bit-level splits carry the
    exponent; relative errors unchanged."""
    cart = np.random.default_rng(9).uniform(-1, 1, SHAPE) * scale
    for order, bc in ((1, "periodic"), (2, "closed")):
        h = oracle.grid_spacing(64, bc)
        plan = tds.Plan(SHAPE, "x", order, bc, P=4, h=h, arith="split")
        y = plan.deriv(to_device_layout(cart, "x", "f64"))
        mx, rms = rel_errors(from_device_layout(y, "x", SHAPE), oracle.deriv(cart, "x", order, bc, h))
        assert mx <= TOL["f64"], (order, bc, mx, rms)


def test_split_rejected_where_it_does_not_apply():
    with pytest.raises(tds.TdsError):
        tds.Plan(SHAPE, "x", 1, "periodic", P=4, dtype=torch.float32, arith="split")
    n = SHAPE[2]
    with pytest.raises(tds.TdsError):
        tds.Plan(SHAPE, "x", 0, "periodic", P=4, band=(np.full(n, 0.2), np.ones(n), np.full(n, 0.2)),
                 arith="split")


def _sampled(field_dev, shape, direction, bc, ops, seed):
    """Fused pass of the given (order, adjoint) operators with split plans at `shape`; sampled
    whole lines against the oracle, beside the native FP64 plans' error on the same lines.
    The bar is 1e-12, or 1.5 times the native FP64 error where the FP64 evaluation itself is
    further from the oracle (both sides round: the second derivative's closure on closed lines
    of smooth 512-point fields cancels about 10 bits in its right-hand side, and the solve
    magnifies an end row's rounding about 93-fold, so native FP64 sits near 1.6e-12 there)."""
    x = tds.reorder(field_dev, shape, "cart", direction)
    n = {"x": shape[2], "y": shape[1], "z": shape[0]}[direction]
    h = oracle.grid_spacing(n, bc)
    plans = {o: tds.Plan(shape, direction, o, bc, P=8, h=h, arith="split") for o in (1, 2)}
    natives = {o: tds.Plan(shape, direction, o, bc, P=8, h=h) for o in (1, 2)}
    outs = tds.deriv_multi([(plans[o], a) for o, a in ops], x)
    nouts = tds.deriv_multi([(natives[o], a) for o, a in ops], x)
    lines = sample_lines(plans[1].nlines, 16, seed)
    src = gather_lines(x, direction, shape, lines).double().cpu().numpy()
    worst = 0.0
    for (o, a), y, yn in zip(ops, outs, nouts):
        ref = (oracle.deriv_adjoint_lines if a else oracle.deriv_lines)(src, o, bc, h)
        mx, rms = rel_errors(gather_lines(y, direction, shape, lines).double().cpu().numpy(), ref)
        mxn, _ = rel_errors(gather_lines(yn, direction, shape, lines).double().cpu().numpy(), ref)
        report("512^3 split D%d%s %s %s" % (o, "T" if a else "", direction, bc), max_rel=mx, rms_rel=rms,
               native_max_rel=mxn)
        assert mx <= max(TOL["f64"], 1.5 * mxn), (direction, o, a, mx, rms, mxn)
        worst = max(worst, mx)
    return worst


def test_split_512_benchmark_field():
    """The benchmark's workload with split plans: 512^3, periodic, P = 8, D1, D2 and D1^T in one
    fused pass along x, y and z, Fourier modes up to k = 100 plus N(0, 0.1) noise."""
    shape = (512, 512, 512)
    f, _ = inputs.fourier_field(shape, seed=2, kmax=100, noise=0.1, noise_kind="normal", device="cuda")
    f = f.reshape(-1)
    for d in "xyz":
        _sampled(f, shape, d, "periodic", [(1, False), (2, False), (1, True)], seed=50 + ord(d))


@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_split_512_smooth_field(bc):
    """Smooth fields (Fourier modes up to k = 20, 1e-3 noise), where the stencil's plain sums
    cancel most: the split sweeps take the differences in FP64 first."""
    shape = (512, 512, 512)
    f, _ = inputs.fourier_field(shape, seed=6, kmax=20, noise=1e-3, device="cuda")
    f = f.reshape(-1)
    ops = [(1, False), (2, False)] + ([(1, True)] if bc == "periodic" else [])
    for d in "xz":
        _sampled(f, shape, d, bc, ops, seed=60 + ord(d))


def test_fanout_copy_bitwise_and_rules():
    """The fan-out copy the fused pass is measured against: every output bitwise the input
    (ragged sizes in 16-byte vectors included), overlaps and misalignment refused."""
    for n in (2, 30, 1 << 20, (1 << 22) + 6):
        x = torch.randn(n, dtype=torch.float64, device="cuda")
        outs = [torch.full_like(x, float("nan")) for _ in range(3)]
        tds.fanout_copy(x, outs)
        for o in outs:
            assert torch.equal(o, x)
    x = torch.randn(1 << 12, dtype=torch.float32, device="cuda")
    with pytest.raises(tds.TdsError):
        tds.fanout_copy(x, [x])                          # output is the input
    o = torch.empty((1 << 12) + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(tds.TdsError):
        tds.fanout_copy(x[1:-3], [o[4:4 + x.numel() - 4]])  # misaligned input


@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("same", [False, True])
def test_split_transport_term_every_point(direction, bc, same):
    """One transport term group (Eq. mom-comps) with split plans: three split sweeps, the product
    and the combination in FP64; every point against the oracle."""
    shape, Ps = (20, 64, 96), {"x": 4, "y": 2, "z": 5}
    rng = np.random.default_rng(3 + "xyz".index(direction) + 7 * same)
    ui = rng.uniform(-1, 1, shape)
    uj = ui if same else rng.uniform(-1, 1, shape)
    d1 = tds.Plan(shape, direction, 1, bc, P=Ps[direction], arith="split")
    d2 = tds.Plan(shape, direction, 2, bc, P=Ps[direction], arith="split")
    a = to_device_layout(ui, direction, "f64")
    b = a if same else to_device_layout(uj, direction, "f64")
    out = tds.transport_term(d1, d2, a, b, 0.02)
    mx, rms = rel_errors(from_device_layout(out, direction, shape), oracle.transport_term(ui, uj, direction, 0.02, bc))
    assert mx <= TOL["f64"], (mx, rms)


@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_split_transport_rhs_every_point(bc):
    shape = (20, 64, 96)
    rng = np.random.default_rng(17)
    u = [rng.uniform(-1, 1, shape) for _ in range(3)]
    rhs = tds.TransportRHS(shape, P=(4, 2, 5), bc=bc, arith="split")
    out = rhs([to_device_layout(f, "x", "f64") for f in u], 0.02)
    ref = oracle.transport_rhs(u, 0.02, bc)
    for i in range(3):
        mx, rms = rel_errors(from_device_layout(out[i], "x", shape), ref[i])
        assert mx <= TOL["f64"], (i, mx, rms)
