"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Small grids: every output compared with the oracle, over dtype x variant x direction x order
x boundary x P, sized to span several groups and chunks with a ragged group count.
Full sizes (the workloads of the benchmark): sampled whole lines compared one by one with
the oracle.  Bars: max|d|/max|ref| <= 1e-12 (FP64) and <= 1e-5 (FP32, against the oracle
on the FP32-rounded input)."""
import math

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


SMALL = (12, 40, 32)   # (nz, ny, nx): x lines 480 (15 groups), y lines 384, z lines 1280
PS = {"x": [1, 2, 8], "y": [1, 2, 5], "z": [1, 3]}


def small_case(direction, order, bc, P, dtype, variant, adjoint, seed):
    cart = np.random.default_rng(seed).uniform(-1, 1, SMALL)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    n = {"x": SMALL[2], "y": SMALL[1], "z": SMALL[0]}[direction]
    h = oracle.grid_spacing(n, bc)
    plan = tds.Plan(SMALL, direction, order, bc, P=P, h=h, dtype=TORCH[dtype], variant=variant)
    x = to_device_layout(cart, direction, dtype)
    y = plan.adjoint(x) if adjoint else plan.deriv(x)
    torch.cuda.synchronize()
    got = from_device_layout(y, direction, SMALL)
    ref = (oracle.deriv_adjoint if adjoint else oracle.deriv)(cart, direction, order, bc, h)
    return rel_errors(got, ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["resident", "pipelined", "streaming"])
@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_small_grid_every_point(dtype, variant, direction, order, bc, adjoint):
    for i, P in enumerate(PS[direction]):
        mx, rms = small_case(direction, order, bc, P, dtype, variant, adjoint, seed=11 + i)
        assert mx <= TOL[dtype], (P, mx, rms)


WSHAPE = (32, 48, 64)   # x lines 1536 (48 groups), y lines 2048, z lines 3072
WIDTH_P = {16: {"x": 4, "y": 4, "z": 4}, 8: {"x": 8, "y": 12, "z": 8}}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["resident", "pipelined"])
@pytest.mark.parametrize("width", [16, 8])
@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_resident_width_every_point(dtype, variant, width, direction, order, bc, adjoint):
    """A group split over 32/width CTAs (rows moved as 2-D TMA tensor boxes), one CTA per unit
    or persistent CTAs walking the units: every point against the oracle."""
    P = WIDTH_P[width][direction]
    cart = np.random.default_rng(width + P).uniform(-1, 1, WSHAPE)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    n = {"x": WSHAPE[2], "y": WSHAPE[1], "z": WSHAPE[0]}[direction]
    h = oracle.grid_spacing(n, bc)
    plan = tds.Plan(WSHAPE, direction, order, bc, P=P, h=h, dtype=TORCH[dtype], variant=variant,
                    width=width)
    assert plan.width == width and plan.variant == variant
    x = to_device_layout(cart, direction, dtype)
    y = plan.adjoint(x) if adjoint else plan.deriv(x)
    got = from_device_layout(y, direction, WSHAPE)
    ref = (oracle.deriv_adjoint if adjoint else oracle.deriv)(cart, direction, order, bc, h)
    mx, rms = rel_errors(got, ref)
    assert mx <= TOL[dtype], (P, mx, rms)


def test_resident_width_choice_and_limits():
    """The planner's width among those that let two CTAs share an SM: FP64 the smallest, FP32
    the largest; impossible widths are refused."""
    cube = (512, 512, 512)
    assert tds.Plan(cube, "x", 1, "periodic", P=8).width == 8                       # FP64 512^3
    assert tds.Plan(cube, "x", 1, "periodic", P=8, dtype=torch.float32).width == 32
    assert tds.Plan((1024,) * 3, "z", 1, "periodic", P=8, dtype=torch.float32).width == 16
    assert tds.Plan((1024,) * 3, "z", 1, "periodic", P=8).width == 8
    assert tds.Plan((16, 16, 64), "x", 1, "periodic", P=2).width == 32              # 2 warps rule
    for bad in (4, 24, 64):
        with pytest.raises(tds.TdsError):
            tds.Plan((16, 16, 64), "x", 1, "periodic", P=8, width=bad)
    with pytest.raises(tds.TdsError):   # 2 x 8 lines: fewer than two warps per CTA
        tds.Plan((16, 16, 64), "x", 1, "periodic", P=2, width=8)


HOST_CASES = [   # (shape, direction, P, variant, width): groups = lines / 32
    ((12, 40, 32), "x", 8, "resident", None),     # 15 groups: ragged slabs
    ((16, 48, 64), "x", 8, "resident", 8),        # 24 groups, 4 CTAs per group
    ((12, 40, 32), "z", 3, "streaming", None),    # 40 groups
    ((12, 40, 32), "y", 5, "pipelined", None),    # 12 groups
    ((1, 32, 2048), "x", 4, "segmented", None),   # 1 group: fewer groups than slabs
    ((2, 32, 256), "x", 2, "resident", None),     # 2 groups
    ((4, 32, 512), "x", 1, "segmented", None),    # 4 groups, periodic: the adjoint on the segments
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", range(len(HOST_CASES)))
def test_host_entry_points_match_device_calls(dtype, case):
    """tds_deriv_host / tds_deriv_adjoint_host (slab-pipelined copies) give bitwise the result
    of tds_deriv / tds_deriv_adjoint on device buffers, with and without the input copy."""
    shape, direction, P, variant, width = HOST_CASES[case]
    bc = "closed" if case % 2 else "periodic"
    plan = tds.Plan(shape, direction, 1, bc, P=P, dtype=TORCH[dtype], variant=variant, width=width)
    numel = plan.numel
    g = torch.Generator(device="cuda").manual_seed(case)
    x = torch.rand(numel, generator=g, device="cuda", dtype=TORCH[dtype]) - 0.5
    ref_f = plan.deriv(x)
    ref_a = plan.adjoint(x)
    host_in = x.cpu().pin_memory()
    outs = [torch.full((numel,), float("nan"), dtype=TORCH[dtype]).pin_memory() for _ in range(3)]
    d_in = torch.zeros_like(x)
    d_out = torch.empty_like(x)
    plan.deriv_host(host_in, outs[0], d_in, d_out)          # copies the input in
    plan.deriv_host(None, outs[1], d_in, d_out)             # input already in d_in
    plan.adjoint_host(None, outs[2], d_in, d_out)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(outs[0], ref_f.cpu())
    assert torch.equal(outs[1], ref_f.cpu())
    assert torch.equal(outs[2], ref_a.cpu())
    assert torch.equal(d_in, x)


def oracle_solve_lines(lines, order, bc, h):
    """x = A^{-1} d per line with the oracle's band and its (cyclic) Thomas solver."""
    n = lines.shape[1]
    a, b, c, _ = oracle.bands(n, order, bc, h)
    return np.stack([oracle.tridiag_solve(a, b, c, d, bc == "periodic") for d in lines])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["resident", "pipelined", "streaming", "segmented"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_solve_every_point(dtype, variant, order, bc):
    """tds_solve (A^{-1} d, the DistD2 solve alone) against the oracle's Thomas / Sherman-Morrison
    solve of the same band, every point, several chunk counts."""
    shape = (2, 32, 512) if variant == "segmented" else (4, 40, 64)
    n = shape[2]
    h = oracle.grid_spacing(n, bc)
    cart = np.random.default_rng(order + 3).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    ref = oracle.from_lines_view(oracle_solve_lines(oracle.lines_view(cart, "x"), order, bc, h), "x", shape)
    for P in ((1, 2, 4) if variant == "segmented" else (1, 2, 8)):
        try:
            plan = tds.Plan(shape, "x", order, bc, P=P, h=h, dtype=TORCH[dtype], variant=variant)
        except tds.TdsError:
            continue   # segments need chunks of at least 64 rows
        y = plan.solve(to_device_layout(cart, "x", dtype))
        mx, rms = rel_errors(from_device_layout(y, "x", shape), ref)
        assert mx <= TOL[dtype], (P, mx, rms)


def random_band(n, P, periodic, seed):
    """A diagonally dominant band with a uniform interior and its own first / last rows (one
    class per first / interior / last chunk)."""
    rng = np.random.default_rng(seed)
    ai, ci = rng.uniform(-0.45, 0.45, 2)
    bi = 1.0 + rng.uniform(0.0, 0.5)
    a = np.full(n, ai); b = np.full(n, bi); c = np.full(n, ci)
    if not periodic:   # distinct closure rows in the first and last chunk
        k = min(3, n // P)
        a[:k] = rng.uniform(-0.4, 0.4, k); b[:k] = rng.uniform(1.0, 2.0, k); c[:k] = rng.uniform(-0.4, 0.4, k)
        a[-k:] = rng.uniform(-0.4, 0.4, k); b[-k:] = rng.uniform(1.0, 2.0, k); c[-k:] = rng.uniform(-0.4, 0.4, k)
    return a, b, c


def variable_band(n, seed, kind):
    """Bands whose coefficients vary along the whole line, as ADI systems have them:
    "random" -- independent diagonally dominant rows; "grid" -- backward-Euler diffusion
    (I - dt d/dx (kappa d/dx)) on a stretched grid with a variable diffusivity kappa(x), the time
    step chosen so that the largest dt kappa / dx^2 is 100 (condition number about 400)."""
    rng = np.random.default_rng(seed)
    if kind == "random":
        a = rng.uniform(-0.45, 0.45, n); c = rng.uniform(-0.45, 0.45, n)
        b = (np.abs(a) + np.abs(c)) * rng.uniform(1.2, 2.0, n) + rng.uniform(0.1, 0.3, n)
        b *= np.where(rng.uniform(size=n) < 0.3, -1.0, 1.0)   # dominant diagonal of either sign
        return a, b, c
    return inputs.diffusion_band(n, seed, dmax=100.0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("variant", ["resident", "streaming"])
def test_band_plan_solve(dtype, bc, variant):
    """A caller-given band: every point of tds_solve against the oracle's (cyclic) Thomas solve of
    the same band, for several chunk counts and directions: bands with one class per first /
    interior / last chunk, and bands whose rows all differ (every chunk its own class)."""
    shape = (8, 40, 64)
    cart = np.random.default_rng(31).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    for direction, Ps in (("x", (1, 2, 8, 16)), ("y", (1, 5, 10)), ("z", (1, 2))):
        n = {"x": shape[2], "y": shape[1], "z": shape[0]}[direction]
        for P in Ps:
            for kind in ("classes", "random", "grid"):
                a, b, c = (random_band(n, P, bc == "periodic", seed=n + P) if kind == "classes"
                           else variable_band(n, seed=n + P, kind=kind))
                plan = tds.Plan(shape, direction, 0, bc, P=P, dtype=TORCH[dtype], variant=variant, band=(a, b, c))
                y = plan.solve(to_device_layout(cart, direction, dtype))
                lines = oracle.lines_view(cart, direction)
                ref = np.stack([oracle.tridiag_solve(a, b, c, d, bc == "periodic") for d in lines])
                mx, rms = rel_errors(from_device_layout(y, direction, shape),
                                     oracle.from_lines_view(ref, direction, shape))
                assert mx <= TOL[dtype], (direction, P, kind, mx, rms)


@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_band_plan_long_lines_many_chunks(bc):
    """Variable bands on long lines cut into many chunks (every chunk its own class): n = 4096,
    P = 64 (streaming) and n = 1024, P = 16 (resident), FP64 and FP32, every point."""
    for n, P, variant in ((4096, 64, "streaming"), (1024, 16, "resident")):
        shape = (1, 32, n)
        cart = np.random.default_rng(n).uniform(-1, 1, shape)
        a, b, c = variable_band(n, seed=P, kind="grid")
        for dtype in ("f64", "f32"):
            src = cart.astype(np.float32).astype(np.float64) if dtype == "f32" else cart
            plan = tds.Plan(shape, "x", 0, bc, P=P, dtype=TORCH[dtype], variant=variant, band=(a, b, c))
            y = plan.solve(to_device_layout(src, "x", dtype))
            ref = np.stack([oracle.tridiag_solve(a, b, c, d, bc == "periodic") for d in oracle.lines_view(src, "x")])
            mx, rms = rel_errors(from_device_layout(y, "x", shape), oracle.from_lines_view(ref, "x", shape))
            report("band %s n=%d P=%d" % (bc, n, P), dtype=dtype, variant=plan.variant, max_rel=mx, rms_rel=rms)
            assert mx <= TOL[dtype], (n, P, dtype, mx, rms)


def test_band_plan_rules():
    shape = (8, 32, 64)
    a, b, c = random_band(64, 4, False, seed=1)
    # a non-finite entry
    bad = b.copy(); bad[20] = np.nan
    with pytest.raises(tds.TdsError):
        tds.Plan(shape, "x", 0, "closed", P=4, band=(a, bad, c))
    # a zero pivot
    z = b.copy(); z[0] = 0.0
    with pytest.raises(tds.TdsError):
        tds.Plan(shape, "x", 0, "closed", P=4, band=(np.zeros(64), z, c))
    # a band plan has no stencil: the derivative calls are refused
    plan = tds.Plan(shape, "x", 0, "closed", P=4, band=(a, b, c))
    x = torch.zeros(plan.numel, dtype=torch.float64, device="cuda")
    for fn in (plan.deriv, plan.adjoint):
        with pytest.raises(tds.TdsError):
            fn(x)
    with pytest.raises(tds.TdsError):
        tds.deriv_multi([(plan, False)], x)


@pytest.mark.parametrize("width", [16, 8])
def test_solve_split_groups(width):
    P = WIDTH_P[width]["x"]
    cart = np.random.default_rng(width).uniform(-1, 1, WSHAPE)
    for bc in ("periodic", "closed"):
        h = oracle.grid_spacing(WSHAPE[2], bc)
        plan = tds.Plan(WSHAPE, "x", 1, bc, P=P, h=h, variant="resident", width=width)
        y = plan.solve(to_device_layout(cart, "x", "f64"))
        ref = oracle.from_lines_view(oracle_solve_lines(oracle.lines_view(cart, "x"), 1, bc, h), "x", WSHAPE)
        mx, rms = rel_errors(from_device_layout(y, "x", WSHAPE), ref)
        assert mx <= TOL["f64"], (bc, mx, rms)


@pytest.fixture(params=["ilv", "seq"])
def multi_form(request, monkeypatch):
    """Both forms of the fused pass: one CTA per (unit, operator) (the default) and one CTA per
    unit sweeping the operators in turn (TDS_MULTI_FORM=seq, read at every launch)."""
    if request.param == "seq":
        monkeypatch.setenv("TDS_MULTI_FORM", "seq")
    else:
        monkeypatch.delenv("TDS_MULTI_FORM", raising=False)
    return request.param


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("width", [None, 16, 8])
def test_multi_operator_pass_matches_single_calls(dtype, bc, width, multi_form):
    """tds_deriv_multi (D1, D2 and D1^T of one input; one fused pass when the operators have
    the forward form, one after another otherwise) gives bitwise the single calls' results."""
    shape = (16, 48, 64)
    t = TORCH[dtype]
    p1 = tds.Plan(shape, "x", 1, bc, P=8, dtype=t, width=width)
    p2 = tds.Plan(shape, "x", 2, bc, P=8, dtype=t, width=width)
    x = inputs.uniform_field(shape, seed=21, device="cuda", dtype=t).reshape(-1)
    refs = [p1.deriv(x), p2.deriv(x), p1.adjoint(x)]
    outs = tds.deriv_multi([(p1, False), (p2, False), (p1, True)], x)
    for r, o in zip(refs, outs):
        assert torch.equal(r, o)
    # one operator, and a repeated operator
    o1 = tds.deriv_multi([(p2, False)], x)[0]
    assert torch.equal(o1, refs[1])
    o2 = tds.deriv_multi([(p1, False), (p2, False), (p1, False), (p2, False)], x)
    assert torch.equal(o2[2], refs[0]) and torch.equal(o2[3], refs[1])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multi_operator_pass_512_sampled_lines(dtype):
    """The fused pass the benchmark times, at its size: 512^3, periodic, P = 8, D1, D2 and D1^T
    of one input in one launch (one CTA per unit and operator), along x, y and z, on the
    benchmark's field (Fourier modes up to k = 100 plus N(0, 0.1) noise).  Sampled whole lines
    of every result against the oracle on the same (FP32-rounded for FP32) lines."""
    shape = (512, 512, 512)
    t = TORCH[dtype]
    f, _ = inputs.fourier_field(shape, seed=2, kmax=100, noise=0.1, noise_kind="normal", device="cuda")
    cart = f.to(t).reshape(-1)
    del f
    h = oracle.grid_spacing(512, "periodic")
    for direction in "xyz":
        x = tds.reorder(cart, shape, "cart", direction)
        p1 = tds.Plan(shape, direction, 1, "periodic", P=8, h=h, dtype=t)
        p2 = tds.Plan(shape, direction, 2, "periodic", P=8, h=h, dtype=t)
        assert p1.variant == p2.variant == "resident" and p1.width == p2.width   # one fused launch
        outs = tds.deriv_multi([(p1, False), (p2, False), (p1, True)], x)
        lines = sample_lines(p1.nlines, 16, seed=40 + ord(direction))
        src = gather_lines(x, direction, shape, lines).double().cpu().numpy()
        refs = [oracle.deriv_lines(src, 1, "periodic", h), oracle.deriv_lines(src, 2, "periodic", h),
                oracle.deriv_adjoint_lines(src, 1, "periodic", h)]
        for name, o, ref in zip(("D1", "D2", "D1T"), outs, refs):
            got = gather_lines(o, direction, shape, lines).double().cpu().numpy()
            mx, rms = rel_errors(got, ref)
            report("512^3 fused %s %s periodic P=8" % (name, direction), dtype=dtype, max_rel=mx, rms_rel=rms)
            assert mx <= TOL[dtype], (direction, name, mx, rms)
        del x, outs


def test_multi_operator_pass_fallbacks_and_errors():
    shape = (12, 40, 32)
    x = inputs.uniform_field(shape, seed=22, device="cuda").reshape(-1)
    ps = tds.Plan(shape, "z", 1, "periodic", P=3, variant="streaming")
    pr = tds.Plan(shape, "z", 2, "periodic", P=3)
    outs = tds.deriv_multi([(ps, False), (pr, False), (ps, True)], x)
    assert torch.equal(outs[0], ps.deriv(x)) and torch.equal(outs[1], pr.deriv(x))
    assert torch.equal(outs[2], ps.adjoint(x))
    other = tds.Plan(shape, "y", 1, "periodic", P=5)   # another direction: another layout
    with pytest.raises(tds.TdsError):
        tds.deriv_multi([(pr, False), (other, False)], x)
    with pytest.raises(tds.TdsError):   # an output aliasing the input
        tds.deriv_multi([(pr, False)], x, outs=[x])
    o = torch.empty_like(x)
    with pytest.raises(tds.TdsError):   # two outputs aliasing each other
        tds.deriv_multi([(pr, False), (pr, False)], x, outs=[o, o])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("order", [1, 2])
def test_segmented_long_lines(dtype, bc, order):
    """Lines longer than one CTA's shared memory: segments of 64..256 rows subdivide the chunks
    (two kernels); every point against the oracle, for several chunk lengths."""
    shape = (1, 32, 2048)
    cart = np.random.default_rng(order).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    h = oracle.grid_spacing(2048, bc)
    ref = oracle.deriv(cart, "x", order, bc, h)
    for P in (1, 2, 4, 8, 16):
        plan = tds.Plan(shape, "x", order, bc, P=P, h=h, dtype=TORCH[dtype], variant="segmented")
        y = plan.deriv(to_device_layout(cart, "x", dtype))
        mx, rms = rel_errors(from_device_layout(y, "x", shape), ref)
        assert mx <= TOL[dtype], (P, mx, rms)
        # the adjoint of a segmented plan (streaming pipeline)
        ya = plan.adjoint(to_device_layout(cart, "x", dtype))
        mx, _ = rel_errors(from_device_layout(ya, "x", shape), oracle.deriv_adjoint(cart, "x", order, bc, h))
        assert mx <= TOL[dtype], (P, "adjoint", mx)


def test_segmented_is_chosen_for_long_lines():
    assert tds.Plan((1, 32, 2048), "x", 1, "periodic", P=4).variant == "segmented"
    assert tds.Plan((1, 32, 4096), "x", 1, "periodic", P=4, dtype=torch.float32).variant == "segmented"
    assert tds.Plan((1, 32, 512), "x", 1, "periodic", P=8).variant == "resident"
    # few chunks: resident CTAs would leave fewer than 6 warps per SM, segments give more
    assert tds.Plan((8, 32, 256), "x", 1, "periodic", P=1).variant == "segmented"   # 3 warps / SM
    assert tds.Plan((8, 32, 256), "x", 1, "periodic", P=2).variant == "resident"    # 6 warps / SM
    assert tds.Plan((1, 32, 512), "x", 1, "periodic", P=2).variant == "segmented"   # 2 warps / SM
    # FP32 stays resident (thin plans run on finer chunks) ...
    assert tds.Plan((1, 32, 512), "x", 1, "periodic", P=1, dtype=torch.float32).variant == "resident"
    # ... unless the lines need 8-line CTAs: segments read the input about 1.2 times
    assert tds.Plan((1, 32, 2048), "x", 1, "periodic", P=8, dtype=torch.float32).variant == "segmented"
    assert tds.Plan((1, 32, 1024), "x", 1, "periodic", P=8, dtype=torch.float32).variant == "resident"
    # a single 64-row segment per line: resident
    assert tds.Plan((8, 32, 64), "x", 1, "periodic", P=1).variant == "resident"
    # chunks too short for 64-row segments fall back to streaming
    assert tds.Plan((1, 32, 2048), "x", 1, "periodic", P=64).variant == "streaming"


@pytest.mark.parametrize("variant", ["resident", "pipelined", "streaming"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_minimum_chunk_and_line(variant, bc):
    """n = 8 (the smallest line) and m = 4 (the smallest chunk)."""
    shape = (1, 32, 8)
    cart = np.random.default_rng(5).uniform(-1, 1, shape)
    for P in (1, 2):
        for order in (1, 2):
            for dtype in ("f64", "f32"):
                c = cart.astype(np.float32).astype(np.float64) if dtype == "f32" else cart
                h = oracle.grid_spacing(8, bc)
                plan = tds.Plan(shape, "x", order, bc, P=P, h=h, variant=variant, dtype=TORCH[dtype])
                y = plan.deriv(to_device_layout(c, "x", dtype))
                got = from_device_layout(y, "x", shape)
                mx, _ = rel_errors(got, oracle.deriv(c, "x", order, bc, h))
                assert mx <= TOL[dtype], (P, order, dtype, mx)


@pytest.mark.parametrize("variant", ["resident", "pipelined", "streaming"])
def test_p_invariance(variant):
    """Chunking does not change the result (order-of-accuracy study of Sec. 4.2: the
    partitioned solver matches the single-rank solver)."""
    shape = (2, 16, 256)
    cart = np.random.default_rng(9).uniform(-1, 1, shape)
    x = to_device_layout(cart, "x", "f64")
    for bc in ("periodic", "closed"):
        base = tds.Plan(shape, "x", 1, bc, P=1, variant=variant).deriv(x)
        for P in (2, 4, 8, 16, 32, 64):
            if variant != "streaming" and P > 16:
                continue
            y = tds.Plan(shape, "x", 1, bc, P=P, variant=variant).deriv(x)
            mx, _ = rel_errors(y.cpu().numpy(), base.cpu().numpy())
            assert mx <= 1e-13, (bc, P, mx)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_variants_agree(dtype):
    """The fused resident sweep and the three-kernel streaming pipeline (the paper's phase
    order) agree: to rounding in FP64; each within the FP32 bar of the oracle in FP32."""
    shape = (4, 8, 128)
    cart = np.random.default_rng(2).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    x = to_device_layout(cart, "x", dtype)
    for order in (1, 2):
        ref = oracle.deriv(cart, "x", order, "closed")
        ys = [tds.Plan(shape, "x", order, "closed", P=4, variant=v, dtype=TORCH[dtype]).deriv(x)
              for v in ("resident", "pipelined", "streaming")]
        for y in ys:
            mx, _ = rel_errors(from_device_layout(y, "x", shape), ref)
            assert mx <= TOL[dtype], (order, mx)
        if dtype == "f64":
            for y in ys[1:]:
                mx, _ = rel_errors(y.cpu().numpy(), ys[0].cpu().numpy())
                assert mx <= 1e-14, (order, mx)


def test_bitwise_deterministic():
    shape = (4, 8, 256)
    x = to_device_layout(np.random.default_rng(3).uniform(-1, 1, shape), "x", "f64")
    for variant in ("resident", "pipelined", "streaming"):
        plan = tds.Plan(shape, "x", 2, "periodic", P=4, variant=variant)
        a = plan.deriv(x); b = plan.deriv(x)
        assert torch.equal(a, b)


@pytest.mark.parametrize("m", [8, 16, 32])
def test_paper_drop_mode_error_bound(m):
    """Dropping the two couplings per chunk (Fig. alg) costs O(|lambda|^m), lambda the
    decay ratio of A^{-1} (0.382 for alpha = 1/3)."""
    P = 4; n = P * m
    shape = (1, 32, n)
    cart = np.random.default_rng(m).uniform(-1, 1, shape)
    lam = (1 - math.sqrt(1 - 4 / 9)) / (2 / 3)
    for variant in ("resident", "pipelined", "streaming"):
        y = tds.Plan(shape, "x", 1, "periodic", P=P, mode="paper_drop", variant=variant).deriv(
            to_device_layout(cart, "x", "f64"))
        mx, _ = rel_errors(from_device_layout(y, "x", shape), oracle.deriv(cart, "x", 1, "periodic"))
        assert mx <= 8 * lam ** m + 1e-13, (variant, mx, lam ** m)


@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("P", [1, 3, 8])
def test_reduced_system_against_dense_solve(bc, P):
    shape = (1, 32, 8 * P)
    plan = tds.Plan(shape, "x", 1, bc, P=P)
    sub, sup = plan.reduced_coeffs()
    R = 2 * P
    M = np.eye(R)
    for i in range(R):
        if i > 0: M[i, i - 1] += sub[i]
        elif bc == "periodic": M[i, R - 1] += sub[i]
        if i < R - 1: M[i, i + 1] += sup[i]
        elif bc == "periodic": M[i, 0] += sup[i]
    rhs = np.random.default_rng(P).normal(size=(plan.nlines, R))
    x = plan.reduced_solve(torch.from_numpy(rhs).cuda()).cpu().numpy()
    ref = np.linalg.solve(M, rhs.T).T
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_argument_errors_on_device():
    shape = (1, 32, 64)
    plan = tds.Plan(shape, "x", 1, "periodic", P=2, variant="streaming")
    x = torch.zeros(plan.numel, dtype=torch.float64, device="cuda")
    with pytest.raises(tds.TdsError) as e:
        plan.deriv(x, out=x)
    assert e.value.status == 3  # alias
    with pytest.raises(tds.TdsError) as e:
        plan.deriv(x, ws=torch.empty(plan.ws_bytes // 2, dtype=torch.uint8, device="cuda"))
    assert e.value.status == 4  # workspace too small
    buf = torch.zeros(plan.numel + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(tds.TdsError) as e:
        plan.deriv(buf[1:])
    assert e.value.status == 1  # misaligned


# ------------------------------------------------------------------------------ reorders

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_reorder_bitwise(dtype):
    shape = (3, 64, 96)
    cart = np.random.default_rng(4).uniform(-1, 1, shape)
    t = torch.from_numpy(cart.reshape(-1).copy()).cuda().to(TORCH[dtype])
    ref_cart = t.cpu().double().numpy().reshape(shape)
    lay = {"cart": t}
    for d in "xyz":
        lay[d] = tds.reorder(t, shape, "cart", d)
        want = oracle.to_layout(ref_cart, d, 32)
        assert np.array_equal(lay[d].cpu().double().numpy(), want), d
    for a in lay:
        for b in lay:
            got = tds.reorder(lay[a], shape, a, b)
            assert torch.equal(got, lay[b]), (a, b)
    # round trip x -> y -> z -> x
    rt = tds.reorder(tds.reorder(tds.reorder(lay["x"], shape, "x", "y"), shape, "y", "z"), shape, "z", "x")
    assert torch.equal(rt, lay["x"])


# --------------------------------------------------------------------- full-size workloads

def sampled_check(field_cart_dev, shape, direction, order, bc, P, dtype, adjoint=False,
                  nsample=48, seed=0, vs_fp64=False):
    """Reorder the device field to the direction layout, run the plan, compare sampled lines
    with the oracle.  Returns (max-rel, rms-rel) against the oracle on the same input; with
    vs_fp64 also (max-rel, rms-rel) against the oracle on the original FP64 field."""
    t = field_cart_dev.to(TORCH[dtype])
    x = tds.reorder(t, shape, "cart", direction)
    del t
    n = {"x": shape[2], "y": shape[1], "z": shape[0]}[direction]
    h = oracle.grid_spacing(n, bc)
    plan = tds.Plan(shape, direction, order, bc, P=P, h=h, dtype=TORCH[dtype])
    y = plan.adjoint(x) if adjoint else plan.deriv(x)
    lines = sample_lines(plan.nlines, nsample, seed)
    fin = gather_lines(x, direction, shape, lines).double().cpu().numpy()
    fout = gather_lines(y, direction, shape, lines).double().cpu().numpy()
    del x, y
    ref = (oracle.deriv_adjoint_lines if adjoint else oracle.deriv_lines)(fin, order, bc, h)
    if not vs_fp64:
        return rel_errors(fout, ref)
    x64 = tds.reorder(field_cart_dev.to(torch.float64), shape, "cart", direction)
    f64 = gather_lines(x64, direction, shape, lines).double().cpu().numpy()
    del x64
    ref64 = (oracle.deriv_adjoint_lines if adjoint else oracle.deriv_lines)(f64, order, bc, h)
    return rel_errors(fout, ref) + rel_errors(fout, ref64)


def test_config_64cubed_fourier_x_periodic_p1():
    shape = (64, 64, 64)
    f, _ = inputs.fourier_field(shape, seed=0, kmax=20, noise=1e-3, device="cuda")
    cart = f.cpu().numpy()
    x = tds.reorder(f, shape, "cart", "x")
    y = tds.Plan(shape, "x", 1, "periodic", P=1).deriv(x)
    got = from_device_layout(y, "x", shape)
    mx, rms = rel_errors(got, oracle.deriv(cart, "x", 1, "periodic"))
    report("64^3 D1 x periodic P=1 f64", max_rel=mx, rms_rel=rms)
    assert mx <= 1e-12, (mx, rms)


@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_config_256cubed_orders_dirs_bcs_p1_p4(direction, bc):
    shape = (256, 256, 256)
    f = inputs.uniform_field(shape, seed=1, device="cuda")
    for order in (1, 2):
        for P in (1, 4):
            mx, rms = sampled_check(f, shape, direction, order, bc, P, "f64", seed=order * 10 + P)
            report("256^3 D%d %s %s P=%d f64" % (order, direction, bc, P), max_rel=mx, rms_rel=rms)
            assert mx <= 1e-12, (order, P, mx, rms)


@pytest.mark.parametrize("direction", ["x", "y", "z"])
def test_config_512cubed_fp32_vs_fp64(direction):
    shape = (512, 512, 512)
    f, _ = inputs.fourier_field(shape, seed=2, kmax=100, noise=0.1, noise_kind="normal",
                                device="cuda")
    for order in (1, 2):
        mx, rms = sampled_check(f, shape, direction, order, "periodic", 8, "f64", nsample=24)
        report("512^3 D%d %s periodic P=8 f64" % (order, direction), max_rel=mx, rms_rel=rms)
        assert mx <= 1e-12, ("f64", order, mx, rms)
        mx, rms, mx64, rms64 = sampled_check(f, shape, direction, order, "periodic", 8, "f32", nsample=24,
                                             vs_fp64=True)
        report("512^3 D%d %s periodic P=8 f32" % (order, direction), max_rel=mx, rms_rel=rms,
               max_rel_vs_fp64_input=mx64, rms_rel_vs_fp64_input=rms64)
        assert mx <= 1e-5, ("f32", order, mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_config_256cubed_adjoint_z_closed_p4(dtype):
    shape = (256, 256, 256)
    g = inputs.normal_field(shape, seed=3, device="cuda")
    res = sampled_check(g, shape, "z", 1, "closed", 4, dtype, adjoint=True, vs_fp64=(dtype == "f32"))
    mx, rms = res[0], res[1]
    extra = dict(max_rel_vs_fp64_input=res[2], rms_rel_vs_fp64_input=res[3]) if dtype == "f32" else {}
    report("256^3 D1^T z closed P=4 %s" % dtype, max_rel=mx, rms_rel=rms, **extra)
    assert mx <= TOL[dtype], (mx, rms)


def test_config_1d_batch_long_lines_p64():
    shape = (1, 256, 262144)
    f = inputs.uniform_field(shape, seed=5, device="cuda")
    mx, rms = sampled_check(f, shape, "x", 1, "periodic", 64, "f64", nsample=6)
    report("256 x 262144 D1 x periodic P=64 f64", max_rel=mx, rms_rel=rms)
    assert mx <= 1e-12, (mx, rms)


@pytest.mark.slow
@pytest.mark.parametrize("P", [8, 2])
def test_config_1024cubed_three_directions(P):
    shape = (1024, 1024, 1024)
    f = inputs.uniform_field(shape, seed=4, device="cuda")
    for direction in "xyz":
        mx, rms = sampled_check(f, shape, direction, 1, "periodic", P, "f64", nsample=16)
        report("1024^3 D1 %s periodic P=%d f64" % (direction, P), max_rel=mx, rms_rel=rms)
        assert mx <= 1e-12, (direction, mx, rms)
    del f
    torch.cuda.empty_cache()


# ------------------------------------------------------------------------- adjoint / autograd

@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_adjoint_dot_product_on_device(bc, dtype):
    shape = (8, 16, 64)
    plan = tds.Plan(shape, "x", 1, bc, P=4, dtype=TORCH[dtype])
    f = inputs.uniform_field(shape, seed=7, device="cuda", dtype=TORCH[dtype]).reshape(-1)
    g = inputs.normal_field(shape, seed=8, device="cuda", dtype=TORCH[dtype]).reshape(-1)
    lhs = torch.dot(plan.deriv(f).double(), g.double())
    rhs = torch.dot(f.double(), plan.adjoint(g).double())
    scale = torch.sum(torch.abs(plan.deriv(f).double() * g.double()))
    assert abs(float(lhs - rhs)) <= (1e-13 if dtype == "f64" else 1e-5) * float(scale)


def test_gradcheck_small_full_jacobian():
    shape = (8, 4, 8)   # z lines: 32, n = 8
    plan = tds.Plan(shape, "z", 1, "closed", P=2)
    x = torch.randn(plan.numel, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: tds.compact_deriv(v, plan), (x,), eps=1e-6,
                                    atol=1e-8, rtol=1e-6)


def test_gradcheck_32cubed_fast_mode():
    shape = (32, 32, 32)
    plan = tds.Plan(shape, "z", 1, "closed", P=4)
    x = torch.randn(plan.numel, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: tds.compact_deriv(v, plan), (x,), eps=1e-6,
                                    atol=1e-7, rtol=1e-6, fast_mode=True)


def test_device_wait_timeout_is_reported_and_context_survives():
    """The bounded-wait failure path: a wait that nothing completes gives up, the status word
    says TDS_ERR_TIMEOUT, and the context keeps working (no trap, no fault)."""
    import ctypes
    from paper_2411_13532_gb300 import _lib
    L = _lib.lib()
    assert tds.device_status() == 0
    assert L.tds_selftest_timeout(ctypes.c_double(0.05), None) == _lib.OK
    assert tds.device_status() == _lib.ERR_TIMEOUT
    assert tds.device_status() == 0          # reading clears it
    assert L.tds_selftest_timeout(ctypes.c_double(5.0), None) == _lib.ERR_ARG
    shape = (1, 32, 64)
    cart = np.random.default_rng(1).uniform(-1, 1, shape)
    y = tds.Plan(shape, "x", 1, "periodic", P=2).deriv(to_device_layout(cart, "x", "f64"))
    mx, _ = rel_errors(from_device_layout(y, "x", shape), oracle.deriv(cart, "x", 1, "periodic"))
    assert mx <= 1e-12


@pytest.mark.parametrize("n", [256, 512, 1024])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_fp32_thin_plans_run_on_finer_chunks(n, bc):
    """AUTO FP32 plans whose one-warp-per-chunk CTAs would be thin run on finer chunks: the same
    operator to rounding.  Every point against the oracle (derivative, adjoint, solve, host entry
    point, fused pass), and a fixed variant keeps the plan's own chunks."""
    shape = (2, 32, n)
    cart = np.random.default_rng(n).uniform(-1, 1, shape).astype(np.float32).astype(np.float64)
    h = oracle.grid_spacing(n, bc)
    auto = tds.Plan(shape, "x", 1, bc, P=1, h=h, dtype=torch.float32)
    fixed = tds.Plan(shape, "x", 1, bc, P=1, h=h, dtype=torch.float32, variant="resident")
    assert auto.variant == "resident" and auto.run_chunks > 1 and fixed.run_chunks == 1
    assert auto.P == 1
    x = to_device_layout(cart, "x", "f32")
    for plan in (auto, fixed):
        mx, _ = rel_errors(from_device_layout(plan.deriv(x), "x", shape), oracle.deriv(cart, "x", 1, bc, h))
        assert mx <= TOL["f32"], (plan.run_chunks, mx)
        mx, _ = rel_errors(from_device_layout(plan.adjoint(x), "x", shape),
                           oracle.deriv_adjoint(cart, "x", 1, bc, h))
        assert mx <= TOL["f32"], (plan.run_chunks, "adjoint", mx)
        lines = oracle.lines_view(cart, "x")
        ref = oracle.from_lines_view(oracle_solve_lines(lines, 1, bc, h), "x", shape)
        mx, _ = rel_errors(from_device_layout(plan.solve(x), "x", shape), ref)
        assert mx <= TOL["f32"], (plan.run_chunks, "solve", mx)
    # host entry point and fused pass run the finer chunks too (bitwise the device call)
    host_out = torch.empty(auto.numel, dtype=torch.float32).pin_memory()
    auto.deriv_host(x.cpu().pin_memory(), host_out, torch.empty_like(x), torch.empty_like(x))
    torch.cuda.current_stream().synchronize()
    assert torch.equal(host_out, auto.deriv(x).cpu())
    d2 = tds.Plan(shape, "x", 2, bc, P=1, h=h, dtype=torch.float32)
    outs = tds.deriv_multi([(auto, False), (d2, False)], x)
    assert torch.equal(outs[0], auto.deriv(x)) and torch.equal(outs[1], d2.deriv(x))


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("direction", ["x", "z"])
def test_fp32_closed_lines_smooth_field_512(order, direction, adjoint):
    """FP32 on closed lines with a smooth field (Fourier modes, kmax 20).  Two things keep the
    usual bar here: the closure and interior taps are applied to differences of nearby values
    (exact on smooth data, where the plain sums of a second derivative cancel 6 to 10 bits), and
    the four closure rows at each end of the line run in FP64 (the closure makes the chunk ends
    ill-conditioned: an error at row 1 reaches row 0 multiplied by about 100).  Sampled whole
    lines, both ends included, against the oracle on the FP32-rounded field."""
    shape = (512, 512, 512)
    f, _ = inputs.fourier_field(shape, seed=6, kmax=20, noise=1e-3, device="cuda")
    mx, rms = sampled_check(f, shape, direction, order, "closed", 8, "f32", adjoint=adjoint, nsample=24)
    report("512^3 D%d%s %s closed P=8 f32 smooth" % (order, "T" if adjoint else "", direction),
           max_rel=mx, rms_rel=rms)
    assert mx <= TOL["f32"], (mx, rms)


@pytest.mark.parametrize("variant", ["resident", "pipelined", "segmented", "streaming"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("adjoint", [False, True])
def test_fp32_closed_smooth_every_variant(variant, order, adjoint):
    """The FP64 closure rows and the difference forms in every FP32 code path (resident,
    persistent pipelined, segment ends, three-kernel streaming): 128 closed lines of 512 points
    of a smooth field, P = 8, every point against the oracle on the FP32-rounded field."""
    shape = (4, 32, 512)
    f, _ = inputs.fourier_field(shape, seed=9, kmax=20, noise=1e-3)
    cart = f.numpy().astype(np.float32).astype(np.float64)
    h = oracle.grid_spacing(512, "closed")
    plan = tds.Plan(shape, "x", order, "closed", P=8, h=h, dtype=torch.float32, variant=variant)
    x = to_device_layout(cart, "x", "f32")
    y = plan.adjoint(x) if adjoint else plan.deriv(x)
    ref = (oracle.deriv_adjoint if adjoint else oracle.deriv)(cart, "x", order, "closed", h)
    mx, rms = rel_errors(from_device_layout(y, "x", shape), ref)
    report("closed smooth D%d%s f32" % (order, "T" if adjoint else ""), variant=plan.variant, max_rel=mx,
           rms_rel=rms)
    assert mx <= TOL["f32"], (mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kind", [1, 2, "interp"])
@pytest.mark.parametrize("fold", ["0", "1"])
def test_closed_adjoint_fold_forms(dtype, kind, fold, monkeypatch):
    """The closed-line adjoint with x = B^T y folded into the back-substitution (chunks of at least
    16 rows; FP32 plans by default) and as a separate pass, both forced through TDS_ADJOINT_FOLD
    (read at plan creation): every point against the oracle, for chunks of 16 to 128 rows in the
    first, interior and last positions (P = 1 has the line's closures at both ends of one chunk)."""
    monkeypatch.setenv("TDS_ADJOINT_FOLD", fold)
    shape = (4, 32, 128)
    cart = np.random.default_rng(41).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    if kind == "interp":
        ref = oracle.apply_op(cart, "x", oracle.INTERP, "closed", adjoint=True)
    else:
        h = oracle.grid_spacing(128, "closed")
        ref = oracle.deriv_adjoint(cart, "x", kind, "closed", h)
    x = to_device_layout(cart, "x", dtype)
    for P in (1, 2, 4, 8):
        for variant in ("resident", "pipelined"):
            if kind == "interp":
                plan = tds.Plan(shape, "x", "interp", "closed", P=P, dtype=TORCH[dtype], variant=variant)
            else:
                plan = tds.Plan(shape, "x", kind, "closed", P=P, h=h, dtype=TORCH[dtype], variant=variant)
            mx, rms = rel_errors(from_device_layout(plan.adjoint(x), "x", shape), ref)
            assert mx <= TOL[dtype], (P, variant, mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("lanes", ["2", "4"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_lines_per_thread_every_point(dtype, lanes, bc, monkeypatch):
    """Two or four lines per thread in the whole-group resident kernels (TDS_RESIDENT_LANES, read at
    plan creation; four lines for FP32 only): every point of the derivatives and their adjoints
    against the oracle, with chunks in the first, interior and last positions."""
    if dtype == "f64" and lanes == "4":
        pytest.skip("four lines per thread are FP32 only")
    monkeypatch.setenv("TDS_RESIDENT_LANES", lanes)
    shape = (4, 64, 128)
    cart = np.random.default_rng(43).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    h = oracle.grid_spacing(128, bc)
    x = to_device_layout(cart, "x", dtype)
    for order in (1, 2):
        for adjoint in (False, True):
            ref = (oracle.deriv_adjoint if adjoint else oracle.deriv)(cart, "x", order, bc, h)
            for P in (1, 2, 4):
                plan = tds.Plan(shape, "x", order, bc, P=P, h=h, dtype=TORCH[dtype], variant="resident", width=32)
                y = plan.adjoint(x) if adjoint else plan.deriv(x)
                mx, rms = rel_errors(from_device_layout(y, "x", shape), ref)
                assert mx <= TOL[dtype], (order, adjoint, P, mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("rows", ["64", "512"])
def test_segment_length_knob_every_point(dtype, rows, monkeypatch):
    """TDS_SEG_ROWS (the longest segment of SEGMENTED plans, read at plan creation) changes the
    internal partition only: every point of long lines against the oracle, both boundaries."""
    monkeypatch.setenv("TDS_SEG_ROWS", rows)
    shape = (1, 32, 4096)
    cart = np.random.default_rng(47).uniform(-1, 1, shape)
    if dtype == "f32":
        cart = cart.astype(np.float32).astype(np.float64)
    x = to_device_layout(cart, "x", dtype)
    for bc in ("periodic", "closed"):
        h = oracle.grid_spacing(4096, bc)
        ref = oracle.deriv(cart, "x", 1, bc, h)
        for P in (1, 4):
            plan = tds.Plan(shape, "x", 1, bc, P=P, h=h, dtype=TORCH[dtype], variant="segmented")
            assert plan.variant == "segmented"
            mx, rms = rel_errors(from_device_layout(plan.deriv(x), "x", shape), ref)
            assert mx <= TOL[dtype], (bc, P, mx, rms)
