"""GPU parity of the transport-equation path (Sec. 5, Eq. mom-comps) against the FP64 oracle.

* ``tds_transport``: one fused term group along each direction, every point, over dtype x
  direction x boundary x (i != j, i = j) x CTA width;
* ``tds_reorder_add``: every layout pair, bit-exact against the oracle's layout maps plus one
  addition in the field's dtype;
* ``TransportRHS``: the whole right-hand side (9 term groups, 6 reorders, 6 accumulations),
  every point on a small box and sampled points (whole lines through them, in each direction)
  at the benchmark's 512^3 size.
Bars as for the derivatives: max|d| / max|ref| <= 1e-12 (FP64), <= 1e-5 (FP32, against the
oracle on the FP32-rounded inputs)."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_util import TOL, TORCH, from_device_layout, rel_errors, report, to_device_layout

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


NU = 0.02


def rand_fields(shape, count, dtype, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        f = rng.uniform(-1, 1, shape)
        if dtype == "f32":
            f = f.astype(np.float32).astype(np.float64)
        out.append(f)
    return out


# (shape, P per direction, width): default width on a grid with ragged group counts, and the
# 16- and 8-line CTAs (2-D TMA tensor boxes) on a grid whose chunks suit them
TERM_CASES = {
    "w_auto": ((20, 64, 96), {"x": 4, "y": 2, "z": 5}, None),
    "w16": ((32, 48, 64), {"x": 4, "y": 4, "z": 4}, 16),
    "w8": ((32, 48, 64), {"x": 8, "y": 12, "z": 8}, 8),
}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("direction", ["x", "y", "z"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("same", [False, True])
@pytest.mark.parametrize("case", sorted(TERM_CASES))
def test_transport_term_every_point(dtype, direction, bc, same, case):
    shape, Ps, width = TERM_CASES[case]
    P = Ps[direction]
    seed = 100 * (dtype == "f32") + 10 * "xyz".index(direction) + 3 * (bc == "closed") + len(case)
    ui, uj = rand_fields(shape, 2, dtype, seed=seed)
    if same:
        uj = ui
    d1 = tds.Plan(shape, direction, 1, bc, P=P, dtype=TORCH[dtype], width=width)
    d2 = tds.Plan(shape, direction, 2, bc, P=P, dtype=TORCH[dtype], width=width)
    if width is not None:
        assert d1.width == width and d2.width == width
    a = to_device_layout(ui, direction, dtype)
    b = a if same else to_device_layout(uj, direction, dtype)
    out = tds.transport_term(d1, d2, a, b, NU)
    torch.cuda.synchronize()
    got = from_device_layout(out, direction, shape)
    ref = oracle.transport_term(ui, uj, direction, NU, bc)
    mx, rms = rel_errors(got, ref)
    report("transport_term", dtype=dtype, direction=direction, bc=bc, same=same, grid=case,
           max_rel=mx, rms_rel=rms)
    assert mx <= TOL[dtype], (mx, rms)


def test_transport_term_argument_rules():
    shape = (20, 64, 96)
    d1 = tds.Plan(shape, "x", 1, "periodic", P=4)
    d2 = tds.Plan(shape, "x", 2, "periodic", P=4)
    d2p = tds.Plan(shape, "x", 2, "periodic", P=2)
    d2y = tds.Plan(shape, "y", 2, "periodic", P=2)
    d2f = tds.Plan(shape, "x", 2, "periodic", P=4, dtype=torch.float32)
    u = torch.rand(d1.numel, dtype=torch.float64, device="cuda")
    v = torch.rand(d1.numel, dtype=torch.float64, device="cuda")
    L = tds._lib.lib()
    import ctypes

    def call(a, b, ui, uj, out):
        return L.tds_transport(a._handle, b._handle, ctypes.c_void_p(ui.data_ptr()),
                               ctypes.c_void_p(uj.data_ptr()), NU, ctypes.c_void_p(out.data_ptr()), None)
    out = torch.empty_like(u)
    assert call(d2, d1, u, v, out) == tds._lib.ERR_ARG      # orders swapped
    assert call(d1, d2p, u, v, out) == tds._lib.ERR_ARG     # different chunks
    assert call(d1, d2y, u, v, out) == tds._lib.ERR_ARG     # different direction
    assert call(d1, d2f, u, v, out) == tds._lib.ERR_ARG     # different dtype
    assert call(d1, d2, u, v, u) == tds._lib.ERR_ALIAS      # out overwrites ui
    assert call(d1, d2, u, v, v) == tds._lib.ERR_ALIAS      # out overwrites uj
    assert call(d1, d2, u, v, out) == tds._lib.OK
    torch.cuda.synchronize()


LAYS = ["cart", "x", "y", "z"]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("src", LAYS)
@pytest.mark.parametrize("dst", LAYS)
def test_reorder_add_bit_exact(dtype, src, dst):
    shape = (5, 64, 96)
    rng = np.random.default_rng(7)
    npdt = np.float64 if dtype == "f64" else np.float32
    cart = rng.uniform(-1, 1, shape).astype(npdt)
    acc = rng.uniform(-1, 1, cart.size).astype(npdt)

    def lay(c, name):
        return c.reshape(-1) if name == "cart" else oracle.to_layout(c, name, 32).astype(npdt)
    x = torch.from_numpy(np.ascontiguousarray(lay(cart, src))).cuda()
    out = torch.from_numpy(acc.copy()).cuda()
    tds.reorder_add(x, shape, src, dst, out)
    torch.cuda.synchronize()
    want = acc + lay(cart, dst)            # one IEEE addition in the field's dtype
    assert np.array_equal(out.cpu().numpy(), want)


def rhs_case(shape, Ps, bc, dtype, seed):
    u = rand_fields(shape, 3, dtype, seed)
    rhs = tds.TransportRHS(shape, P=(Ps["x"], Ps["y"], Ps["z"]), bc=bc, dtype=TORCH[dtype])
    dev = [to_device_layout(f, "x", dtype) for f in u]
    out = rhs(dev, NU)
    torch.cuda.synchronize()
    got = [from_device_layout(o, "x", shape) for o in out]
    ref = oracle.transport_rhs(u, NU, bc)
    return got, ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_transport_rhs_every_point(dtype, bc):
    shape, Ps, _ = TERM_CASES["w_auto"]
    got, ref = rhs_case(shape, Ps, bc, dtype, seed=5)
    for i in range(3):
        mx, rms = rel_errors(got[i], ref[i])
        report("transport_rhs", dtype=dtype, bc=bc, component=i, max_rel=mx, rms_rel=rms)
        assert mx <= TOL[dtype], (i, mx, rms)


def test_transport_rhs_reuse_and_i_equals_j_layout():
    """Two calls on one object give identical results (the temporaries are fully rewritten), and
    a velocity field constant in y and z reduces the y and z terms to zero."""
    shape = (20, 64, 96)
    rhs = tds.TransportRHS(shape, P=(4, 2, 5))
    u = rand_fields(shape, 3, "f64", seed=9)
    dev = [to_device_layout(f, "x", "f64") for f in u]
    a = [t.clone() for t in rhs(dev, NU)]
    b = rhs(dev, NU)
    assert all(torch.equal(p, q) for p, q in zip(a, b))
    # fields that vary along x only: the y and z derivatives vanish (rows of A^{-1} B sum to 0)
    x = np.arange(shape[2]) * 2 * np.pi / shape[2]
    ux = [np.broadcast_to(np.cos(k * x + k)[None, None, :], shape).copy() for k in (1, 2, 3)]
    devx = [to_device_layout(f, "x", "f64") for f in ux]
    out = rhs(devx, NU)
    ref = [oracle.transport_term(ux[i], ux[0], "x", NU, "periodic") for i in range(3)]
    for i in range(3):
        mx, _ = rel_errors(from_device_layout(out[i], "x", shape), ref[i])
        assert mx <= TOL["f64"]


FULL = (512, 512, 512)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc,field", [("periodic", "fourier"), ("closed", "fourier"), ("closed", "uniform")])
def test_transport_rhs_full_size_sampled(dtype, bc, field):
    """The benchmark's workload (512^3, P = 8; periodic, and closed lines too): the right-hand
    side at sampled points, each from the whole x, y and z lines through the point (the oracle
    on lines), the box's corners and faces included."""
    from paper_2411_13532_gb300 import inputs
    shape = FULL
    rhs = tds.TransportRHS(shape, P=8, bc=bc, dtype=TORCH[dtype])
    if field == "fourier":   # smooth velocity components: a few 3D Fourier modes plus small noise
        u = [inputs.fourier_field(shape, seed=21 + c, device="cuda", dtype=TORCH[dtype])[0].reshape(-1)
             for c in range(3)]
    else:                    # i.i.d. U(-1, 1), as the closed-line derivative configurations use
        u = [inputs.uniform_field(shape, seed=21 + c, device="cuda", dtype=TORCH[dtype]).reshape(-1)
             for c in range(3)]
    ux = [tds.reorder(f, shape, "cart", "x") for f in u]
    out = rhs(ux, NU)
    outc = [tds.reorder(o, shape, "x", "cart").view(shape) for o in out]
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    pts = [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(24)] + [
        (0, 0, 0), (511, 511, 511), (1, 510, 2), (255, 0, 511), (3, 3, 508)]
    cu = [f.view(shape) for f in u]
    n = 512
    worst = 0.0
    for (z, y, x) in pts:
        lines = {"x": [f[z, y, :] for f in cu], "y": [f[z, :, x] for f in cu], "z": [f[:, y, x] for f in cu]}
        pos = {"x": x, "y": y, "z": z}
        h = oracle.grid_spacing(n, bc)
        for i in range(3):
            val = 0.0
            for j, d in enumerate("xyz"):
                li = lines[d][i].double().cpu().numpy()[None, :]
                lj = lines[d][j].double().cpu().numpy()[None, :]
                val += oracle.transport_term_lines(li, lj, NU, bc, h)[0, pos[d]]
            got = float(outc[i][z, y, x])
            worst = max(worst, abs(got - val))
    # normwise scale: the largest |rhs| over the sampled lines' terms
    scale = max(float(o.abs().max()) for o in outc)
    report("transport_rhs_512", dtype=dtype, bc=bc, field=field, max_rel=worst / scale)
    assert worst / scale <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_transport_rhs_host_entry_matches_device_call(dtype):
    """call_host (pinned host in and out, copies overlapped with the kernels) gives bitwise the
    results of the device call, on two calls in a row (the device buffers are reused)."""
    shape = (20, 64, 96)
    rhs = tds.TransportRHS(shape, P=(4, 2, 5), dtype=TORCH[dtype])
    t = TORCH[dtype]
    for seed in (1, 2):
        u = rand_fields(shape, 3, dtype, seed=seed)
        dev = [to_device_layout(f, "x", dtype) for f in u]
        want = [o.cpu() for o in rhs(dev, NU)]
        hu = [torch.empty(d.numel(), dtype=t, pin_memory=True) for d in dev]
        for h, d in zip(hu, dev):
            h.copy_(d)
        ho = [torch.empty(d.numel(), dtype=t, pin_memory=True) for d in dev]
        ud = [torch.empty_like(d) for d in dev]
        od = [torch.empty_like(d) for d in dev]
        rhs.call_host(hu, ho, NU, ud, od)
        torch.cuda.current_stream().synchronize()
        for a, b in zip(ho, want):
            assert torch.equal(a, b)
    with pytest.raises(ValueError):
        rhs.call_host([torch.empty(5)] * 3, ho, NU, ud, od)


def test_transport_rhs_fp32_with_finer_chunk_plans():
    """FP32 x lines of 512 points with P = 1 run on finer chunks (AUTO); the transport term
    kernel follows the plans' choice: every point against the oracle."""
    shape = (8, 32, 512)
    rhs = tds.TransportRHS(shape, P=(1, 1, 2), dtype=torch.float32)
    assert rhs.d1["x"].run_chunks > 1 and rhs.d1["x"].run_chunks == rhs.d2["x"].run_chunks
    u = rand_fields(shape, 3, "f32", seed=4)
    out = rhs([to_device_layout(f, "x", "f32") for f in u], NU)
    ref = oracle.transport_rhs(u, NU, "periodic")
    for i in range(3):
        mx, rms = rel_errors(from_device_layout(out[i], "x", shape), ref[i])
        assert mx <= TOL["f32"], (i, mx, rms)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_transport_rhs_cuda_graph_replay(dtype):
    """One evaluation captured as a CUDA graph replays to bitwise the eager results, also after
    the inputs change in place."""
    shape = (20, 64, 96)
    rhs = tds.TransportRHS(shape, P=(4, 2, 5), dtype=TORCH[dtype])
    u = [to_device_layout(f, "x", dtype) for f in rand_fields(shape, 3, dtype, seed=12)]
    out = [torch.empty_like(t) for t in u]
    g = rhs.graph(u, NU, out)
    for seed in (13, 14):
        for t, f in zip(u, rand_fields(shape, 3, dtype, seed=seed)):
            t.copy_(to_device_layout(f, "x", dtype))
        g.replay()
        torch.cuda.synchronize()
        want = [o.clone() for o in rhs(u, NU)]
        assert all(torch.equal(a, b) for a, b in zip(out, want))
