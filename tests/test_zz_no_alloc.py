"""tds_deriv_noalloc: the derivative for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (or any allocator): the library then uses its built-in
scratch array instead of a caller workspace.  This file checks, through the C ABI, two calls in
a row with different inputs: every point against the FP64 oracle (on the same, FP32-rounded
where the plan is FP32, field), and against the ordinary tds_deriv with its workspace; and that
a plan too large for the built-in scratch is refused before any launch.  It is named to run
last so that a failure here does not stop the other tests from running first.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

SZ = 32


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_13532_gb300 import build, _lib
    build.build()
    oracle.build()
    return _lib.lib()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dtype,bc,order,P,shape,tol", [
    (torch.float64, "periodic", 1, 4, (8, 64, 256), 1e-12),
    (torch.float64, "closed", 2, 8, (8, 64, 256), 1e-12),
    (torch.float32, "periodic", 1, 2, (8, 64, 256), 1e-5),
    # FP32, P = 1 on 512-point lines: tds_deriv runs such an AUTO plan on finer chunks, the
    # allocation-free call on the plan's own single chunk
    (torch.float32, "closed", 2, 1, (4, 32, 512), 1e-5),
])
def test_noalloc_against_oracle_on_two_calls(L, dtype, bc, order, P, shape, tol):
    import paper_2411_13532_gb300 as tds
    from paper_2411_13532_gb300 import _lib
    n = shape[2]
    h = oracle.grid_spacing(n, bc)
    plan = tds.Plan(shape, "x", order, bc, P=P, h=h, dtype=dtype)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):                      # two calls in a row, different inputs
        cart = np.random.default_rng(100 + call).uniform(-1, 1, shape)
        if dtype == torch.float32:
            cart = cart.astype(np.float32).astype(np.float64)
        x = torch.from_numpy(oracle.to_layout(cart, "x", SZ)).to(device="cuda", dtype=dtype)
        got = torch.full_like(x, float("nan"))
        st = L.tds_deriv_noalloc(plan._handle, _ptr(x), _ptr(got), stream)
        assert st == _lib.OK, _lib.status_string(st)
        ref = torch.empty_like(x)
        ws = plan.workspace()
        st = L.tds_deriv(plan._handle, _ptr(x), _ptr(ref), _ptr(ws) if ws is not None else None,
                         ws.numel() if ws is not None else 0, stream)
        assert st == _lib.OK
        torch.cuda.synchronize()
        g = oracle.from_layout(got.double().cpu().numpy(), "x", shape, SZ)
        assert np.all(np.isfinite(g))
        expect = oracle.deriv(cart, "x", order, bc, h)
        scale = np.max(np.abs(expect))
        assert np.max(np.abs(g - expect)) <= tol * scale, ("oracle", call)
        r = oracle.from_layout(ref.double().cpu().numpy(), "x", shape, SZ)
        assert np.max(np.abs(g - r)) <= tol * scale, ("tds_deriv", call)
    assert tds.device_status() == 0


def test_noalloc_rejects_plans_beyond_the_scratch(L):
    import paper_2411_13532_gb300 as tds
    from paper_2411_13532_gb300 import _lib
    # N * P * 16 bytes = 131072 * 16 * 16 = 32 MiB > 16 MiB of built-in scratch
    shape = (256, 512, 64)                      # x lines: 131072, n = 64
    plan = tds.Plan(shape, "x", 1, "periodic", P=16)
    x = torch.zeros(plan.numel, device="cuda", dtype=torch.float64)
    out = torch.zeros_like(x)
    st = L.tds_deriv_noalloc(plan._handle, _ptr(x), _ptr(out), None)
    assert st == _lib.ERR_WORKSPACE
    assert L.tds_deriv_noalloc(plan._handle, _ptr(x), _ptr(x), None) == _lib.ERR_ALIAS
