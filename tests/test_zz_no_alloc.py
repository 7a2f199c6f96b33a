"""tds_deriv_noalloc: the derivative for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (or any allocator): the library then uses its built-in
scratch array instead of a caller workspace.  This file checks, through the C ABI, that two
calls in a row give the same result as the ordinary tds_deriv (with its workspace), and that
a plan too large for the built-in scratch is refused before any launch.  It is named to run
last so that a failure here does not stop the other tests from running first.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_13532_gb300 import build, _lib
    build.build()
    return _lib.lib()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dtype,bc,order,P,tol", [
    (torch.float64, "periodic", 1, 4, 1e-12),
    (torch.float64, "closed", 2, 8, 1e-12),
    (torch.float32, "periodic", 1, 2, 1e-5),
])
def test_noalloc_matches_tds_deriv_on_two_calls(L, dtype, bc, order, P, tol):
    import paper_2411_13532_gb300 as tds
    from paper_2411_13532_gb300 import _lib
    shape = (8, 64, 256)                       # x lines: 512, n = 256
    plan = tds.Plan(shape, "x", order, bc, P=P, dtype=dtype)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda")
    for call in range(2):                      # two calls in a row, different inputs
        gen.manual_seed(100 + call)
        x = (torch.rand(plan.numel, generator=gen, device="cuda", dtype=torch.float64) * 2 - 1).to(dtype)
        ref = torch.empty_like(x)
        ws = plan.workspace()
        st = L.tds_deriv(plan._handle, _ptr(x), _ptr(ref), _ptr(ws) if ws is not None else None,
                         ws.numel() if ws is not None else 0, stream)
        assert st == _lib.OK
        got = torch.full_like(x, float("nan"))
        st = L.tds_deriv_noalloc(plan._handle, _ptr(x), _ptr(got), stream)
        assert st == _lib.OK, _lib.status_string(st)
        torch.cuda.synchronize()
        r = ref.double().cpu().numpy(); g = got.double().cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) <= tol * np.max(np.abs(r)), call
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
