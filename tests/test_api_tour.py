"""A tour of the public API on a small grid (GPU): every entry point a user starts with runs
and agrees with the others."""
import pytest
import torch

pytestmark = pytest.mark.gpu

tds = pytest.importorskip("paper_2411_13532_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_13532_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_api_tour():
    shape = (64, 64, 64)
    f = torch.rand(shape, dtype=torch.float64, device="cuda")
    fx = tds.reorder(f.reshape(-1), shape, "cart", "x")
    d1 = tds.Plan(shape, "x", 1, "periodic", P=8)
    d2 = tds.Plan(shape, "x", 2, "periodic", P=8)
    y = d1.deriv(fx)
    g = d1.adjoint(fx)
    y1, y2, y1t = tds.deriv_multi([(d1, False), (d2, False), (d1, True)], fx)
    assert torch.equal(y1, y) and torch.equal(y1t, g) and torch.equal(y2, d2.deriv(fx))
    x = d1.solve(fx)
    # A x = f with A = tridiag(1/3, 1, 1/3), cyclic: the residual vanishes to rounding
    X = x.reshape(-1, 64, 32)
    F = fx.reshape(-1, 64, 32)
    R = (torch.roll(X, 1, dims=1) + torch.roll(X, -1, dims=1)) / 3.0 + X - F
    assert R.abs().max().item() <= 1e-12 * F.abs().max().item()
    u = torch.rand(d1.numel, dtype=torch.float64, device="cuda", requires_grad=True)
    du = tds.compact_deriv(u, d1)
    du.sum().backward()
    assert torch.allclose(u.grad, d1.adjoint(torch.ones_like(u)))
    a, b, c = (torch.full((64,), v, dtype=torch.float64) for v in (-0.25, 1.5, -0.25))
    adi = tds.Plan(shape, "x", 0, "periodic", P=8, band=(a, b, c))
    xa = adi.solve(fx)
    # residual of the band system, line by line in the interleaved layout (x lines: row j of
    # group g at j*32 + lane): a x_{j-1} + b x_j + c x_{j+1} = f_j with cyclic wrap
    X = xa.reshape(-1, 64, 32)
    F = fx.reshape(-1, 64, 32)
    R = -0.25 * torch.roll(X, 1, dims=1) + 1.5 * X - 0.25 * torch.roll(X, -1, dims=1) - F
    assert R.abs().max().item() <= 1e-13 * F.abs().max().item() * 10
    assert tds.device_status() == 0
