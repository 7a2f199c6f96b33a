"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the derivative method: it only draws random fields
and evaluates sums of Fourier modes on a uniform periodic grid.  Nothing here is used
to compute an expected value.

Recipes (the workloads of the paper's Sec. 5 are batches of lines of a 3D field; the
paper prints no field, so these stand in for it):
  * ``fourier_field``: sum of ``n_modes`` modes A_m cos(kx x + ky y + kz z + phi_m),
    integer wavenumbers k ~ U{1..kmax} per direction, A_m ~ U(-1,1), phi_m ~ U(0, 2 pi),
    nodes x_i = 2 pi i / nx (likewise y, z), plus noise drawn last: ``noise`` * U(-1,1)
    or N(0, ``noise``).
  * ``uniform_field``: i.i.d. U(-1,1).
  * ``normal_field``: i.i.d. N(0,1).
  * ``diffusion_band``: a variable-coefficient tridiagonal band (implicit diffusion on a
    stretched grid), the input of the batched solve.
Mode parameters come from ``numpy.random.default_rng(seed)``; bulk random numbers come
from a ``torch.Generator`` seeded with ``seed`` on the target device (CPU and CUDA
generators give different streams, so a field is generated once and then copied).
"""
import math

import numpy as np
import torch


def fourier_modes(seed, n_modes=4, kmax=20):
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=(n_modes, 3))
    amp = rng.uniform(-1.0, 1.0, size=n_modes)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    return k, amp, phase


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def fourier_field(shape, seed, n_modes=4, kmax=20, noise=1e-3, noise_kind="uniform",
                  device="cpu", dtype=torch.float64):
    """Cartesian field of shape (nz, ny, nx); returns (field, (k, amp, phase))."""
    nz, ny, nx = shape
    k, amp, phase = fourier_modes(seed, n_modes, kmax)
    x = torch.arange(nx, device=device, dtype=torch.float64) * (2.0 * math.pi / nx)
    y = torch.arange(ny, device=device, dtype=torch.float64) * (2.0 * math.pi / ny)
    z = torch.arange(nz, device=device, dtype=torch.float64) * (2.0 * math.pi / nz)
    f = torch.zeros(shape, device=device, dtype=torch.float64)
    for m in range(n_modes):
        arg = (float(k[m, 0]) * x[None, None, :] + float(k[m, 1]) * y[None, :, None]
               + float(k[m, 2]) * z[:, None, None] + float(phase[m]))
        f += float(amp[m]) * torch.cos(arg)
        del arg
    if noise:
        g = _gen(seed, device)
        if noise_kind == "uniform":
            f += noise * (torch.rand(shape, generator=g, device=device, dtype=torch.float64)
                          * 2.0 - 1.0)
        elif noise_kind == "normal":
            f += noise * torch.randn(shape, generator=g, device=device, dtype=torch.float64)
        else:
            raise ValueError(noise_kind)
    return f.to(dtype), (k, amp, phase)


def diffusion_band(n, seed, dmax=100.0):
    """A variable-coefficient tridiagonal band (a, b, c), numpy arrays of n entries: one
    backward-Euler step of d/dx (kappa d/dx) on a tanh-stretched grid of n cells (faces clustered
    at both ends), kappa(x) = 1 + 0.8 sin(3 x + phase) with a seeded phase, the step chosen so
    that the largest dt kappa / dx^2 is ``dmax``: the implicit system of an ADI sweep, a[i] x[i-1]
    + b[i] x[i] + c[i] x[i+1] = d[i] (b = 1 + the two couplings: diagonally dominant by 1)."""
    rng = np.random.default_rng(seed)
    s = np.linspace(0.0, 1.0, n + 1)
    x = np.tanh(2.0 * (s - 0.5)) / np.tanh(1.0)
    dxf = np.diff(x)
    xc = 0.5 * (x[1:] + x[:-1])
    kappa = 1.0 + 0.8 * np.sin(3.0 * xc + rng.uniform(0.0, 2.0 * math.pi))
    kf = 0.5 * (kappa + np.roll(kappa, -1))
    dxc = 0.5 * (dxf + np.roll(dxf, -1))
    gp = kf / (dxc * dxf)
    gm = np.roll(kf, 1) / (np.roll(dxc, 1) * dxf)
    dt = dmax / max(gp.max(), gm.max())
    gp, gm = dt * gp, dt * gm
    return -gm, 1.0 + gm + gp, -gp


def uniform_field(shape, seed, device="cpu", dtype=torch.float64):
    g = _gen(seed, device)
    return (torch.rand(shape, generator=g, device=device, dtype=torch.float64) * 2.0
            - 1.0).to(dtype)


def normal_field(shape, seed, device="cpu", dtype=torch.float64):
    g = _gen(seed, device)
    return torch.randn(shape, generator=g, device=device, dtype=torch.float64).to(dtype)
