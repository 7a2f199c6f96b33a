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


def uniform_field(shape, seed, device="cpu", dtype=torch.float64):
    g = _gen(seed, device)
    return (torch.rand(shape, generator=g, device=device, dtype=torch.float64) * 2.0
            - 1.0).to(dtype)


def normal_field(shape, seed, device="cpu", dtype=torch.float64):
    g = _gen(seed, device)
    return torch.randn(shape, generator=g, device=device, dtype=torch.float64).to(dtype)
