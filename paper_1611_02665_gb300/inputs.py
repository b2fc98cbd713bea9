"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random-number recipes only, none of the method's
arithmetic, so that the oracle and the CUDA path can both be fed from it.
Recipes (the paper publishes no data; its miniQMC driver draws random
positions, Sec. "Baseline and miniQMC", Fig. (alg:bspline_thd)):

* ``uniform_coefs``: periodic table [nx][ny][nz][N], float32 uniform in [-1, 1].
* ``plane_wave_coefs``: smooth periodic orbitals, per orbital a sum of
  ``nmodes`` cosines with integer wavevectors in [-kmax, kmax]^3, amplitudes
  uniform in [-1, 1] / sqrt(nmodes), phases uniform in [0, 2 pi), plus
  ``noise`` * uniform[-1, 1] per coefficient.
* ``uniform_positions``: fractional coordinates uniform in [0, 1)^3, float64.
* ``batched_workload``: several tables of uneven N and grid, each with a set
  of walkers holding 1..8 positions.

numpy's PCG64 drives everything drawn on the host; the plane-wave noise is
drawn with a torch generator on the device that builds the table.
"""
from __future__ import annotations

import math

import numpy as np


def uniform_coefs(grid, N, seed):
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(nx, ny, nz, N)).astype(np.float32)


def uniform_coefs_device(grid, N, seed, device="cuda"):
    """Like uniform_coefs but drawn on ``device`` with a seeded torch generator (large tables)."""
    import torch

    nx, ny, nz = grid
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 7919 + 5)
    t = torch.empty((nx, ny, nz, N), dtype=torch.float32, device=device)
    t.uniform_(-1.0, 1.0, generator=gen)
    return t


def uniform_positions(npos, seed):
    rng = np.random.default_rng(seed)
    r = rng.random((3, npos))
    return r[0].copy(), r[1].copy(), r[2].copy()


def plane_wave_params(N, seed, nmodes=32, kmax=4):
    rng = np.random.default_rng(seed)
    k = rng.integers(-kmax, kmax + 1, size=(N, nmodes, 3))
    amp = rng.uniform(-1.0, 1.0, size=(N, nmodes)) / math.sqrt(nmodes)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=(N, nmodes))
    return k, amp, theta


def plane_wave_coefs(grid, N, seed, device="cpu", nmodes=32, kmax=4, noise=1e-3, chunk=256):
    """float32 torch tensor [nx][ny][nz][N] on ``device``.

    p[i,j,k,n] = sum_m a_nm cos(2 pi (kx i/nx + ky j/ny + kz k/nz) + theta_nm) + noise * xi.
    Evaluated as the real part of a rank-``nmodes`` product of three 1-D
    complex exponentials, ``chunk`` orbitals at a time.
    """
    import torch

    nx, ny, nz = grid
    k, amp, theta = plane_wave_params(N, seed, nmodes, kmax)
    dev = torch.device(device)
    out = torch.empty((nx, ny, nz, N), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 1000003 + 17)
    axes = [torch.arange(m, dtype=torch.float64, device=dev) / m for m in (nx, ny, nz)]
    for n0 in range(0, N, chunk):
        n1 = min(N, n0 + chunk)
        kk = torch.as_tensor(k[n0:n1], dtype=torch.float64, device=dev)
        c = torch.as_tensor(amp[n0:n1], device=dev) * torch.exp(
            1j * torch.as_tensor(theta[n0:n1], device=dev))
        ex = [torch.exp(2j * math.pi * kk[:, :, d, None] * axes[d][None, None, :]) for d in range(3)]
        xy = (c[:, :, None, None] * ex[0][:, :, :, None] * ex[1][:, :, None, :])  # [n, m, i, j]
        nc = n1 - n0
        t = torch.bmm(xy.reshape(nc, nmodes, nx * ny).transpose(1, 2).to(torch.complex64),
                      ex[2].to(torch.complex64))  # [n, ij, k]
        blk = t.real.reshape(nc, nx, ny, nz).permute(1, 2, 3, 0)
        xi = torch.rand((nx, ny, nz, nc), generator=gen, device=dev, dtype=torch.float32) * 2.0 - 1.0
        out[..., n0:n1] = blk.to(torch.float32) + noise * xi
    return out


def batched_workload(seed, tables=((256, 32), (512, 40), (1024, 48), (2048, 56), (4096, 64)),
                     walkers=(64, 256, 512, 1024, 2048), max_pos_per_walker=8):
    """Per table: (N, grid, walker_offsets CSR int32, npos). Positions per walker uniform in 1..8."""
    rng = np.random.default_rng(seed)
    out = []
    for (N, g), nw in zip(tables, walkers):
        counts = rng.integers(1, max_pos_per_walker + 1, size=nw)
        offs = np.zeros(nw + 1, dtype=np.int32)
        offs[1:] = np.cumsum(counts)
        out.append({"N": N, "grid": (g, g, g), "walker_offsets": offs, "npos": int(offs[-1])})
    return out
