"""Seeded synthetic catalogs shaped like the paper's halo samples (inputs only).

The paper measures halo catalogs from N-body boxes (Sec. 3) and 50x random
catalogs (Sec. 4); none of those data are available, so every input here is a
seeded stand-in.  This module holds none of the estimator's arithmetic: it only
draws point positions and weights.

Positions are returned in the canonical fixed-point form used by both the CUDA
path and the CPU oracle: a coordinate x in [0, L) is the unsigned 32-bit
integer u = floor(x / L * 2^32), so one unit is L / 2^32.  Uniform draws are made
directly in that integer form; continuous draws are quantised with the floor
rule in float64.

Recipes (stated once, reused by tests and the benchmark):

* ``poisson``: N points uniform in the cube (integers uniform in [0, 2^32)).
* ``lognormal``: a Gaussian field G on an n^3 mesh with spectrum
  P_G(k) ~ k^slope exp(-(k/k_cut)^2), rescaled to standard deviation sigma_G;
  delta = exp(G - sigma_G^2/2) - 1; exactly N mesh cells drawn with probability
  proportional to (1 + delta) (inverse-CDF sampling), positions uniform inside
  each drawn cell; then a Kaiser-like shift along the line of sight z by
  f * Psi_z, with the Zel'dovich displacement Psi(k) = i k / k^2 G(k) read at
  the drawn cell, wrapped back into [0, L).
* ``randoms``: uniform points (as ``poisson``) with unit weights.

The lognormal generator runs on any torch device; the same seed on the same
device and torch build gives the same catalog.
"""
from __future__ import annotations

import math

import numpy as np
import torch

TWO32 = 4294967296.0


def poisson(n: int, seed: int):
    """Uniform catalog: (xyz uint32 [n,3], w float32 [n]) with unit weights."""
    rng = np.random.default_rng(seed)
    xyz = rng.integers(0, 2**32, size=(n, 3), dtype=np.uint32)
    return xyz, np.ones(n, dtype=np.float32)


def randoms(n: int, seed: int):
    """Unclustered random catalog with unit weights (same draw as ``poisson``)."""
    return poisson(n, seed)


def quantize(x: np.ndarray, box: float) -> np.ndarray:
    """Float positions in [0, box) -> uint32 fixed point, u = floor(x / box * 2^32)."""
    u = np.floor(np.asarray(x, dtype=np.float64) / box * TWO32)
    return np.clip(u, 0, TWO32 - 1).astype(np.uint32)


def lognormal_positions(n: int, box: float, seed: int, mesh: int = 256,
                        slope: float = -1.5, k_cut: float = 0.5,
                        sigma_g: float = 1.0, f_rsd: float = 0.8,
                        device: str | torch.device = "cpu") -> torch.Tensor:
    """Float64 positions [n, 3] in [0, box) of a seeded lognormal catalog."""
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    white = torch.randn((mesh, mesh, mesh), generator=gen, device=dev, dtype=torch.float32)
    wk = torch.fft.rfftn(white)
    del white
    kf = 2.0 * math.pi / box
    kx = torch.fft.fftfreq(mesh, d=1.0 / mesh, device=dev, dtype=torch.float32) * kf
    kz = torch.fft.rfftfreq(mesh, d=1.0 / mesh, device=dev, dtype=torch.float32) * kf
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    pos = k2 > 0
    amp = torch.where(pos, k2.clamp_min(1e-30) ** (slope / 4.0)
                      * torch.exp(-0.5 * k2 / (k_cut * k_cut)), torch.zeros_like(k2))
    gk = wk * amp
    del wk, amp
    field = torch.fft.irfftn(gk, s=(mesh, mesh, mesh))
    scale = sigma_g / field.std()
    field = field * scale
    gk = gk * scale
    one_plus_delta = torch.exp(field - 0.5 * sigma_g * sigma_g)
    del field
    # Zel'dovich displacement along z: Psi_z(k) = i k_z / k^2 G(k)
    psi_k = torch.where(pos, 1j * kz[None, None, :] / k2.clamp_min(1e-30), torch.zeros_like(k2)) * gk
    del gk, k2, pos
    psi_z = torch.fft.irfftn(psi_k, s=(mesh, mesh, mesh))
    del psi_k
    cum = torch.cumsum(one_plus_delta.reshape(-1).to(torch.float64), 0)
    del one_plus_delta
    u = torch.rand(n, generator=gen, device=dev, dtype=torch.float64) * cum[-1]
    idx = torch.searchsorted(cum, u).clamp_max(mesh ** 3 - 1)
    del cum, u
    cell = box / mesh
    ix = idx // (mesh * mesh)
    iy = (idx // mesh) % mesh
    iz = idx % mesh
    off = torch.rand((n, 3), generator=gen, device=dev, dtype=torch.float64)
    x = (ix.to(torch.float64) + off[:, 0]) * cell
    y = (iy.to(torch.float64) + off[:, 1]) * cell
    z = (iz.to(torch.float64) + off[:, 2]) * cell
    z = z + f_rsd * psi_z.reshape(-1)[idx].to(torch.float64)
    z = torch.remainder(z, box)
    out = torch.stack([x, y, z], dim=1)
    return torch.where(out >= box, out - box, out)


def lognormal(n: int, box: float, seed: int, mesh: int = 256, **kw):
    """Lognormal catalog as (xyz uint32 [n,3], w float32 [n]) with unit weights."""
    p = lognormal_positions(n, box, seed, mesh=mesh, **kw).cpu().numpy()
    return quantize(p, box), np.ones(n, dtype=np.float32)


def lognormal_device(n: int, box: float, seed: int, mesh: int = 256, device="cuda", **kw):
    """Lognormal catalog made on ``device``: (xyz int32 bit patterns [n,3], w float32 [n])."""
    p = lognormal_positions(n, box, seed, mesh=mesh, device=device, **kw)
    u = torch.floor(p / box * TWO32).clamp_(0, TWO32 - 1).to(torch.int64)
    u = torch.where(u >= 2**31, u - 2**32, u).to(torch.int32)
    return u.contiguous(), torch.ones(n, dtype=torch.float32, device=p.device)


def mock_sizes(n_mocks: int, n_lo: int, n_hi: int, seed: int) -> np.ndarray:
    """Uneven mock sizes drawn uniformly in [n_lo, n_hi] (the covariance batch)."""
    rng = np.random.default_rng(seed)
    return rng.integers(n_lo, n_hi + 1, size=n_mocks).astype(np.int64)


def as_int32_bits(xyz: np.ndarray) -> np.ndarray:
    """View uint32 coordinates as int32 bit patterns (torch has no uint32 kernels)."""
    return np.ascontiguousarray(xyz, dtype=np.uint32).view(np.int32)
