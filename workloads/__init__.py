"""Seeded synthetic initial fields for the TVLBM workloads.

This module only draws and shapes input data (density, velocity and
temperature fields on the cell centres).  It holds none of the method's
arithmetic: no equilibrium, no streaming, no moments.  Both the FP64 oracle
and the CUDA path receive exactly these arrays, so their inputs are identical.

All fields are float64 numpy arrays of shape (ny, nx), x fastest, cell (i, j)
centred at (i, j) in lattice units (dx = dy = 1).

Workload shapes follow the paper's test problems (Sec. "Measuring the
transport coefficients": sinusoidal shear and thermal modes of amplitude
0.01; Sec. "Avoiding temperature and velocity slip": thermal Couette flow
between walls at different temperatures and velocities), scaled to the
lattice sizes the library is measured on.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "shear_wave",
    "heat_mode",
    "gaussian_bump_random_flow",
    "couette_linear",
    "random_smooth",
    "batched_domains",
]


def _grid(nx: int, ny: int):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def shear_wave(nx: int, ny: int, eps: float = 0.01, rho0: float = 1.0, T0: float = 1.0):
    """Transverse shear wave u_x = eps sin(2 pi y / ny), u_y = 0, uniform rho and T."""
    _, y = _grid(nx, ny)
    rho = np.full((ny, nx), rho0)
    ux = eps * np.sin(2.0 * np.pi * y / ny)
    uy = np.zeros((ny, nx))
    T = np.full((ny, nx), T0)
    return rho, ux, uy, T


def heat_mode(nx: int, ny: int, eps: float = 0.01, p0: float = 1.0):
    """Thermal diffusion mode at uniform pressure: T = 1 + eps sin(2 pi y/ny), rho = p0/T, u = 0."""
    _, y = _grid(nx, ny)
    T = 1.0 + eps * np.sin(2.0 * np.pi * y / ny)
    rho = p0 / T
    z = np.zeros((ny, nx))
    return rho, z.copy(), z.copy(), T


def _fourier_component(rng, nx, ny, kmax):
    """Real part of sum over integer wave vectors 1 <= max(|kx|,|ky|) <= kmax of
    A_k exp(2 pi i (kx x/nx + ky y/ny)), A_k ~ (N(0,1) + i N(0,1)) / |k|."""
    spec = np.zeros((ny, nx), dtype=np.complex128)
    for ky in range(-kmax, kmax + 1):
        for kx in range(-kmax, kmax + 1):
            if max(abs(kx), abs(ky)) == 0:
                continue
            a = (rng.standard_normal() + 1j * rng.standard_normal()) / np.hypot(kx, ky)
            spec[ky % ny, kx % nx] += a
    field = np.fft.ifft2(spec) * (nx * ny)
    return field.real


def gaussian_bump_random_flow(nx: int = 1024, ny: int = 1024, seed: int = 1, amp_u: float = 0.02,
                              kmax: int = 8, bump: float = 0.05, sigma: float = 64.0, rho0: float = 1.0):
    """rho = rho0, T = 1 + bump * exp(-r^2 / (2 sigma^2)) with r the periodic distance to the
    domain centre, u from seeded random Fourier modes with |k|_inf <= kmax, each component
    scaled so that max|u_c| = amp_u."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    dx = np.abs(x - nx / 2.0)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - ny / 2.0)
    dy = np.minimum(dy, ny - dy)
    T = 1.0 + bump * np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
    comps = []
    for _ in range(2):
        c = _fourier_component(rng, nx, ny, kmax)
        comps.append(c * (amp_u / np.max(np.abs(c))))
    rho = np.full((ny, nx), rho0)
    return rho, comps[0], comps[1], T


def couette_linear(nx: int, ny: int, T_lo: float, T_hi: float, rho0: float = 1.0):
    """Gas at rest between walls at y = -1/2 and y = ny - 1/2, T linear between the wall values."""
    _, y = _grid(nx, ny)
    T = T_lo + (T_hi - T_lo) * (y + 0.5) / ny
    rho = np.full((ny, nx), rho0)
    z = np.zeros((ny, nx))
    return rho, z.copy(), z.copy(), T


def random_smooth(nx: int, ny: int, seed: int, amp_u: float = 0.05, amp_T: float = 0.05,
                  amp_rho: float = 0.05, kmax: int = 3, rho0: float = 1.0):
    """Generic seeded smooth fields for parity tests: a few low Fourier modes per field,
    scaled to the stated maximum deviation from (rho0, 0, 0, 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for amp in (amp_rho, amp_u, amp_u, amp_T):
        if amp == 0.0:
            out.append(np.zeros((ny, nx)))
            continue
        c = _fourier_component(rng, nx, ny, kmax)
        m = np.max(np.abs(c))
        out.append(c * (amp / m) if m > 0 else c)
    return rho0 + out[0], out[1], out[2], 1.0 + out[3]


def batched_domains(count: int = 256, seed: int = 3, sizes=(128, 256, 512, 768, 1024)):
    """Parameters of a batch of independent periodic domains: side length drawn uniformly from
    `sizes`, tau ~ U[0.55, 1.5], Mach ~ U[0.05, 0.3], and a per-domain seed for its fields."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sizes), size=count)
    tau = rng.uniform(0.55, 1.5, size=count)
    mach = rng.uniform(0.05, 0.3, size=count)
    seeds = seed * 100003 + np.arange(count)
    return [dict(n=int(side[i]), tau=float(tau[i]), mach=float(mach[i]), seed=int(seeds[i])) for i in range(count)]


def tanh_faces(ny: int, height: float, beta: float):
    """Cell faces of a channel crowded towards both walls (the tanh law of Eq. NONUNI2 applied to
    the faces, as in Sec. "Grid Refinement for simple unidirectional flows"):
    F_k = H/2 (1 + tanh(beta (2k/ny - 1)) / tanh(beta)), k = 0..ny, the walls F_0 = 0 and
    F_ny = H exactly.  Mesh geometry (input data), not the method's arithmetic."""
    k = np.arange(ny + 1, dtype=np.float64)
    F = 0.5 * height * (1.0 + np.tanh(beta * (2.0 * k / ny - 1.0)) / np.tanh(beta))
    F[0], F[-1] = 0.0, float(height)
    return F


def random_faces(ny: int, seed: int, lo: float = 0.4, hi: float = 1.6):
    """Seeded cell faces with heights drawn uniformly from [lo, hi] (F_0 = 0)."""
    rng = np.random.default_rng(seed)
    return np.concatenate([[0.0], np.cumsum(rng.uniform(lo, hi, ny))])

