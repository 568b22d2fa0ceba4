"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module draws random numbers and samples smooth analytic fields; it holds
none of the solver's arithmetic (no stencil, no smoothing, no restriction, no
interpolation, no projection).  Every generator returns plain float64 numpy
arrays in row-major (y, x) layout.

Workload shapes follow the benchmark setups of the paper (Sec. 4.3, the
lid-driven cavity of Sec. 4.2 and the turbulent jet of Sec. 4.3.2) restated
as synthetic inputs:

* ``smooth_rhs``: the divergence of a smooth random velocity field built from
  8x8 Fourier modes with N(0,1) amplitudes decaying as 1/k^2.  The field has
  zero normal velocity on the four walls, so its divergence is a sum of
  cos(k pi x) cos(l pi y) modes and is compatible with all-Neumann walls.
* ``smooth_velocity``: the matching staggered (MAC) face velocities.
* ``jet_inflow``: a top-hat inlet profile with seeded white-noise perturbation
  and a coflow, as drawn by the caller of the projection step.
* ``batch_shapes``: uneven domain sizes for the batched ensemble.
"""
from __future__ import annotations

import numpy as np

__all__ = ["smooth_rhs", "smooth_velocity", "jet_inflow", "batch_shapes",
           "random_field"]


def _mode_amplitudes(seed: int, nmodes: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((nmodes, nmodes))
    b = rng.standard_normal((nmodes, nmodes))
    k = np.arange(1, nmodes + 1, dtype=np.float64)
    k2 = k[None, :] ** 2 + k[:, None] ** 2          # [l-1, k-1] -> k^2 + l^2
    return a / k2, b / k2, k


def smooth_velocity(nx: int, ny: int, seed: int = 0, nmodes: int = 8):
    """MAC face velocities of a smooth random field on the unit square.

    u(x, y) = sum_{k,l} A_lk sin(k pi x) cos(l pi y)   on x-faces, shape (ny, nx+1)
    v(x, y) = sum_{k,l} B_lk cos(k pi x) sin(l pi y)   on y-faces, shape (ny+1, nx)

    with A, B ~ N(0,1)/(k^2+l^2).  u vanishes on x=0,1 and v on y=0,1.
    x is measured in units of the domain width, y of the domain height.
    """
    A, B, k = _mode_amplitudes(seed, nmodes)
    xf = np.arange(nx + 1) / nx
    xc = (np.arange(nx) + 0.5) / nx
    yf = np.arange(ny + 1) / ny
    yc = (np.arange(ny) + 0.5) / ny
    sx_f = np.sin(np.pi * np.outer(k, xf))          # (K, nx+1)
    cy_c = np.cos(np.pi * np.outer(k, yc))          # (L, ny)
    cx_c = np.cos(np.pi * np.outer(k, xc))
    sy_f = np.sin(np.pi * np.outer(k, yf))
    u = cy_c.T @ A @ sx_f                           # (ny, nx+1)
    v = sy_f.T @ B @ cx_c                           # (ny+1, nx)
    u[:, 0] = 0.0                                   # sin(0), sin(k pi): exact zeros
    u[:, -1] = 0.0
    v[0, :] = 0.0
    v[-1, :] = 0.0
    return u, v


def smooth_rhs(nx: int, ny: int, seed: int = 0, nmodes: int = 8):
    """Cell-centred right-hand side: the analytic divergence of
    ``smooth_velocity`` sampled at cell centres, scaled to the flux units of
    the pressure equation on a unit cell (multiplied by hx*hy).

    Every sampled mode cos(k pi x_c) cos(l pi y_c) with k, l >= 1 sums to zero
    over the cell centres, so the field is mean-free up to rounding.
    """
    A, B, k = _mode_amplitudes(seed, nmodes)
    xc = (np.arange(nx) + 0.5) / nx
    yc = (np.arange(ny) + 0.5) / ny
    cx = np.cos(np.pi * np.outer(k, xc))
    cy = np.cos(np.pi * np.outer(k, yc))
    # d/dx of A sin(k pi x) cos(l pi y) = A k pi cos cos ; d/dy of B cos sin = B l pi cos cos
    kk = k[None, :] * np.pi                         # over k (columns)
    ll = k[:, None] * np.pi                         # over l (rows)
    coef = A * kk + B * ll
    div = cy.T @ coef @ cx                          # (ny, nx), in 1/length^2 of the unit square
    return div / (nx * ny)


def random_field(nx: int, ny: int, seed: int = 0):
    """Plain N(0,1) cell field (white noise), for operator and smoother tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((ny, nx))


def jet_inflow(ny: int, width: int = 64, u_jet: float = 1.0, coflow: float = 0.05,
               noise: float = 0.01, seed: int = 0):
    """West-face inlet profile of the planar jet, length ny.

    Top-hat of height ``u_jet`` over ``width`` cells centred in y, ``coflow``
    elsewhere, times (1 + noise * N(0,1)) inside the jet (seeded white noise).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    prof = np.full(ny, coflow, dtype=np.float64)
    j0 = (ny - width) // 2
    prof[j0:j0 + width] = u_jet * (1.0 + noise * rng.standard_normal(width))
    return prof


def batch_shapes(n: int = 256, seed: int = 0, lo: int = 128, hi: int = 1024):
    """Uneven domain sizes: nx uniform over multiples of 32 in [lo, hi],
    aspect ratio r uniform in [1, 4], ny = clamp(round32(nx / r or nx * r)),
    orientation random.  Returns a list of (nx, ny)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.arange(lo, hi + 1, 32)
    out = []
    for _ in range(n):
        nx = int(rng.choice(sides))
        r = float(rng.uniform(1.0, 4.0))
        wide = bool(rng.integers(0, 2))
        ny = nx / r if wide else nx * r
        ny = int(np.clip(32 * round(ny / 32), lo, hi))
        out.append((nx, ny))
    return out
