"""Seeded synthetic inputs shaped like the workloads of plane-wave DFT.

This module is the only code that both the CUDA path's tests/bench and the
FP64 oracle consume.  It draws random numbers and lays out grids; it holds
none of the transform's arithmetic.  Everything is NumPy ``default_rng(seed)``
so the same seed gives the same bytes on every machine.

Recipes (the paper uses CP2K grids of an H2O molecule, which are not
available; these stand in for them):

* ``uniform_grids``     -- re and im iid U[-1, 1).
* ``gaussian_sum_grids``-- per grid, 8 periodic Gaussians with centres
  U[0, N)^3 (grid units), widths sigma U[0.5, 2] grid units, complex
  amplitude |a| U[0.5, 1] with phase U[0, 2 pi), plus iid U[-1e-3, 1e-3)
  noise on re and im.  Each Gaussian is a * exp(-|r - R|^2 / (2 sigma^2))
  summed over the 27 nearest periodic images.
* ``mixed_sizes``       -- grid edges drawn uniformly from
  {32, 48, 64, 80, 96, 128} (2, 3 and 5 smooth).
* ``hartree_density``   -- a periodic cubic cell of side L bohr holding
  64 normalised Gaussians (2 pi s^2)^(-3/2) exp(-|r - R|^2 / (2 s^2)), centres
  U[0, L)^3, s U[0.3, 1.0] bohr, weights u ~ U(0, 1] rescaled to sum to the
  electron count (128), 27 nearest images.
"""
from __future__ import annotations

import math

import numpy as np

MIXED_EDGE_CHOICES = (32, 48, 64, 80, 96, 128)


def _periodic_gauss_1d(coord: np.ndarray, centre: float, sigma: float, period: float) -> np.ndarray:
    """sum over images m in {-1, 0, 1} of exp(-(coord - centre - m*period)^2 / (2 sigma^2))."""
    acc = np.zeros_like(coord, dtype=np.float64)
    for m in (-1.0, 0.0, 1.0):
        d = coord - centre - m * period
        acc += np.exp(-0.5 * d * d / (sigma * sigma))
    return acc


def uniform_grids(n, batch: int = 1, seed: int = 0, dtype=np.complex64) -> np.ndarray:
    """``batch`` grids of shape ``n`` (int -> cubic, or (nz, ny, nx)) with
    re, im iid U[-1, 1).  Returns shape (batch, nz, ny, nx)."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=(batch,) + shape)
    im = rng.uniform(-1.0, 1.0, size=(batch,) + shape)
    return (re + 1j * im).astype(dtype)


def gaussian_sum_grids(n: int, batch: int = 1, seed: int = 0, count: int = 8,
                       noise: float = 1e-3, dtype=np.complex64) -> np.ndarray:
    """``batch`` cubic n^3 grids, each a sum of ``count`` periodic complex
    Gaussians plus uniform noise (recipe in the module docstring)."""
    rng = np.random.default_rng(seed)
    coord = np.arange(n, dtype=np.float64)
    out = np.empty((batch, n, n, n), dtype=np.complex128)
    for b in range(batch):
        g = np.zeros((n, n, n), dtype=np.complex128)
        centres = rng.uniform(0.0, n, size=(count, 3))
        sigmas = rng.uniform(0.5, 2.0, size=count)
        mags = rng.uniform(0.5, 1.0, size=count)
        phases = rng.uniform(0.0, 2.0 * math.pi, size=count)
        for c, s, m, p in zip(centres, sigmas, mags, phases):
            gx = _periodic_gauss_1d(coord, c[0], s, n)
            gy = _periodic_gauss_1d(coord, c[1], s, n)
            gz = _periodic_gauss_1d(coord, c[2], s, n)
            a = m * complex(math.cos(p), math.sin(p))
            g += a * (gz[:, None, None] * gy[None, :, None] * gx[None, None, :])
        g += rng.uniform(-noise, noise, size=(n, n, n))
        g += 1j * rng.uniform(-noise, noise, size=(n, n, n))
        out[b] = g
    return out.astype(dtype)


def mixed_sizes(count: int = 64, seed: int = 0, choices=MIXED_EDGE_CHOICES) -> list[int]:
    """``count`` cubic grid edges drawn uniformly from ``choices``."""
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=count)]


def mixed_grids(sizes, seed: int = 0, dtype=np.complex64) -> list[np.ndarray]:
    """One uniform U[-1, 1) grid per edge in ``sizes``."""
    rng = np.random.default_rng(seed)
    grids = []
    for n in sizes:
        re = rng.uniform(-1.0, 1.0, size=(n, n, n))
        im = rng.uniform(-1.0, 1.0, size=(n, n, n))
        grids.append((re + 1j * im).astype(dtype))
    return grids


def hartree_density(n: int, L: float = 10.0, seed: int = 0, count: int = 64,
                    electrons: float = 128.0, sigma_range=(0.3, 1.0)):
    """Real periodic density on an n^3 grid of a cubic cell of side L (bohr),
    r_j = (L/n) * (x, y, z).  Returns (rho[z, y, x] float64, centres (count, 3)
    as (x, y, z) in bohr, sigmas, weights)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, L, size=(count, 3))
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=count)
    u = 1.0 - rng.uniform(0.0, 1.0, size=count)          # (0, 1]
    weights = u * (electrons / u.sum())
    coord = np.arange(n, dtype=np.float64) * (L / n)
    rho = np.zeros((n, n, n), dtype=np.float64)
    for c, s, w in zip(centres, sigmas, weights):
        norm = w * (2.0 * math.pi * s * s) ** -1.5
        gx = _periodic_gauss_1d(coord, c[0], s, L)
        gy = _periodic_gauss_1d(coord, c[1], s, L)
        gz = _periodic_gauss_1d(coord, c[2], s, L)
        rho += norm * (gz[:, None, None] * gy[None, :, None] * gx[None, None, :])
    return rho, centres, sigmas, weights
