"""Pins for the oracle's plane-wave Hartree energy and gradient (CPU only).

* E_H is a quadratic form in rho, so the central finite difference
  (E(rho + h e_j) - E(rho - h e_j)) / 2h equals dE/drho_j exactly in exact
  arithmetic; the oracle's analytic gradient (Omega/N^3) V_H(r_j) must match
  it at every point of a 16^3 grid.
* For a density made of normalised periodic Gaussians the Fourier
  coefficients are known in closed form; on the 128^3 grid of a 10 bohr cell
  the aliasing of the sampled density is below exp(-70), so the oracle's
  E_H and V_H must match the closed-form series to ~1e-10.
"""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_2006_08435_gb300 import synth

L = 10.0


def test_kernel_and_g_grid():
    k = oracle.hartree_kernel(8, L)
    assert k[0, 0, 0] == 0.0
    m = oracle.g_index(8)
    assert list(m) == [0, 1, 2, 3, -4, -3, -2, -1]
    assert k[0, 0, 1] == pytest.approx(4 * math.pi / (2 * math.pi / L) ** 2)
    assert k[1, 0, 0] == k[0, 1, 0] == k[0, 0, 1] == k[0, 0, 7]


def test_gradient_matches_finite_differences_16():
    rho, _, _, _ = synth.hartree_density(16, L, seed=3)
    grad = oracle.hartree_gradient(rho, L)
    rng = np.random.default_rng(0)
    idx = [tuple(rng.integers(0, 16, size=3)) for _ in range(24)] + [(0, 0, 0), (15, 15, 15)]
    h = 1e-3
    scale = np.abs(grad).max()
    for j in idx:
        p = rho.copy(); p[j] += h
        m = rho.copy(); m[j] -= h
        fd = (oracle.hartree_energy(p, L) - oracle.hartree_energy(m, L)) / (2 * h)
        assert fd == pytest.approx(grad[j], abs=1e-8 * scale)


def test_energy_is_quadratic_and_neutral():
    rho, _, _, _ = synth.hartree_density(16, L, seed=4)
    e1 = oracle.hartree_energy(rho, L)
    assert e1 > 0
    assert oracle.hartree_energy(2.5 * rho, L) == pytest.approx(6.25 * e1, rel=1e-12)
    # a uniform background changes only G = 0, which is excluded
    assert oracle.hartree_energy(rho + 0.37, L) == pytest.approx(e1, rel=1e-12)


@pytest.mark.slow
def test_energy_and_potential_match_closed_form_128():
    n = 128
    rho, c, s, w = synth.hartree_density(n, L, seed=0)
    rhohat_exact = oracle.analytic_rhohat_gaussians(n, L, c, s, w)
    kern = oracle.hartree_kernel(n, L)
    e_exact = 0.5 * L ** 3 * float(np.sum(kern * np.abs(rhohat_exact) ** 2))
    e_oracle = oracle.hartree_energy(rho, L)
    assert e_oracle == pytest.approx(e_exact, rel=1e-10)
    # V_H at sampled grid points from the closed-form series
    v = oracle.hartree_potential(rho, L)
    g = oracle.g_index(n) * (2 * math.pi / L)
    coef = kern * rhohat_exact
    rng = np.random.default_rng(1)
    for _ in range(8):
        z, y, x = rng.integers(0, n, size=3)
        r = np.array([x, y, z]) * (L / n)
        ph = (np.exp(1j * g * r[2])[:, None, None] * np.exp(1j * g * r[1])[None, :, None]
              * np.exp(1j * g * r[0])[None, None, :])
        v_exact = float(np.sum(coef * ph).real)
        assert v[z, y, x] == pytest.approx(v_exact, rel=1e-9, abs=1e-9 * np.abs(v).max())
