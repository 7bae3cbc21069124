"""Hartree energy and gradient on the GPU against the FP64 oracle and the
closed form (cubic cell L = 10 bohr, 64 normalised Gaussians, 128
electrons).

Tolerances: the energy is a sum of positive terms built from FP32 spectra
(relative error ~1e-7 per term) accumulated in FP64 -> 2e-6 relative; the
gradient goes through two FP32 transforms -> 2e-5 relative L2 (of the
gradient's norm)."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

CELL = 10.0


def _rho(n, seed=0):
    rho, c, s, w = synth.hartree_density(n, CELL, seed=seed)
    return rho, c, s, w


def test_energy_128_matches_oracle_and_closed_form(cuda):
    from paper_2006_08435_gb300 import hartree_energy
    n = 128
    rho, c, s, w = _rho(n)
    e_gpu = float(hartree_energy(torch.from_numpy(rho.astype(np.float32)).cuda(), CELL))
    # the oracle on the same FP32-rounded density
    e_ref = oracle.hartree_energy(rho.astype(np.float32).astype(np.float64), CELL)
    assert e_gpu == pytest.approx(e_ref, rel=2e-6)
    rhohat = oracle.analytic_rhohat_gaussians(n, CELL, c, s, w)
    e_exact = 0.5 * CELL ** 3 * float(np.sum(oracle.hartree_kernel(n, CELL) * np.abs(rhohat) ** 2))
    assert e_gpu == pytest.approx(e_exact, rel=2e-6)


def test_gradient_128_matches_oracle_and_potential(cuda):
    from paper_2006_08435_gb300 import hartree_energy
    n = 128
    rho, c, s, w = _rho(n, seed=1)
    x = torch.from_numpy(rho.astype(np.float32)).cuda().requires_grad_(True)
    e = hartree_energy(x, CELL)
    e.backward()
    g = x.grad.double().cpu().numpy()
    ref = oracle.hartree_gradient(rho.astype(np.float32).astype(np.float64), CELL)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 2e-5
    # (n^3 / Omega) dE/drho is the Hartree potential; compare at a few grid
    # points with the closed-form Fourier series of the Gaussians
    rhohat = oracle.analytic_rhohat_gaussians(n, CELL, c, s, w)
    coef = oracle.hartree_kernel(n, CELL) * rhohat
    gi = oracle.g_index(n) * (2 * math.pi / CELL)
    v = g * n ** 3 / CELL ** 3
    rng = np.random.default_rng(3)
    for _ in range(4):
        z, y, xx = rng.integers(0, n, size=3)
        r = np.array([xx, y, z]) * (CELL / n)
        ph = (np.exp(1j * gi * r[2])[:, None, None] * np.exp(1j * gi * r[1])[None, :, None]
              * np.exp(1j * gi * r[0])[None, None, :])
        v_exact = float(np.sum(coef * ph).real)
        assert v[z, y, xx] == pytest.approx(v_exact, abs=2e-5 * np.abs(v).max())


def test_gradient_16_matches_fp64_finite_differences(cuda):
    """E_H is a quadratic form: the FP64 central difference of the oracle's
    energy is exact up to rounding, for any step."""
    from paper_2006_08435_gb300 import hartree_energy
    n = 16
    rho, _, _, _ = _rho(n, seed=2)
    rho32 = rho.astype(np.float32).astype(np.float64)
    x = torch.from_numpy(rho32.astype(np.float32)).cuda().requires_grad_(True)
    hartree_energy(x, CELL).backward()
    g = x.grad.double().cpu().numpy()
    scale = np.abs(g).max()
    rng = np.random.default_rng(0)
    for _ in range(12):
        j = tuple(rng.integers(0, n, size=3))
        h = 0.5
        p = rho32.copy(); p[j] += h
        m = rho32.copy(); m[j] -= h
        fd = (oracle.hartree_energy(p, CELL) - oracle.hartree_energy(m, CELL)) / (2 * h)
        assert g[j] == pytest.approx(fd, abs=2e-5 * scale)


def test_batch_and_reproducibility(cuda):
    """A batch gives each grid's energy (two real grids share one complex
    transform, so a grid's FP32 rounding depends on its partner: equal to
    within the energy tolerance, not bit for bit), and the same call twice
    gives the same bits (fixed reduction order)."""
    from paper_2006_08435_gb300 import hartree_energy
    n = 32
    a = _rho(n, seed=5)[0].astype(np.float32)
    b = _rho(n, seed=6)[0].astype(np.float32)
    both = torch.from_numpy(np.stack([a, b])).cuda()
    e2 = hartree_energy(both, CELL)
    ea = hartree_energy(torch.from_numpy(a).cuda(), CELL)
    eb = hartree_energy(torch.from_numpy(b).cuda(), CELL)
    assert e2.shape == (2,)
    assert float(e2[0]) == pytest.approx(float(ea), rel=2e-6)
    assert float(e2[1]) == pytest.approx(float(eb), rel=2e-6)
    assert float(hartree_energy(torch.from_numpy(a).cuda(), CELL)) == float(ea)
    assert torch.equal(hartree_energy(both, CELL), e2)
    assert float(ea) == pytest.approx(oracle.hartree_energy(a.astype(np.float64), CELL), rel=2e-6)


@pytest.mark.parametrize("n", [16, 64])
def test_half_spectrum_kernels_match_full_spectrum(cuda, n):
    """The half-spectrum energy (mirrored points counted twice) equals the
    full-spectrum energy of the same density to FP64 summation order, and
    the half-spectrum seed through the real inverse transform gives the
    full path's gradient."""
    from paper_2006_08435_gb300 import fft3d, irfft3d, rfft3d
    from paper_2006_08435_gb300 import hartree as H
    rho = np.stack([_rho(n, seed=s)[0] for s in (4, 5)]).astype(np.float32)
    x = torch.from_numpy(rho).cuda()
    full = fft3d(H.real_to_complex(x))
    half = rfft3d(x)
    e_full = H.energy_from_spectrum(full, CELL).cpu().numpy()
    e_half = H.energy_from_half_spectrum(half, CELL).cpu().numpy()
    assert np.allclose(e_half, e_full, rtol=1e-7, atol=0.0)
    g = torch.tensor([1.0, -2.5], dtype=torch.float64, device="cuda")
    grad_full = H.complex_to_real(fft3d(H.seed_from_spectrum(full, CELL, g), inverse=True))
    grad_half = irfft3d(H.seed_from_half_spectrum(half, CELL, g))
    gf, gh = grad_full.double().cpu().numpy(), grad_half.double().cpu().numpy()
    assert np.linalg.norm(gh - gf) / np.linalg.norm(gf) <= 1e-5


def test_odd_edge_uses_the_complex_path(cuda):
    """An odd edge (15^3: no half spectrum) goes through the complex
    transforms and still matches the oracle."""
    from paper_2006_08435_gb300 import hartree_energy
    n = 15
    rho = _rho(n, seed=6)[0].astype(np.float32)
    x = torch.from_numpy(rho).cuda().requires_grad_(True)
    e = hartree_energy(x, CELL)
    e.backward()
    ref_e = oracle.hartree_energy(rho.astype(np.float64), CELL)
    ref_g = oracle.hartree_gradient(rho.astype(np.float64), CELL)
    assert float(e.detach()) == pytest.approx(ref_e, rel=2e-6)
    g = x.grad.double().cpu().numpy()
    assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) <= 2e-5
