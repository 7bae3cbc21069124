"""Pins for the FP64 oracle (CPU only).

The oracle is checked against things other than itself: the literal triple
sum of Eq. 1, exact integer arithmetic, closed forms of the DFT, its
invariants (Parseval, shift, linearity, Hermitian symmetry, round trip) and
an independent library routine.  Each check is chosen so that a plausible
mistake in the oracle (dropped term, wrong sign, transposed axis, wrong
root of unity per axis) fails at least one of them.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle
from paper_2006_08435_gb300 import synth
from tests.ref_numpy import dft3d_tensordot

SHAPES_TINY = [(2, 2, 2), (3, 3, 3), (4, 4, 4), (5, 5, 5), (4, 3, 2), (2, 5, 3)]


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("shape", SHAPES_TINY)
@pytest.mark.parametrize("sign", [-1, 1])
def test_separable_matches_triple_sum(shape, sign):
    """Eq. 1 written as a triple sum equals the x-then-y-then-z form."""
    x = _rand(shape, 1)
    a = oracle.dft3d(x, sign)
    b = oracle.dft3d_brute(x, sign)
    assert oracle.rel_l2(a, b) < 1e-13


def _exact_dft_n4(x_int):
    """Exact 4^3 DFT of a Gaussian-integer grid: W_4 = -i, so every twiddle
    is one of 1, -i, -1, i and the result is a Gaussian integer.  Python
    ints only (complex held as (re, im) pairs)."""
    n = 4
    pow_mi = [(1, 0), (0, -1), (-1, 0), (0, 1)]     # (-i)^m
    out = {}
    for kz, ky, kx in itertools.product(range(n), repeat=3):
        re = im = 0
        for z, y, xx in itertools.product(range(n), repeat=3):
            m = (xx * kx + y * ky + z * kz) % n
            wr, wi = pow_mi[m]
            ar, ai = x_int[z][y][xx]
            re += ar * wr - ai * wi
            im += ar * wi + ai * wr
        out[(kz, ky, kx)] = (re, im)
    return out


def test_exact_gaussian_integers_n4():
    rng = np.random.default_rng(7)
    vals = rng.integers(-9, 10, size=(4, 4, 4, 2))
    x_int = [[[(int(vals[z, y, x, 0]), int(vals[z, y, x, 1])) for x in range(4)]
              for y in range(4)] for z in range(4)]
    exact = _exact_dft_n4(x_int)
    got = oracle.dft3d(vals[..., 0] + 1j * vals[..., 1], -1)
    for (kz, ky, kx), (re, im) in exact.items():
        assert got[kz, ky, kx].real == pytest.approx(re, abs=1e-9)
        assert got[kz, ky, kx].imag == pytest.approx(im, abs=1e-9)


def test_n2_is_hadamard():
    """W_2 = -1: the 2^3 DFT is the Walsh-Hadamard matrix H (x) H (x) H."""
    h = np.array([[1.0, 1.0], [1.0, -1.0]])
    h3 = np.kron(np.kron(h, h), h)
    x = _rand((2, 2, 2), 3)
    assert np.allclose(oracle.dft3d(x).ravel(), h3 @ x.ravel(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [6, 8, 15])
def test_delta_closed_forms(n):
    x = np.zeros((n, n, n), complex)
    x[0, 0, 0] = 1.0
    assert np.allclose(oracle.dft3d(x), 1.0, atol=1e-13)
    a, b, c = 1, 2, n - 1          # delta at x=a, y=b, z=c
    x = np.zeros((n, n, n), complex)
    x[c, b, a] = 1.0
    k = np.arange(n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    expect = np.exp(-2j * np.pi * ((a * kx + b * ky + c * kz) % n) / n)
    assert np.allclose(oracle.dft3d(x, -1), expect, atol=1e-12)
    assert np.allclose(oracle.dft3d(x, +1), np.conj(expect), atol=1e-12)


@pytest.mark.parametrize("shape", [(4, 6, 8), (5, 5, 5)])
def test_constant_and_plane_wave(shape):
    nz, ny, nx = shape
    c = 0.3 - 0.7j
    out = oracle.dft3d(np.full(shape, c))
    expect = np.zeros(shape, complex)
    expect[0, 0, 0] = c * nx * ny * nz
    assert np.allclose(out, expect, atol=1e-12)
    k0 = (1, 2, 3)          # (kx, ky, kz)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wave = np.exp(2j * np.pi * (k0[0] * x / nx + k0[1] * y / ny + k0[2] * z / nz))
    out = oracle.dft3d(wave, -1)
    expect = np.zeros(shape, complex)
    expect[k0[2] % nz, k0[1] % ny, k0[0] % nx] = nx * ny * nz
    assert np.allclose(out, expect, atol=1e-10)


def test_separable_product_uses_each_axis_length():
    """g(x) h(y) p(z) on a non-cubic grid -> outer product of 1D DFTs of
    the right lengths (catches a wrong root of unity per axis or a swapped
    axis order)."""
    rng = np.random.default_rng(11)
    g = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    h = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    p = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    x = p[:, None, None] * h[None, :, None] * g[None, None, :]
    expect = (np.fft.fft(p)[:, None, None] * np.fft.fft(h)[None, :, None]
              * np.fft.fft(g)[None, None, :])
    assert oracle.rel_l2(oracle.dft3d(x), expect) < 1e-13


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 12)])
def test_invariants(shape):
    nz, ny, nx = shape
    npts = nx * ny * nz
    x = _rand(shape, 5)
    y = _rand(shape, 6)
    fx = oracle.dft3d(x)
    # Parseval
    assert np.sum(np.abs(fx) ** 2) == pytest.approx(npts * np.sum(np.abs(x) ** 2), rel=1e-12)
    # linearity
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    assert oracle.rel_l2(oracle.dft3d(a * x + b * y), a * fx + b * oracle.dft3d(y)) < 1e-13
    # shift theorem: f(x - s) -> F(k) W^(k s)
    s = (1, 2, 3)     # shift in x, y, z
    xs = np.roll(x, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = np.exp(-2j * np.pi * (kx * s[0] / nx + ky * s[1] / ny + kz * s[2] / nz))
    assert oracle.rel_l2(oracle.dft3d(xs), fx * ph) < 1e-12
    # Hermitian symmetry for real input: F(-k) = conj F(k)
    r = oracle.dft3d(x.real)
    flip = np.roll(r[::-1, ::-1, ::-1], shift=(1, 1, 1), axis=(0, 1, 2))
    assert np.allclose(flip, np.conj(r), atol=1e-11)
    # forward then inverse = N^3 identity
    assert oracle.rel_l2(oracle.dft3d(fx, +1), npts * x) < 1e-13


@pytest.mark.parametrize("shape", [(16, 16, 16), (3, 5, 12)])
def test_against_numpy_library(shape):
    x = _rand(shape, 9)
    assert oracle.rel_l2(oracle.dft3d(x), np.fft.fftn(x)) < 1e-13
    assert oracle.rel_l2(oracle.dft3d(x, +1), np.fft.ifftn(x) * np.prod(shape)) < 1e-13
    assert oracle.rel_l2(oracle.dft3d(x), dft3d_tensordot(x)) < 1e-13


def test_batch_is_independent_grids():
    x = synth.uniform_grids(6, batch=3, seed=2, dtype=np.complex128)
    out = oracle.dft3d(x)
    for b in range(3):
        assert oracle.rel_l2(out[b], oracle.dft3d(x[b])) == 0.0


def _mutant_dft3d(x, mistake):
    """The separable x, y, z transform with one planted slip."""
    a = np.asarray(x, dtype=np.complex128)
    nz, ny, nx = a.shape

    def mat(n, sign=-1, off=0):
        j = np.arange(n)
        return np.exp(sign * 2j * np.pi * ((np.outer(j, j) + off) % n) / n)

    mx = mat(nx, +1 if mistake == "sign" else -1)
    my = mat(nz if mistake == "root" else ny)[:ny, :ny]
    mz = mat(nz, off=1 if mistake == "index" else 0)
    a = a @ mx
    a = np.einsum("zyx,yk->zkx", a, my)
    if mistake != "skip_z":
        a = np.einsum("zyx,zk->kyx", a, mz)
    return a


@pytest.mark.parametrize("mistake", ["sign", "root", "index", "skip_z"])
def test_planted_mistakes_are_caught(mistake):
    """A plausible slip in a separable DFT (wrong sign, wrong root of unity
    for an axis, shifted index, dropped axis) is caught by the triple-sum
    pin, while the unmutated mutant passes it."""
    x = _rand((4, 3, 5), 4)
    truth = oracle.dft3d_brute(x, -1)
    assert oracle.rel_l2(_mutant_dft3d(x, None), truth) < 1e-13
    assert oracle.rel_l2(_mutant_dft3d(x, mistake), truth) > 1e-3


def test_synth_deterministic_and_in_range():
    a = synth.uniform_grids(8, 2, seed=3)
    b = synth.uniform_grids(8, 2, seed=3)
    assert np.array_equal(a, b)
    assert np.abs(a.real).max() <= 1.0 and np.abs(a.imag).max() <= 1.0
    g = synth.gaussian_sum_grids(16, 1, seed=1)
    assert g.shape == (1, 16, 16, 16) and np.abs(g).max() < 8.0
    sizes = synth.mixed_sizes(64, seed=0)
    assert len(sizes) == 64 and set(sizes) <= set(synth.MIXED_EDGE_CHOICES)
    rho, c, s, w = synth.hartree_density(16, 10.0, seed=0)
    assert w.sum() == pytest.approx(128.0) and (w > 0).all()
    assert (s >= 0.3).all() and (s <= 1.0).all() and (rho > 0).all()


def test_hartree_density_holds_its_electrons():
    """The density's grid sum times the cell volume per point is the total
    charge: for normalised periodic Gaussians sampled at spacing h the
    error is of order exp(-2 pi^2 sigma^2 / h^2) (Poisson summation), about
    1e-8 at sigma >= 0.3 bohr and h = 10/32 bohr."""
    for seed in (0, 1):
        rho, _, _, w = synth.hartree_density(32, 10.0, seed=seed)
        assert rho.sum() * (10.0 / 32) ** 3 == pytest.approx(w.sum(), rel=1e-6)
        assert w.sum() == pytest.approx(128.0, rel=1e-12)


# ------------------------------------------------ single outputs (dft3d_points)

@pytest.mark.parametrize("shape", SHAPES_TINY + [(3, 4, 5)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_points_match_triple_sum_everywhere(shape, sign):
    """Every output of dft3d_points equals the literal triple sum of Eq. 1
    (non-cubic shapes, so a swapped axis or index order fails)."""
    x = _rand(shape, 11)
    ref = oracle.dft3d_brute(x, sign)
    pts = np.array(list(itertools.product(*[range(s) for s in shape])))
    got = oracle.dft3d_points(x, pts, sign)
    assert np.max(np.abs(got - ref.ravel())) <= 1e-12 * np.max(np.abs(ref))


def test_points_match_library_on_a_larger_non_cubic_grid():
    x = _rand((12, 20, 45), 12)
    ref = np.fft.fftn(x)
    rng = np.random.default_rng(13)
    pts = np.stack([rng.integers(0, s, 40) for s in x.shape], axis=1)
    got = oracle.dft3d_points(x, pts, -1)
    want = ref[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(ref))


def test_points_plane_wave_closed_form():
    """exp(+2 pi i (kx0 x/nx + ky0 y/ny + kz0 z/nz)) has the forward
    transform nx ny nz at (kz0, ky0, kx0) and 0 elsewhere."""
    nz, ny, nx = 24, 30, 40
    k0 = (5, 7, 33)
    z, y, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.exp(2j * np.pi * (k0[2] * xx / nx + k0[1] * y / ny + k0[0] * z / nz))
    pts = np.array([k0, (0, 0, 0), (5, 7, 32), (k0[0], (k0[1] + 1) % ny, k0[2])])
    got = oracle.dft3d_points(f, pts, -1)
    assert abs(got[0] - nx * ny * nz) <= 1e-9 * nx * ny * nz
    assert np.max(np.abs(got[1:])) <= 1e-9 * nx * ny * nz


def test_points_reject_out_of_range():
    x = _rand((2, 3, 4), 14)
    for bad in ((2, 0, 0), (0, 3, 0), (0, 0, 4), (-1, 0, 0)):
        with pytest.raises(RuntimeError):
            oracle.dft3d_points(x, [bad], -1)
