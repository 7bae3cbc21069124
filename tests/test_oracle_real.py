"""Pins for the real-grid oracle (``rdft3d`` / ``irdft3d``; CPU only).

Eq. 1 applied to a real grid has F(-k) = conj(F(k)), so the forward
transform keeps the half spectrum kx <= nx/2 and the inverse rebuilds the
rest by that symmetry.  The checks reach past the oracle itself: the literal
triple sum, closed forms, an independent library routine (NumPy's real
transforms, including its treatment of half spectra that are not exactly
Hermitian), the round trip, and planted slips in the Hermitian extension
that each of them must catch.
"""
import numpy as np
import pytest

from oracle import oracle

SHAPES = [(2, 2, 2), (3, 4, 4), (4, 3, 6), (5, 5, 4), (4, 4, 8)]


def _real(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _half(shape, seed):
    nz, ny, nx = shape[-3:]
    rng = np.random.default_rng(seed)
    s = shape[:-1] + (nx // 2 + 1,)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


@pytest.mark.parametrize("shape", SHAPES)
def test_rdft3d_is_the_triple_sum_half(shape):
    """The kept bins are exactly the triple sum of Eq. 1 at kx <= nx/2."""
    r = _real(shape, 1)
    full = oracle.dft3d_brute(r.astype(np.complex128), -1)
    half = oracle.rdft3d(r)
    assert half.shape == shape[:-1] + (shape[-1] // 2 + 1,)
    assert oracle.rel_l2(half, full[..., : shape[-1] // 2 + 1]) < 1e-13
    # and the dropped bins are the mirrored conjugates of kept ones
    assert oracle.rel_l2(oracle.hermitian_extend(half, shape[-1]), full) < 1e-13


@pytest.mark.parametrize("shape", SHAPES + [(3, 4, 4, 6)])
def test_against_numpy_real_transforms(shape):
    """Independent library routine in both directions; the inverse on half
    spectra that are NOT Hermitian in the self-mirrored planes, where the
    library likewise keeps the real part."""
    r = _real(shape, 2)
    assert oracle.rel_l2(oracle.rdft3d(r), np.fft.rfftn(r, axes=(-3, -2, -1))) < 1e-13
    h = _half(shape, 3)
    ref = np.fft.irfftn(h, s=shape[-3:], axes=(-3, -2, -1), norm="forward")
    got = oracle.irdft3d(h, shape[-1])
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES)
def test_round_trip(shape):
    """Unnormalised forward then inverse multiplies a real grid by nz ny nx."""
    r = _real(shape, 4)
    back = oracle.irdft3d(oracle.rdft3d(r), shape[-1])
    assert np.abs(back - np.prod(shape) * r).max() < 1e-12 * np.prod(shape)


def test_closed_forms():
    """A real delta at (x0, y0, z0) has F(k) = W^(k . x0); a cosine along x
    with m cycles has F = n^3 / 2 at kx = m (and nothing else kept, m < n/2);
    a constant has only the DC bin."""
    nz, ny, nx = 4, 6, 8
    r = np.zeros((nz, ny, nx))
    x0, y0, z0 = 3, 5, 2
    r[z0, y0, x0] = 1.0
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx // 2 + 1), indexing="ij")
    expect = np.exp(-2j * np.pi * (kx * x0 / nx + ky * y0 / ny + kz * z0 / nz))
    assert np.abs(oracle.rdft3d(r) - expect).max() < 1e-13
    m = 3
    xs = np.arange(nx)
    c = np.broadcast_to(np.cos(2 * np.pi * m * xs / nx), (nz, ny, nx))
    h = oracle.rdft3d(c)
    peak = np.zeros_like(h)
    peak[0, 0, m] = nz * ny * nx / 2
    assert np.abs(h - peak).max() < 1e-12
    h1 = oracle.rdft3d(np.full((nz, ny, nx), 2.5))
    dc = np.zeros_like(h1)
    dc[0, 0, 0] = 2.5 * nz * ny * nx
    assert np.abs(h1 - dc).max() < 1e-12


def test_self_mirrored_imaginary_parts_drop_out():
    """Bins with k = -k (kx in {0, nx/2}, ky, kz in {0, n/2}) carry only a
    real part in a real grid's spectrum; the inverse ignores their imaginary
    parts, while the same change in any other kept bin changes the grid."""
    shape = (4, 4, 6)
    h = _half(shape, 5)
    base = oracle.irdft3d(h, shape[-1])
    for k in [(0, 0, 0), (0, 0, 3), (2, 0, 0), (2, 2, 3)]:
        g = h.copy()
        g[k] += 1j * 0.75
        assert np.abs(oracle.irdft3d(g, shape[-1]) - base).max() < 1e-12
    g = h.copy()
    g[1, 2, 1] += 1j * 0.75
    assert np.abs(oracle.irdft3d(g, shape[-1]) - base).max() > 0.1


def _mutant_extend(half, nx, mistake):
    """hermitian_extend with one planted slip."""
    h = np.asarray(half, dtype=np.complex128)
    nz, ny = h.shape[-3], h.shape[-2]
    full = np.empty(h.shape[:-1] + (nx,), dtype=np.complex128)
    full[..., : nx // 2 + 1] = h
    mz = (-np.arange(nz)) % nz if mistake != "no_mirror_z" else np.arange(nz)
    my = (-np.arange(ny)) % ny if mistake != "no_mirror_y" else np.arange(ny)
    for kx in range(nx // 2 + 1, nx):
        src = nx - kx if mistake != "off_by_one" else nx - kx - 1
        col = h[..., src][..., mz, :][..., :, my]
        full[..., kx] = col if mistake == "no_conj" else np.conj(col)
    return full


@pytest.mark.parametrize("mistake", ["no_conj", "no_mirror_z", "no_mirror_y", "off_by_one"])
def test_planted_extension_mistakes_are_caught(mistake):
    """A slip in rebuilding the dropped bins (missing conjugate, missing
    mirror of one axis, shifted column) breaks the round trip that the
    unmutated extension passes."""
    shape = (4, 6, 8)
    r = _real(shape, 6)
    half = oracle.rdft3d(r)
    good = oracle.dft3d(_mutant_extend(half, shape[-1], None), +1).real
    assert np.abs(good - np.prod(shape) * r).max() < 1e-10
    bad = oracle.dft3d(_mutant_extend(half, shape[-1], mistake), +1).real
    assert np.abs(bad - np.prod(shape) * r).max() > 1e-3
