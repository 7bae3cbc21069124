"""The Hartree entry points of the C ABI on a machine without a GPU: the
workspace size and every argument check that must answer before a device
is touched (null pointers, edges and batches out of range, a cell that is
not a positive finite length, odd edges on the half-spectrum entry points,
a workspace that is too small, misaligned spectra).  The fake device
addresses are never dereferenced: each call returns at its check."""
import ctypes
import math

import pytest

from paper_2006_08435_gb300 import _lib as L

P = 1 << 20          # an aligned fake device address
MIS = (1 << 20) + 4  # a fake address that is not 8-byte aligned
CELL = 10.0


def test_workspace_bytes(fft3d_lib):
    ws = fft3d_lib.fft3d_hartree_workspace_bytes
    assert ws(1, 4) == 0 and ws(16, 0) == 0 and ws(-3, 2) == 0
    for n in (2, 16, 64, 128, 256):
        prev = 0
        for batch in (1, 2, 32, 1000):
            b = ws(n, batch)
            # at least one FP64 partial and one counter per grid, and no
            # more than 512 partials per grid (plus the counters' alignment)
            assert 12 * batch <= b <= 8 * 512 * batch + 256 + 4 * batch
            assert b > prev
            prev = b


def _energy_calls(lib):
    return [lib.fft3d_hartree_energy, lib.fft3d_hartree_energy_half]


def _seed_calls(lib):
    return [lib.fft3d_hartree_seed, lib.fft3d_hartree_seed_half]


def test_energy_argument_checks(fft3d_lib):
    need = fft3d_lib.fft3d_hartree_workspace_bytes(16, 2)
    for f in _energy_calls(fft3d_lib):
        assert f(None, 16, 2, CELL, P, P, need, None) == L.FFT3D_ERR_NULL_PTR
        assert f(P, 16, 2, CELL, None, P, need, None) == L.FFT3D_ERR_NULL_PTR
        assert f(P, 16, 2, CELL, P, None, need, None) == L.FFT3D_ERR_NULL_PTR
        for n, batch, cell in ((1, 2, CELL), (2048, 1, CELL), (16, 0, CELL), (16, 70000, CELL),
                               (16, 2, 0.0), (16, 2, -1.0), (16, 2, math.inf), (16, 2, math.nan)):
            assert f(P, n, batch, cell, P, P, 1 << 40, None) == L.FFT3D_ERR_INVALID_ARG, (n, batch, cell)
        assert f(P, 16, 2, CELL, P, P, need - 1, None) == L.FFT3D_ERR_INVALID_ARG
        assert f(MIS, 16, 2, CELL, P, P, need, None) == L.FFT3D_ERR_MISALIGNED
        assert f(P, 16, 2, CELL, P, MIS, need, None) == L.FFT3D_ERR_MISALIGNED
    # odd edges: the full spectrum passes the checks that the half one fails
    assert fft3d_lib.fft3d_hartree_energy_half(
        P, 15, 1, CELL, P, P, 1 << 40, None) == L.FFT3D_ERR_INVALID_ARG
    assert fft3d_lib.fft3d_hartree_energy(
        MIS, 15, 1, CELL, P, P, 1 << 40, None) == L.FFT3D_ERR_MISALIGNED


def test_seed_argument_checks(fft3d_lib):
    for f in _seed_calls(fft3d_lib):
        assert f(None, 16, 2, CELL, P, P, None) == L.FFT3D_ERR_NULL_PTR
        assert f(P, 16, 2, CELL, None, P, None) == L.FFT3D_ERR_NULL_PTR
        assert f(P, 16, 2, CELL, P, None, None) == L.FFT3D_ERR_NULL_PTR
        for n, batch, cell in ((1, 2, CELL), (16, 0, CELL), (16, 2, 0.0), (16, 2, math.nan)):
            assert f(P, n, batch, cell, P, P, None) == L.FFT3D_ERR_INVALID_ARG, (n, batch, cell)
        assert f(MIS, 16, 2, CELL, P, P, None) == L.FFT3D_ERR_MISALIGNED
        assert f(P, 16, 2, CELL, P, MIS, None) == L.FFT3D_ERR_MISALIGNED
    assert fft3d_lib.fft3d_hartree_seed_half(P, 15, 1, CELL, P, P, None) == L.FFT3D_ERR_INVALID_ARG


def test_conversions_argument_checks(fft3d_lib):
    for f in (fft3d_lib.fft3d_real_to_complex, fft3d_lib.fft3d_complex_to_real):
        assert f(None, P, 8, None) == L.FFT3D_ERR_NULL_PTR
        assert f(P, None, 8, None) == L.FFT3D_ERR_NULL_PTR
        assert f(P, P, -1, None) == L.FFT3D_ERR_INVALID_ARG
        assert f(P, P, 0, None) == L.FFT3D_SUCCESS  # nothing to do, no launch


@pytest.mark.parametrize("name", ["fft3d_hartree_energy", "fft3d_hartree_energy_half",
                                  "fft3d_hartree_seed", "fft3d_hartree_seed_half",
                                  "fft3d_hartree_workspace_bytes"])
def test_declared_with_the_header_signature(fft3d_lib, name):
    f = getattr(fft3d_lib, name)
    assert f.argtypes and f.restype in (ctypes.c_int, ctypes.c_size_t)
