"""The library's multiply-shift division parameters (make_fastdiv, the host
half of the Granlund-Montgomery division by an invariant integer that the
general-path and Hartree kernels use to turn flat indices into (kz, ky, kx)
and tile coordinates).  The kernels compute q = (hi32(n * mul) + n) >> shift;
here that formula is evaluated in exact 64-bit integers with the library's
own (mul, shift) and compared with floor division -- the definition it must
reproduce -- exhaustively on small ranges and at every quotient boundary
near the top of the ranges the kernels use."""
import ctypes

import numpy as np
import pytest


class _FastDiv(ctypes.Structure):
    _fields_ = [("mul", ctypes.c_uint), ("shift", ctypes.c_int)]


@pytest.fixture(scope="module")
def make_fastdiv(fft3d_lib):
    try:
        f = getattr(fft3d_lib, "_ZN5fft3d12make_fastdivEj")  # fft3d::make_fastdiv(unsigned)
    except AttributeError:
        pytest.skip("make_fastdiv is not an exported symbol of the library")
    f.restype = _FastDiv
    f.argtypes = [ctypes.c_uint]
    return f


def _quotient(n, p):
    n = n.astype(np.uint64)
    return (((n * np.uint64(p.mul)) >> np.uint64(32)) + n) >> np.uint64(p.shift)


# Every divisor the kernels use: pencil lengths and tile counts of the
# general path (up to 512), row lengths n and n/2 + 1 of the Hartree
# kernels (n up to 1024), plus powers of two and their neighbours.
DIVISORS = sorted(set(
    list(range(1, 600)) + [n // 2 + 1 for n in range(2, 1025, 2)] + list(range(600, 1025, 7)) +
    [1 << k for k in range(11, 32)] + [(1 << k) + 1 for k in range(11, 31)] +
    [(1 << k) - 1 for k in range(11, 32)] + [3 * 5 * 7 * 11 * 13, 65537, 1000003]))


def test_exhaustive_small_range(make_fastdiv):
    n = np.arange(1 << 16, dtype=np.uint64)
    for d in DIVISORS:
        p = make_fastdiv(d)
        assert 0 <= p.shift <= 32
        assert np.array_equal(_quotient(n, p), n // np.uint64(d)), d


def test_quotient_boundaries_up_to_2_pow_32(make_fastdiv):
    rng = np.random.default_rng(20060843)
    top = (1 << 32) - 1
    for d in DIVISORS:
        p = make_fastdiv(d)
        qmax = top // d
        # the last quotients below 2^32 and random ones across the range,
        # each checked at k*d - 1, k*d and k*d + d - 1 (clipped to 2^32 - 1)
        k = np.unique(np.concatenate([np.arange(max(qmax - 64, 0), qmax + 1),
                                      rng.integers(0, qmax + 1, size=256)])).astype(np.uint64)
        kd = k * np.uint64(d)
        n = np.concatenate([kd[k > 0] - np.uint64(1), kd, np.minimum(kd + np.uint64(d - 1), np.uint64(top))])
        n = np.concatenate([n, np.arange(top - 4096, top + 1, dtype=np.uint64)])
        assert np.array_equal(_quotient(n, p), n // np.uint64(d)), d


def test_hartree_index_ranges_exhaustive(make_fastdiv):
    """Every flat index of one half spectrum (n^2 (n/2 + 1) points) and of
    one full spectrum (n^3) for the edges up to 128: the row and plane
    divisions recover (kz, ky, kx) exactly."""
    for n in (2, 3, 16, 30, 64, 96, 100, 128):
        for h in ((n // 2 + 1) if n % 2 == 0 else None, n):
            if h is None:
                continue
            i = np.arange(n * n * h, dtype=np.uint64)
            row = _quotient(i, make_fastdiv(h))
            kz = _quotient(row, make_fastdiv(n))
            kx = i - row * np.uint64(h)
            ky = row - kz * np.uint64(n)
            ref_kz, rem = np.divmod(i, np.uint64(n * h))
            ref_ky, ref_kx = np.divmod(rem, np.uint64(h))
            assert np.array_equal(kz, ref_kz) and np.array_equal(ky, ref_ky) and np.array_equal(kx, ref_kx)
