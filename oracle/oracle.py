"""FP64 CPU oracle for the 3D complex-to-complex DFT and the plane-wave
Hartree energy built on it.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  It shares no code with the CUDA path (``paper_2006_08435_gb300``)
and never imports it; the only common module is the seeded input generator,
which holds none of the method's arithmetic.

Contents
--------
* ``dft3d``        -- Eq. 1 of the paper (section "Approach") as a separable
  direct DFT, x then y then z, in plain C (``dft3d.c``), FP64, OpenMP over
  lines.  O(n^4) for an n^3 grid.
* ``dft3d_brute``  -- the literal triple sum of Eq. 1, O(n^6); pins the
  separable form on tiny grids.
* ``dft3d_points`` -- single outputs of Eq. 1, each from the definition
  (sums over x, then y, then z), O(n^3) per output: checks of grids too
  large for ``dft3d`` (256^3 and up).
* ``rdft3d`` / ``irdft3d`` -- Eq. 1 for real grids (a real density, the
  paper's plane-wave DFT setting): the forward transform of a real grid
  keeps the half spectrum kx <= nx/2 (the rest is its complex conjugate
  mirrored); the inverse extends a half spectrum by that symmetry and keeps
  the real part of the inverse transform.  Both are the complex ``dft3d``
  plus that bookkeeping.
* ``hartree_*``    -- the plane-wave Hartree energy of a periodic density and
  its gradient, written from the standard Gaussian-and-plane-wave definition
  (the paper's motivating application, section "Introduction" and
  "Results"): rho_hat(G) = F(rho)(G) / N^3,
  E_H = (Omega/2) sum_{G != 0} 4 pi |rho_hat(G)|^2 / |G|^2, and
  dE_H/drho_j = (Omega / N^3) V_H(r_j).  The paper gives no formulas for this
  part; these are the textbook ones.
* ``analytic_*``   -- the closed-form Fourier coefficients of a sum of
  normalised periodic Gaussians, used to pin the Hartree oracle.

Every function takes and returns NumPy arrays; complex grids have shape
``(..., nz, ny, nx)`` with x fastest.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dft3d.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``dft3d.c`` into ``liboracle.so`` (gcc, -O2, OpenMP, no
    fast-math so IEEE double semantics hold).  Returns the library path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_dft3d.argtypes = [dp, dp] + [ctypes.c_int] * 5
            lib.oracle_dft3d.restype = ctypes.c_int
            lib.oracle_dft3d_brute.argtypes = [dp, dp] + [ctypes.c_int] * 4
            lib.oracle_dft3d_brute.restype = ctypes.c_int
            lib.oracle_dft3d_points.argtypes = [dp] + [ctypes.c_int] * 3 + [
                ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_dft3d_points.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_num_threads())


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dft3d(x, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT of Eq. 1 over the last three axes (z, y, x).

    ``sign`` is the sign of the exponent: -1 forward, +1 inverse.  Leading
    axes are a batch of independent grids.  FP64 throughout."""
    a = _as_c128(x)
    if a.ndim < 3:
        raise ValueError("need at least 3 dims (nz, ny, nx)")
    nz, ny, nx = a.shape[-3:]
    batch = int(np.prod(a.shape[:-3], dtype=np.int64)) if a.ndim > 3 else 1
    out = np.empty_like(a)
    rc = _load().oracle_dft3d(_dp(a), _dp(out), nx, ny, nz, batch, int(sign))
    if rc != 0:
        raise RuntimeError(f"oracle_dft3d failed ({rc})")
    return out


def dft3d_brute(x, sign: int = -1) -> np.ndarray:
    """The literal triple sum of Eq. 1 for one grid (n^6 terms)."""
    a = _as_c128(x)
    if a.ndim != 3:
        raise ValueError("one grid (nz, ny, nx)")
    nz, ny, nx = a.shape
    out = np.empty_like(a)
    rc = _load().oracle_dft3d_brute(_dp(a), _dp(out), nx, ny, nz, int(sign))
    if rc != 0:
        raise RuntimeError(f"oracle_dft3d_brute failed ({rc})")
    return out


def dft3d_points(x, points, sign: int = -1) -> np.ndarray:
    """Selected outputs F(kz, ky, kx) of Eq. 1 for ONE grid (nz, ny, nx),
    each computed by itself from the definition (sums over x, y, z), for
    grids too large for ``dft3d``.  ``points``: (m, 3) integer array of
    (kz, ky, kx).  Returns m complex128 values."""
    a = _as_c128(x)
    if a.ndim != 3:
        raise ValueError("one grid (nz, ny, nx)")
    nz, ny, nx = a.shape
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1, 3))
    out = np.empty(pts.shape[0], dtype=np.complex128)
    rc = _load().oracle_dft3d_points(_dp(a), nx, ny, nz,
                                     pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     pts.shape[0], int(sign), _dp(out))
    if rc != 0:
        raise RuntimeError(f"oracle_dft3d_points failed ({rc})")
    return out


def rdft3d(r) -> np.ndarray:
    """Forward transform (Eq. 1, exponent sign -1, unnormalised) of REAL
    grids over the last three axes (nz, ny, nx), returned as the half
    spectrum kx = 0 .. nx // 2: shape (..., nz, ny, nx // 2 + 1), complex128.
    For real input F(-k) = conj(F(k)), so the dropped bins carry nothing
    new.  FP64 throughout."""
    a = np.asarray(r)
    if np.iscomplexobj(a):
        raise TypeError("rdft3d takes real grids")
    if a.ndim < 3:
        raise ValueError("need at least 3 dims (nz, ny, nx)")
    nx = a.shape[-1]
    return dft3d(a.astype(np.float64), sign=-1)[..., : nx // 2 + 1]


def hermitian_extend(half, nx: int) -> np.ndarray:
    """Full spectrum E(X) of a half spectrum X (..., nz, ny, nx // 2 + 1):
    E(X)(k) = X(k) for kx <= nx // 2 and conj(X(-k)) for kx > nx // 2, with
    -k taken modulo (nz, ny, nx)."""
    h = _as_c128(half)
    if h.ndim < 3 or h.shape[-1] != nx // 2 + 1:
        raise ValueError("need (..., nz, ny, nx // 2 + 1)")
    nz, ny = h.shape[-3], h.shape[-2]
    full = np.empty(h.shape[:-1] + (nx,), dtype=np.complex128)
    full[..., : nx // 2 + 1] = h
    for kx in range(nx // 2 + 1, nx):
        # conj(X(-kz, -ky, nx - kx)) for every (kz, ky)
        mz = (-np.arange(nz)) % nz
        my = (-np.arange(ny)) % ny
        col = h[..., nx - kx]                      # (..., nz, ny)
        full[..., kx] = np.conj(col[..., mz, :][..., :, my])
    return full


def irdft3d(half, nx: int) -> np.ndarray:
    """Inverse transform (exponent sign +1, unnormalised) of half spectra
    (..., nz, ny, nx // 2 + 1) to REAL grids (..., nz, ny, nx): the real part
    of the inverse transform of the Hermitian extension E(X).  For a half
    spectrum of a real grid this is nz ny nx times that grid; for any other
    input it equals the inverse of the Hermitian part of E(X) (the imaginary
    parts of the self-mirrored bins drop out).  FP64 throughout."""
    return dft3d(hermitian_extend(half, nx), sign=+1).real


def rel_l2(y, y_ref) -> float:
    """||y - y_ref||_2 / ||y_ref||_2 in FP64."""
    y = np.asarray(y, dtype=np.complex128)
    r = np.asarray(y_ref, dtype=np.complex128)
    return float(np.linalg.norm((y - r).ravel()) / np.linalg.norm(r.ravel()))


# ---------------------------------------------------------------------------
# Plane-wave Hartree energy (Gaussian and plane-wave DFT, the application the
# paper accelerates).  Cubic periodic cell of side L (bohr), N^3 grid,
# r_j = (L/N) * (x, y, z).
# ---------------------------------------------------------------------------

def g_index(n: int) -> np.ndarray:
    """Signed frequency index of DFT bin k: k for k < n/2, k - n otherwise."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def g_squared(n: int, L: float) -> np.ndarray:
    """|G|^2 on the n^3 DFT bins, G = 2 pi m / L, shape (n, n, n) = (z, y, x)."""
    m = g_index(n).astype(np.float64) * (2.0 * math.pi / L)
    m2 = m * m
    return m2[:, None, None] + m2[None, :, None] + m2[None, None, :]


def hartree_kernel(n: int, L: float) -> np.ndarray:
    """K(G) = 4 pi / |G|^2 for G != 0 and 0 at G = 0 (neutralising
    background)."""
    g2 = g_squared(n, L)
    k = np.zeros_like(g2)
    nz = g2 > 0
    k[nz] = 4.0 * math.pi / g2[nz]
    return k


def hartree_energy(rho, L: float) -> float:
    """E_H = (Omega/2) sum_{G != 0} 4 pi |rho_hat(G)|^2 / |G|^2 with
    rho_hat = F(rho) / N^3 and F the forward DFT of Eq. 1."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[-1]
    assert rho.shape == (n, n, n)
    omega = L ** 3
    rho_hat = dft3d(rho.astype(np.complex128), -1) / float(n) ** 3
    return float(0.5 * omega * np.sum(hartree_kernel(n, L) * np.abs(rho_hat) ** 2))


def hartree_potential(rho, L: float) -> np.ndarray:
    """V_H(r_j) = sum_{G != 0} K(G) rho_hat(G) exp(+i G.r_j), i.e. the
    inverse DFT (sign +1) of K * rho_hat; real part returned."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[-1]
    rho_hat = dft3d(rho.astype(np.complex128), -1) / float(n) ** 3
    v = dft3d(hartree_kernel(n, L) * rho_hat, +1)
    return v.real.copy()


def hartree_gradient(rho, L: float) -> np.ndarray:
    """dE_H/drho_j = (Omega / N^3) V_H(r_j)."""
    n = np.asarray(rho).shape[-1]
    return (L ** 3 / float(n) ** 3) * hartree_potential(rho, L)


def analytic_rhohat_gaussians(n: int, L: float, centres, sigmas, weights) -> np.ndarray:
    """Fourier coefficients (1/Omega) int rho(r) exp(-i G.r) dr of the
    periodic density sum_k w_k (2 pi s_k^2)^(-3/2) exp(-|r - R_k|^2 / 2 s_k^2)
    on the n^3 set of G vectors: (1/Omega) sum_k w_k exp(-s_k^2 |G|^2 / 2)
    exp(-i G.R_k).  Shape (n, n, n) = (z, y, x)."""
    g = g_index(n).astype(np.float64) * (2.0 * math.pi / L)
    g2 = g_squared(n, L)
    out = np.zeros((n, n, n), dtype=np.complex128)
    for (cx, cy, cz), s, w in zip(np.asarray(centres), np.asarray(sigmas), np.asarray(weights)):
        ph = (np.exp(-1j * g * cz)[:, None, None] * np.exp(-1j * g * cy)[None, :, None]
              * np.exp(-1j * g * cx)[None, None, :])
        out += w * np.exp(-0.5 * s * s * g2) * ph
    return out / L ** 3
