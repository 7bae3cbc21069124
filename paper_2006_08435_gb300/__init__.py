"""GB300-native (sm_103a) batched 3D complex-to-complex FFT.

The hot path of Ramaswami et al., "Efficient Ab-Initio Molecular Dynamic
Simulations by Offloading Fast Fourier Transformations to FPGAs": the 3D DFT
of Eq. 1 computed as 1D FFTs along x, then y, then z, behind the C ABI of
``include/fft3d.h`` (``libfft3d.so``).  This package is a thin binding:

* ``fft3d(x, inverse=False, norm="none", precision="fp32")``
* ``Plan`` / ``MixedPlan`` -- explicit plans (batched / mixed edges)
* ``rfft3d`` / ``irfft3d`` / ``RealPlan`` -- real grids (half spectra)
* ``FFT3d`` -- autograd Function whose backward is the adjoint transform
* ``hartree_energy`` -- plane-wave Hartree energy with an adjoint-FFT gradient

Importing the package does not load the CUDA library; the first call does,
and raises if it has not been built (there is no CPU fallback).
"""
from ._lib import FFT3DError  # noqa: F401

__all__ = ["fft3d", "Plan", "MixedPlan", "FFT3d", "FFT3DError", "size_supported",
           "rfft3d", "irfft3d", "RealPlan",
           "hartree_energy", "HartreeEnergy"]


def __getattr__(name):
    if name in ("fft3d", "Plan", "MixedPlan", "FFT3d", "size_supported", "get_plan",
                "rfft3d", "irfft3d", "RealPlan",
                "twiddle_table", "selftest_wait_timeout", "autotune", "autotune_mixed"):
        from . import fft as _fft
        return getattr(_fft, name)
    if name in ("hartree_energy", "HartreeEnergy"):
        from . import hartree as _h
        return getattr(_h, name)
    raise AttributeError(name)
