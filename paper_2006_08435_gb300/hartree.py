"""Plane-wave Hartree energy and its gradient through the C ABI.

E_H(rho) = (Omega/2) sum_{G != 0} 4 pi |rho_hat(G)|^2 / |G|^2 with
rho_hat = F(rho) / n^3 for a periodic cubic cell of side L (bohr); the
gradient dE_H/drho = (Omega/n^3) V_H is the adjoint (inverse, unnormalised)
transform of the seed s F(rho) / |m|^2.  Every step runs in the library's
kernels.  For even n (the usual grids) the density being real, the path
works on half spectra: real-grid forward transform, FP64 energy reduction
over the half spectrum (mirrored points counted twice); seed on the half
spectrum, real-grid inverse transform.  For odd n: real->complex, complex
forward transform, full-spectrum reduction; seed, complex inverse,
complex->real.  To capture a step in a CUDA graph, run it once eagerly
first with the same shapes and stream: that call allocates the reduction
workspace and the transform plans and has the library query its kernels'
occupancy, none of which belongs in a capture.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .fft import _stream_handle, fft3d, irfft3d, rfft3d

_ws_cache: dict = {}


def _workspace(n: int, batch: int, device) -> torch.Tensor:
    """Reduction workspace (partial sums and counters), one per (problem,
    device, stream): calls on two streams must not share the counters."""
    key = (n, batch, device, _stream_handle(None))
    ws = _ws_cache.get(key)
    if ws is None:
        nbytes = int(L.lib().fft3d_hartree_workspace_bytes(n, batch))
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _ws_cache[key] = ws
    return ws


def real_to_complex(x: torch.Tensor) -> torch.Tensor:
    if x.dtype != torch.float32 or not x.is_cuda:
        raise TypeError("float32 CUDA tensor expected")
    x = x.contiguous()
    out = torch.empty(x.shape, dtype=torch.complex64, device=x.device)
    L.check(L.lib().fft3d_real_to_complex(x.data_ptr(), out.data_ptr(), x.numel(),
                                          _stream_handle(None)), "fft3d_real_to_complex")
    return out


def complex_to_real(z: torch.Tensor) -> torch.Tensor:
    if z.dtype != torch.complex64 or not z.is_cuda:
        raise TypeError("complex64 CUDA tensor expected")
    z = z.contiguous()
    out = torch.empty(z.shape, dtype=torch.float32, device=z.device)
    L.check(L.lib().fft3d_complex_to_real(z.data_ptr(), out.data_ptr(), z.numel(),
                                          _stream_handle(None)), "fft3d_complex_to_real")
    return out


def energy_from_spectrum(rhohat: torch.Tensor, cell: float) -> torch.Tensor:
    """E_H per grid from rhohat = F(rho) (complex64, (..., n, n, n)); FP64."""
    n = rhohat.shape[-1]
    batch = rhohat.numel() // n ** 3
    rhohat = rhohat.contiguous()
    e = torch.empty(batch, dtype=torch.float64, device=rhohat.device)
    ws = _workspace(n, batch, rhohat.device)
    L.check(L.lib().fft3d_hartree_energy(rhohat.data_ptr(), n, batch, float(cell), e.data_ptr(),
                                         ws.data_ptr(), ws.numel(), _stream_handle(None)),
            "fft3d_hartree_energy")
    return e.reshape(rhohat.shape[:-3])


def energy_from_half_spectrum(rhohat_half: torch.Tensor, cell: float) -> torch.Tensor:
    """E_H per grid from the half spectrum rfft3d(rho) (complex64,
    (..., n, n, n // 2 + 1), n even); FP64."""
    n = rhohat_half.shape[-2]
    batch = rhohat_half.numel() // (n * n * (n // 2 + 1))
    rhohat_half = rhohat_half.contiguous()
    e = torch.empty(batch, dtype=torch.float64, device=rhohat_half.device)
    ws = _workspace(n, batch, rhohat_half.device)
    L.check(L.lib().fft3d_hartree_energy_half(rhohat_half.data_ptr(), n, batch, float(cell),
                                              e.data_ptr(), ws.data_ptr(), ws.numel(),
                                              _stream_handle(None)), "fft3d_hartree_energy_half")
    return e.reshape(rhohat_half.shape[:-3])


def seed_from_half_spectrum(rhohat_half: torch.Tensor, cell: float,
                            grad_e: torch.Tensor) -> torch.Tensor:
    n = rhohat_half.shape[-2]
    batch = rhohat_half.numel() // (n * n * (n // 2 + 1))
    g = grad_e.to(torch.float64).contiguous().reshape(-1)
    if g.numel() != batch:
        raise ValueError("one gradient per grid")
    seed = torch.empty_like(rhohat_half)
    L.check(L.lib().fft3d_hartree_seed_half(rhohat_half.data_ptr(), n, batch, float(cell),
                                            g.data_ptr(), seed.data_ptr(), _stream_handle(None)),
            "fft3d_hartree_seed_half")
    return seed


def seed_from_spectrum(rhohat: torch.Tensor, cell: float, grad_e: torch.Tensor) -> torch.Tensor:
    n = rhohat.shape[-1]
    batch = rhohat.numel() // n ** 3
    g = grad_e.to(torch.float64).contiguous().reshape(-1)
    if g.numel() != batch:
        raise ValueError("one gradient per grid")
    seed = torch.empty_like(rhohat)
    L.check(L.lib().fft3d_hartree_seed(rhohat.data_ptr(), n, batch, float(cell), g.data_ptr(),
                                       seed.data_ptr(), _stream_handle(None)),
            "fft3d_hartree_seed")
    return seed


class HartreeEnergy(torch.autograd.Function):
    """E_H(rho) for real densities rho of shape (..., n, n, n), float32 CUDA.
    Returns FP64 energies of shape rho.shape[:-3]; backward returns
    dL/drho = grad_E * dE_H/drho (float32) through the adjoint FFT."""

    @staticmethod
    def forward(ctx, rho, cell):
        ctx.cell = float(cell)
        ctx.half = rho.shape[-1] % 2 == 0
        if ctx.half:
            rhohat = rfft3d(rho.contiguous())
            ctx.save_for_backward(rhohat)
            return energy_from_half_spectrum(rhohat, cell)
        rhohat = fft3d(real_to_complex(rho))
        ctx.save_for_backward(rhohat)
        return energy_from_spectrum(rhohat, cell)

    @staticmethod
    def backward(ctx, grad_e):
        (rhohat,) = ctx.saved_tensors
        if ctx.half:
            seed = seed_from_half_spectrum(rhohat, ctx.cell, grad_e)
            return irfft3d(seed), None
        seed = seed_from_spectrum(rhohat, ctx.cell, grad_e)
        return complex_to_real(fft3d(seed, inverse=True)), None


def hartree_energy(rho: torch.Tensor, cell: float) -> torch.Tensor:
    return HartreeEnergy.apply(rho, cell)
