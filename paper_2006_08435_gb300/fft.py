"""PyTorch-facing binding of the C ABI (``include/fft3d.h``).

Argument marshalling only: tensors are passed to the library as raw device
pointers plus the current CUDA stream; every step of the transform runs in
the library's sm_103a kernels.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import collections
import ctypes
import threading

import torch

from . import _lib as L

_PREC = {"fp32": L.FFT3D_FP32, "split_fp16": L.FFT3D_SPLIT_FP16,
         "split_bf16": L.FFT3D_SPLIT_BF16, "fp16": L.FFT3D_FP16, "bfp16": L.FFT3D_BFP16,
         "split_fp8": L.FFT3D_SPLIT_FP8, "fp8": L.FFT3D_FP8}
_NORM = {"none": L.FFT3D_NORM_NONE, "n": L.FFT3D_NORM_BY_N, "by_n": L.FFT3D_NORM_BY_N,
         "ortho": L.FFT3D_NORM_ORTHO}


# The current stream's raw handle and the current device, read without the
# Stream object and device-index normalisation of torch.cuda.current_stream()
# (a few microseconds of host time per call, several calls per transform);
# the public calls where these accessors are missing.
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_current_device = getattr(torch._C, "_cuda_getDevice", None)


def _current_stream_handle(device_index: int | None = None) -> int:
    """Raw handle of the current stream of `device_index` (default: the
    current device)."""
    if _raw_stream is not None and _current_device is not None:
        return int(_raw_stream(_current_device() if device_index is None else device_index))
    s = torch.cuda.current_stream() if device_index is None else torch.cuda.current_stream(device_index)
    return int(s.cuda_stream)


def _stream_handle(stream) -> int:
    if stream is None:
        return _current_stream_handle()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class _on_device:
    """Make `index` the current device for the block, switching only when
    it is not already (the launches must be issued on the stream's device)."""

    def __init__(self, index: int):
        self.index, self.prev = index, None

    def __enter__(self):
        cur = _current_device() if _current_device is not None else torch.cuda.current_device()
        if cur != self.index:
            self.prev = cur
            torch.cuda.set_device(self.index)

    def __exit__(self, *exc):
        if self.prev is not None:
            torch.cuda.set_device(self.prev)


def _check_tensor(t: torch.Tensor, name: str) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex64:
        raise TypeError(f"{name} must be complex64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def size_supported(n: int) -> bool:
    return bool(L.lib().fft3d_size_supported(int(n)))


def twiddle_table(n: int):
    """(L1, L2, table as a list of (re, im) FP32 pairs) the planner uses."""
    buf = (ctypes.c_float * (2 * n))()
    l1, l2 = ctypes.c_int(), ctypes.c_int()
    L.check(L.lib().fft3d_twiddle_table(int(n), buf, ctypes.byref(l1), ctypes.byref(l2)),
            "fft3d_twiddle_table")
    return l1.value, l2.value, [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]


class Plan:
    """A plan for ``batch`` grids of nz x ny x nx complex64 points.

    ``execute(x, out)`` computes Eq. 1 per grid on the current stream."""

    def __init__(self, nx: int, ny: int, nz: int, batch: int = 1, precision: str = "fp32",
                 inverse: bool = False, norm: str = "none"):
        self.shape = (int(nz), int(ny), int(nx))
        self.batch = int(batch)
        self.precision, self.inverse, self.norm = precision, bool(inverse), norm
        h = ctypes.c_void_p()
        L.check(L.lib().fft3d_plan_create(int(nx), int(ny), int(nz), int(batch), _PREC[precision],
                                          L.FFT3D_INVERSE if inverse else L.FFT3D_FORWARD,
                                          _NORM[norm], ctypes.byref(h)), "fft3d_plan_create")
        self._h = h

    @property
    def handle(self) -> int:
        return self._h.value or 0

    @property
    def variant(self) -> int:
        v = ctypes.c_int()
        L.check(L.lib().fft3d_plan_variant(self._h, ctypes.byref(v)), "fft3d_plan_variant")
        return v.value

    def execute(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        _check_tensor(x, "x")
        _check_tensor(out, "out")
        need = self.batch * self.shape[0] * self.shape[1] * self.shape[2]
        if x.numel() != need or out.numel() != need:
            raise ValueError(f"expected {need} points, got {x.numel()} and {out.numel()}")
        L.check(L.lib().fft3d_execute(self._h, x.data_ptr(), out.data_ptr(), _stream_handle(stream)),
                "fft3d_execute")
        return out

    def enable_host_io(self, chunk_grids: int | None = None) -> None:
        """Allocate the staging of execute_host (default: ~32 MB chunks)."""
        if chunk_grids is None:
            grid_bytes = 8 * self.shape[0] * self.shape[1] * self.shape[2]
            chunk_grids = max(1, min(self.batch, (32 << 20) // grid_bytes))
        L.check(L.lib().fft3d_plan_host_io(self._h, int(chunk_grids)), "fft3d_plan_host_io")

    def execute_host(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """x, out: complex64 CPU tensors (pin them for overlapped copies)."""
        for t, name in ((x, "x"), (out, "out")):
            if t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex64 CPU tensor")
        need = self.batch * self.shape[0] * self.shape[1] * self.shape[2]
        if x.numel() != need or out.numel() != need:
            raise ValueError(f"expected {need} points")
        L.check(L.lib().fft3d_execute_host(self._h, x.data_ptr(), out.data_ptr(),
                                           _stream_handle(stream)), "fft3d_execute_host")
        return out

    def device_status(self, stream=None) -> int:
        return L.lib().fft3d_get_device_status(self._h, _stream_handle(stream))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().fft3d_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MixedPlan:
    """Cubic grids of different edges transformed in one persistent launch."""

    def __init__(self, dims, precision: str = "fp32", inverse: bool = False, norm: str = "none"):
        self.dims = [int(d) for d in dims]
        arr = (ctypes.c_int * len(self.dims))(*self.dims)
        h = ctypes.c_void_p()
        L.check(L.lib().fft3d_plan_create_mixed(len(self.dims), arr, _PREC[precision],
                                                L.FFT3D_INVERSE if inverse else L.FFT3D_FORWARD,
                                                _NORM[norm], ctypes.byref(h)),
                "fft3d_plan_create_mixed")
        self._h = h
        self.offsets = []
        for g in range(len(self.dims) + 1):
            o = ctypes.c_int64()
            L.check(L.lib().fft3d_plan_grid_offset(self._h, g, ctypes.byref(o)), "grid_offset")
            self.offsets.append(o.value)
        self.total_points = self.offsets[-1]

    def execute(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """Packed buffers: grid g occupies points [offsets[g], offsets[g+1])."""
        _check_tensor(x, "x")
        _check_tensor(out, "out")
        if x.numel() != self.total_points or out.numel() != self.total_points:
            raise ValueError("packed buffers must hold exactly total_points points")
        L.check(L.lib().fft3d_execute(self._h, x.data_ptr(), out.data_ptr(), _stream_handle(stream)),
                "fft3d_execute")
        return out

    @property
    def variant(self) -> int:
        v = ctypes.c_int()
        L.check(L.lib().fft3d_plan_variant(self._h, ctypes.byref(v)), "fft3d_plan_variant")
        return v.value

    def execute_ptrs(self, in_ptrs: torch.Tensor, out_ptrs: torch.Tensor, stream=None) -> None:
        """``in_ptrs``/``out_ptrs``: int64 CUDA tensors of per-grid device pointers."""
        for t in (in_ptrs, out_ptrs):
            if not (t.is_cuda and t.dtype == torch.int64 and t.numel() == len(self.dims)):
                raise ValueError("pointer arrays must be int64 CUDA tensors, one per grid")
        L.check(L.lib().fft3d_execute_mixed(self._h, in_ptrs.data_ptr(), out_ptrs.data_ptr(),
                                            _stream_handle(stream)), "fft3d_execute_mixed")

    def device_status(self, stream=None) -> int:
        return L.lib().fft3d_get_device_status(self._h, _stream_handle(stream))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().fft3d_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RealPlan:
    """A plan for ``batch`` transforms of real n^3 grids.

    Forward: ``execute(x, out)`` with x float32 (batch, n, n, n) and out
    complex64 (batch, n, n, n // 2 + 1), the half spectrum of Eq. 1.
    Inverse (``inverse=True``): x is the half spectrum and out the float32
    grids, the real part of the inverse transform of the Hermitian extension.
    At 16^3 .. 128^3 in FP32 the library runs dedicated real-grid kernels (a
    whole grid per block at 16^3 and 32^3); elsewhere
    two grids share one complex transform."""

    def __init__(self, n: int, batch: int = 1, precision: str = "fp32", inverse: bool = False,
                 norm: str = "none"):
        self.n, self.batch = int(n), int(batch)
        self.precision, self.inverse, self.norm = precision, bool(inverse), norm
        h = ctypes.c_void_p()
        L.check(L.lib().fft3d_real_plan_create(self.n, self.batch, _PREC[precision],
                                               L.FFT3D_INVERSE if inverse else L.FFT3D_FORWARD,
                                               _NORM[norm], ctypes.byref(h)),
                "fft3d_real_plan_create")
        self._h = h

    def _check(self, t: torch.Tensor, name: str, dtype, points: int) -> None:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype or not t.is_contiguous():
            raise TypeError(f"{name} must be contiguous {dtype}")
        if t.numel() != points:
            raise ValueError(f"{name}: expected {points} elements, got {t.numel()}")

    def execute(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        n, b = self.n, self.batch
        real_pts, half_pts = b * n * n * n, b * n * n * (n // 2 + 1)
        if self.inverse:
            self._check(x, "x", torch.complex64, half_pts)
            self._check(out, "out", torch.float32, real_pts)
        else:
            self._check(x, "x", torch.float32, real_pts)
            self._check(out, "out", torch.complex64, half_pts)
        L.check(L.lib().fft3d_real_execute(self._h, x.data_ptr(), out.data_ptr(),
                                           _stream_handle(stream)), "fft3d_real_execute")
        return out

    def device_status(self, stream=None) -> int:
        return L.lib().fft3d_real_get_device_status(self._h, _stream_handle(stream))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().fft3d_real_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plan_cache: dict = {}
_cache_lock = threading.Lock()


def get_plan(nx, ny, nz, batch, precision="fp32", inverse=False, norm="none", device=None,
             stream=None) -> Plan:
    """The cached plan for this problem on this device AND stream: a plan's
    work counters and status word may serve one stream at a time (executes
    that overlap on two streams would share them), so each stream gets its
    own plan."""
    dev = torch.cuda.current_device() if device is None else device
    key = (nx, ny, nz, batch, precision, bool(inverse), norm, dev, _stream_handle(stream))
    with _cache_lock:
        p = _plan_cache.get(key)
        if p is None:
            with torch.cuda.device(dev):
                p = Plan(nx, ny, nz, batch, precision, inverse, norm)
            _plan_cache[key] = p
    return p


def fft3d(x: torch.Tensor, inverse: bool = False, norm: str = "none", precision: str = "fp32",
          out: torch.Tensor | None = None) -> torch.Tensor:
    """3D DFT (Eq. 1) over the last three dims (nz, ny, nx) of a complex64
    CUDA tensor; leading dims are a batch.  Forward uses exp(-2 pi i/n),
    ``inverse=True`` exp(+2 pi i/n); ``norm`` in {"none", "by_n", "ortho"}."""
    _check_tensor(x, "x")
    if x.dim() < 3:
        raise ValueError("need (..., nz, ny, nx)")
    nz, ny, nx = x.shape[-3:]
    batch = x.numel() // (nz * ny * nx) if x.numel() else 0
    if out is None:
        out = torch.empty_like(x)
    if batch == 0:
        return out
    dev = x.device.index
    with _on_device(dev):
        stream = _current_stream_handle(dev)
        plan = get_plan(nx, ny, nz, batch, precision, inverse, norm, dev, stream)
        return plan.execute(x, out, stream)


# Real plans of the pair scheme own a workspace of ceil(batch/2) n^3 complex
# points (268 MB at 128^3 x 32), so only the most recently used few are kept.  An evicted plan
# is only dropped from the cache, not closed: a caller in another thread may
# still be executing it, and its memory is released (plan destroy, whose
# cudaFree waits for work still using it) once the last reference to it
# goes.  Like complex plans, real plans are kept per stream.
_REAL_CACHE_MAX = 4
_real_cache: "collections.OrderedDict" = collections.OrderedDict()


def _get_real_plan(n, batch, precision, inverse, norm, dev, stream=None) -> RealPlan:
    key = (n, batch, precision, bool(inverse), norm, dev, _stream_handle(stream))
    with _cache_lock:
        p = _real_cache.get(key)
        if p is not None:
            _real_cache.move_to_end(key)
            return p
        with torch.cuda.device(dev):
            p = RealPlan(n, batch, precision, inverse, norm)
        _real_cache[key] = p
        while len(_real_cache) > _REAL_CACHE_MAX:
            _real_cache.popitem(last=False)
    return p


def rfft3d(x: torch.Tensor, norm: str = "none", precision: str = "fp32",
           out: torch.Tensor | None = None) -> torch.Tensor:
    """Half spectrum (..., n, n, n // 2 + 1) of the forward transform (Eq. 1)
    of real float32 CUDA grids (..., n, n, n); leading dims are a batch."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32:
        raise TypeError("x must be a float32 CUDA tensor")
    if x.dim() < 3 or not (x.shape[-1] == x.shape[-2] == x.shape[-3]):
        raise ValueError("need cubic (..., n, n, n)")
    n = x.shape[-1]
    x = x.contiguous()
    batch = x.numel() // (n ** 3) if x.numel() else 0
    if out is None:
        out = torch.empty(x.shape[:-1] + (n // 2 + 1,), dtype=torch.complex64, device=x.device)
    if batch == 0:
        return out
    dev = x.device.index
    with _on_device(dev):
        stream = _current_stream_handle(dev)
        p = _get_real_plan(n, batch, precision, False, norm, dev, stream)
        return p.execute(x, out, stream)


def irfft3d(x: torch.Tensor, norm: str = "none", precision: str = "fp32",
            out: torch.Tensor | None = None) -> torch.Tensor:
    """Real float32 grids (..., n, n, n) from half spectra (..., n, n,
    n // 2 + 1): the real part of the inverse transform (exponent +1) of the
    Hermitian extension; ``x`` is not modified."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.complex64:
        raise TypeError("x must be a complex64 CUDA tensor")
    if x.dim() < 3 or x.shape[-2] != x.shape[-3] or x.shape[-1] != x.shape[-2] // 2 + 1:
        raise ValueError("need (..., n, n, n // 2 + 1)")
    n = x.shape[-2]
    x = x.contiguous()
    batch = x.numel() // (n * n * (n // 2 + 1)) if x.numel() else 0
    if out is None:
        out = torch.empty(x.shape[:-1] + (n,), dtype=torch.float32, device=x.device)
    if batch == 0:
        return out
    dev = x.device.index
    with _on_device(dev):
        stream = _current_stream_handle(dev)
        p = _get_real_plan(n, batch, precision, True, norm, dev, stream)
        return p.execute(x, out, stream)


class FFT3d(torch.autograd.Function):
    """y = F(x) with F the unnormalised forward transform of Eq. 1.

    Backward is the adjoint F^H, i.e. the unnormalised transform with the
    conjugate root exp(+2 pi i/n), run by the same kernels.  (PyTorch's
    convention for complex gradients makes grad_x = F^H grad_y for a linear
    map.)"""

    @staticmethod
    def forward(ctx, x, precision="fp32"):
        ctx.precision = precision
        return fft3d(x.contiguous(), inverse=False, precision=precision)

    @staticmethod
    def backward(ctx, g):
        return fft3d(g.contiguous(), inverse=True, precision=ctx.precision), None


def autotune(n: int, batch: int, precision: str = "fp32", inverse: bool = False,
             cache_path: str | None = None) -> int:
    """Time the kernel variants of an n^3 x batch plan on the current device
    and return (and record in ``cache_path``) the fastest."""
    best = ctypes.c_int()
    L.check(L.lib().fft3d_autotune(int(n), int(batch), _PREC[precision],
                                   L.FFT3D_INVERSE if inverse else L.FFT3D_FORWARD,
                                   cache_path.encode() if cache_path else None, ctypes.byref(best)),
            "fft3d_autotune")
    return best.value


def autotune_mixed(dims, inverse: bool = False, cache_path: str | None = None) -> int:
    arr = (ctypes.c_int * len(dims))(*[int(d) for d in dims])
    best = ctypes.c_int()
    L.check(L.lib().fft3d_autotune_mixed(len(dims), arr,
                                         L.FFT3D_INVERSE if inverse else L.FFT3D_FORWARD,
                                         cache_path.encode() if cache_path else None,
                                         ctypes.byref(best)), "fft3d_autotune_mixed")
    return best.value


def selftest_wait_timeout(timeout_ns: int = 1_000_000) -> int:
    """Run the bounded-wait self test (a wait on a flag nobody sets); returns
    the library's code, FFT3D_ERR_DEVICE_TIMEOUT when the wait gave up."""
    return L.lib().fft3d_selftest_wait_timeout(int(timeout_ns))
