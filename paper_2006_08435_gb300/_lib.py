"""ctypes loader for ``libfft3d.so``.  Argument marshalling only.

The library is the CUDA product path; there is no fallback.  If it has not
been built, every entry point raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfft3d.so")

FFT3D_FP32, FFT3D_SPLIT_FP16, FFT3D_SPLIT_BF16, FFT3D_FP16 = 0, 1, 2, 3
FFT3D_BFP16, FFT3D_SPLIT_FP8, FFT3D_FP8 = 4, 5, 6
FFT3D_FORWARD, FFT3D_INVERSE = -1, 1
FFT3D_NORM_NONE, FFT3D_NORM_BY_N, FFT3D_NORM_ORTHO = 0, 1, 2
FFT3D_SUCCESS = 0
FFT3D_ERR_INVALID_ARG = -1
FFT3D_ERR_UNSUPPORTED_SIZE = -2
FFT3D_ERR_NULL_PTR = -3
FFT3D_ERR_MISALIGNED = -4
FFT3D_ERR_CUDA = -5
FFT3D_ERR_DEVICE_TIMEOUT = -6
FFT3D_ERR_ALLOC = -7
FFT3D_ERR_NO_DEVICE = -8
FFT3D_ERR_UNSUPPORTED_PRECISION = -9
FFT3D_ERR_EXCEEDS_STATIC_SCRATCH = -10
FFT3D_NOALLOC_MAX_BATCH = 4096

# name -> (restype, argtypes); every symbol include/fft3d.h declares
_VP = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "fft3d_size_supported": (_I, [_I]),
    "fft3d_axis_digit_map": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "fft3d_twiddle_table": (_I, [_I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "fft3d_tc_operand_table": (_I, [_I, ctypes.POINTER(ctypes.c_uint16)]),
    "fft3d_plan_create": (_I, [_I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(_VP)]),
    "fft3d_plan_create_mixed": (_I, [_I, ctypes.POINTER(_I), _I, _I, _I, ctypes.POINTER(_VP)]),
    "fft3d_plan_grid_offset": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_int64)]),
    "fft3d_execute": (_I, [_VP, _VP, _VP, _VP]),
    "fft3d_execute_mixed": (_I, [_VP, _VP, _VP, _VP]),
    "fft3d_get_device_status": (_I, [_VP, _VP]),
    "fft3d_plan_destroy": (_I, [_VP]),
    "fft3d_error_string": (ctypes.c_char_p, [_I]),
    "fft3d_selftest_wait_timeout": (_I, [ctypes.c_int64]),
    "fft3d_execute_noalloc": (_I, [_I, _I, _I, _I, _VP, _VP, _VP]),
    "fft3d_noalloc_get_device_status": (_I, [_VP]),
    "fft3d_hartree_workspace_bytes": (ctypes.c_size_t, [_I, _I]),
    "fft3d_hartree_energy": (_I, [_VP, _I, _I, ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP]),
    "fft3d_hartree_seed": (_I, [_VP, _I, _I, ctypes.c_double, _VP, _VP, _VP]),
    "fft3d_hartree_energy_half": (_I, [_VP, _I, _I, ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP]),
    "fft3d_hartree_seed_half": (_I, [_VP, _I, _I, ctypes.c_double, _VP, _VP, _VP]),
    "fft3d_real_to_complex": (_I, [_VP, _VP, ctypes.c_int64, _VP]),
    "fft3d_plan_variant": (_I, [_VP, ctypes.POINTER(_I)]),
    "fft3d_plan_host_io": (_I, [_VP, _I]),
    "fft3d_execute_host": (_I, [_VP, _VP, _VP, _VP]),
    "fft3d_tune_select": (_I, [ctypes.c_char_p, _I, ctypes.POINTER(_I), _VP, _VP, ctypes.c_char_p,
                               ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "fft3d_autotune": (_I, [_I, _I, _I, _I, ctypes.c_char_p, ctypes.POINTER(_I)]),
    "fft3d_autotune_mixed": (_I, [_I, ctypes.POINTER(_I), _I, ctypes.c_char_p, ctypes.POINTER(_I)]),
    "fft3d_complex_to_real": (_I, [_VP, _VP, ctypes.c_int64, _VP]),
    "fft3d_schedule_preview": (_I, [_I, ctypes.POINTER(_I), _I, ctypes.c_double, _I, _I,
                                   ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                   ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "fft3d_real_plan_create": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(_VP)]),
    "fft3d_real_execute": (_I, [_VP, _VP, _VP, _VP]),
    "fft3d_real_get_device_status": (_I, [_VP, _VP]),
    "fft3d_real_plan_destroy": (_I, [_VP]),
}

_lib = None
_lock = threading.Lock()


def exported_symbols() -> list[str]:
    return list(_SIGS)


def lib() -> ctypes.CDLL:
    """Load the library (once).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is not built; the CUDA path has no fallback. "
                    "Build it with `python -m paper_2006_08435_gb300.build` "
                    "or `__graft_entry__.build()`.")
            l = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


# fft3d_tune_timer: double (*)(int variant, void* ctx)
TUNE_TIMER = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int, ctypes.c_void_p)


class FFT3DError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        msg = lib().fft3d_error_string(code).decode()
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")
        self.code = code


def check(code: int, where: str = "") -> None:
    if code != FFT3D_SUCCESS:
        raise FFT3DError(code, where)
