"""Autotuner selection and cache logic (fft3d_tune_select) with a fake
timer: no GPU needed."""
import ctypes
import json

from paper_2006_08435_gb300 import _lib as L


def _select(lib, key, cands, times, cache, calls):
    def timer(variant, ctx):
        calls.append(variant)
        return times[variant]
    cb = L.TUNE_TIMER(timer)
    arr = (ctypes.c_int * len(cands))(*cands)
    best, from_cache = ctypes.c_int(-7), ctypes.c_int(-7)
    rc = lib.fft3d_tune_select(key.encode(), len(cands), arr, ctypes.cast(cb, ctypes.c_void_p),
                               None, cache.encode() if cache else None, ctypes.byref(best),
                               ctypes.byref(from_cache))
    return rc, best.value, from_cache.value


def test_picks_fastest_and_caches(fft3d_lib, tmp_path):
    cache = str(tmp_path / "tune.json")
    calls = []
    rc, best, fc = _select(fft3d_lib, "devA|n128|b32", [0, 1, 2], {0: 3.0, 1: 5.0, 2: 1.5}, cache, calls)
    assert rc == 0 and best == 2 and fc == 0 and calls == [0, 1, 2]
    assert json.load(open(cache)) == {"devA|n128|b32": 2}
    calls.clear()
    rc, best, fc = _select(fft3d_lib, "devA|n128|b32", [0, 1, 2], {0: 0.1, 1: 0.1, 2: 9.0}, cache, calls)
    assert rc == 0 and best == 2 and fc == 1 and calls == []
    # another key is tuned and merged into the same file
    rc, best, fc = _select(fft3d_lib, "devA|n64|b256", [0, 1], {0: 1.0, 1: 2.0}, cache, calls)
    assert best == 0 and fc == 0
    assert json.load(open(cache)) == {"devA|n128|b32": 2, "devA|n64|b256": 0}


def test_failed_candidates_and_ties(fft3d_lib):
    calls = []
    rc, best, _ = _select(fft3d_lib, "k", [0, 1, 2], {0: -1.0, 1: 2.0, 2: 2.0}, None, calls)
    assert rc == 0 and best == 1
    rc, _, _ = _select(fft3d_lib, "k", [0, 1], {0: -1.0, 1: float("nan")}, None, [])
    assert rc == L.FFT3D_ERR_CUDA


def test_cached_value_outside_candidates_is_retuned(fft3d_lib, tmp_path):
    cache = tmp_path / "t.json"
    cache.write_text('{"k": 5}')
    calls = []
    rc, best, fc = _select(fft3d_lib, "k", [0, 1], {0: 2.0, 1: 1.0}, str(cache), calls)
    assert best == 1 and fc == 0 and calls == [0, 1]
    assert json.load(open(cache)) == {"k": 1}


def test_corrupt_cache_is_ignored_and_rewritten(fft3d_lib, tmp_path):
    cache = tmp_path / "t.json"
    cache.write_text('{"k": oops, "other": 1, "k2": }')
    rc, best, fc = _select(fft3d_lib, "k", [0, 1], {0: 2.0, 1: 1.0}, str(cache), [])
    assert rc == 0 and best == 1 and fc == 0
    assert json.load(open(cache)) == {"k": 1, "other": 1}


def test_argument_checks(fft3d_lib):
    arr = (ctypes.c_int * 1)(0)
    best = ctypes.c_int()
    assert fft3d_lib.fft3d_tune_select(None, 1, arr, None, None, None, ctypes.byref(best),
                                       None) == L.FFT3D_ERR_NULL_PTR
    cb = L.TUNE_TIMER(lambda v, c: 1.0)
    assert fft3d_lib.fft3d_tune_select(b"k", 0, arr, ctypes.cast(cb, ctypes.c_void_p), None, None,
                                       ctypes.byref(best), None) == L.FFT3D_ERR_INVALID_ARG
    assert fft3d_lib.fft3d_plan_variant(None, ctypes.byref(best)) == L.FFT3D_ERR_NULL_PTR
