"""The real-plan cache of rfft3d / irfft3d keeps the few most recently used
plans per (problem, device, stream) and forgets the others (each owns a
large workspace); a forgotten plan is released by its last holder, never
closed under a caller that may still be executing it.  CPU only: the plan
class is replaced by a stand-in."""
import contextlib
import gc
import weakref

from paper_2006_08435_gb300 import fft


class _FakePlan:
    made, closed = [], []

    def __init__(self, n, batch, precision, inverse, norm):
        self.key = (n, batch, precision, inverse, norm)
        _FakePlan.made.append(self.key)

    def close(self):
        _FakePlan.closed.append(self.key)


def _setup(monkeypatch):
    monkeypatch.setattr(fft, "RealPlan", _FakePlan)
    monkeypatch.setattr(fft.torch.cuda, "device", lambda dev: contextlib.nullcontext())
    monkeypatch.setattr(fft, "_real_cache", fft.collections.OrderedDict())
    _FakePlan.made.clear()
    _FakePlan.closed.clear()


def test_lru_bound_and_reuse(monkeypatch):
    _setup(monkeypatch)
    get = fft._get_real_plan
    a = get(64, 2, "fp32", False, "none", 0, 0)
    assert get(64, 2, "fp32", False, "none", 0, 0) is a          # reused
    for b in range(3, 3 + fft._REAL_CACHE_MAX):
        get(64, b, "fp32", False, "none", 0, 0)
    # one more than the bound: the least recently used (batch 2) left the
    # cache, but it is not closed while `a` still holds it
    assert len(fft._real_cache) == fft._REAL_CACHE_MAX
    assert all(p.key[1] != 2 for p in fft._real_cache.values())
    assert _FakePlan.closed == []
    # using an entry makes it the most recent
    get(64, 3, "fp32", False, "none", 0, 0)
    get(32, 1, "fp32", True, "by_n", 0, 0)
    assert all(p.key[1] != 4 for p in fft._real_cache.values())
    assert len(_FakePlan.made) == 2 + fft._REAL_CACHE_MAX


def test_evicted_plan_lives_until_its_last_holder_drops_it(monkeypatch):
    _setup(monkeypatch)
    get = fft._get_real_plan
    held = get(16, 1, "fp32", False, "none", 0, 0)
    ref = weakref.ref(held)
    for b in range(2, 2 + fft._REAL_CACHE_MAX):
        get(16, b, "fp32", False, "none", 0, 0)
    gc.collect()
    assert ref() is held                 # evicted, still usable by its holder
    del held
    gc.collect()
    assert ref() is None                 # released with its last reference


def test_plans_are_kept_per_stream(monkeypatch):
    _setup(monkeypatch)
    get = fft._get_real_plan
    a = get(16, 2, "fp32", False, "none", 0, 111)
    b = get(16, 2, "fp32", False, "none", 0, 222)
    assert a is not b
    assert get(16, 2, "fp32", False, "none", 0, 111) is a


def test_binding_rejects_host_tensors_and_wrong_dtypes():
    """The real-grid helpers check their arguments before any library call
    (so these run without a GPU)."""
    import pytest
    import torch
    with pytest.raises(TypeError):
        fft.rfft3d(torch.zeros(2, 8, 8, 8))                       # host tensor
    with pytest.raises(TypeError):
        fft.irfft3d(torch.zeros(2, 8, 8, 5, dtype=torch.complex64))
    with pytest.raises(TypeError):
        fft.rfft3d(torch.zeros(2, 8, 8, 8, dtype=torch.complex64))  # not real
