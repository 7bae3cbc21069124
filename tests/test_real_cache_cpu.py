"""The real-plan cache of rfft3d / irfft3d keeps the few most recently used
plans and releases the others (each owns a large workspace).  CPU only: the
plan class is replaced by a stand-in that records releases."""
import contextlib

from paper_2006_08435_gb300 import fft


class _FakePlan:
    made, closed = [], []

    def __init__(self, n, batch, precision, inverse, norm):
        self.key = (n, batch, precision, inverse, norm)
        _FakePlan.made.append(self.key)

    def close(self):
        _FakePlan.closed.append(self.key)


def test_lru_bound_and_reuse(monkeypatch):
    monkeypatch.setattr(fft, "RealPlan", _FakePlan)
    monkeypatch.setattr(fft.torch.cuda, "device", lambda dev: contextlib.nullcontext())
    monkeypatch.setattr(fft, "_real_cache", fft.collections.OrderedDict())
    _FakePlan.made.clear()
    _FakePlan.closed.clear()
    get = fft._get_real_plan
    a = get(64, 2, "fp32", False, "none", 0)
    assert get(64, 2, "fp32", False, "none", 0) is a          # reused
    for b in range(3, 3 + fft._REAL_CACHE_MAX):
        get(64, b, "fp32", False, "none", 0)
    # one more than the bound: the least recently used (batch 2) went
    assert _FakePlan.closed == [(64, 2, "fp32", False, "none")]
    assert len(fft._real_cache) == fft._REAL_CACHE_MAX
    # using an entry makes it the most recent
    get(64, 3, "fp32", False, "none", 0)
    get(32, 1, "fp32", True, "by_n", 0)
    assert _FakePlan.closed[-1] == (64, 4, "fp32", False, "none")
    assert len(_FakePlan.made) == 2 + fft._REAL_CACHE_MAX


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
