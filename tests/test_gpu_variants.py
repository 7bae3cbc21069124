"""Every kernel variant of every edge it applies to, against the FP64
oracle: 0 plain persistent, 1 twice the threads (16^3 .. 96^3), 3
cluster-fused single pass (16^3, 32^3), 4 double-buffered persistent
(32^3, 48^3, 80^3, 96^3), 5 warp-owned two-phase (64^3, 128^3), 6 split-y
(128^3), 7 and 8 thread-per-pencil one- and two-plane (64^3), 12
whole grid per block (16^3), 13 thread-pair planes (32^3 .. 96^3).  Odd batch
sizes leave a ragged tail of work items / clusters."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6
CASES = [(n, v) for n in (16, 32, 48, 64, 80, 96) for v in (0, 1)] + [(128, 0)]
CASES += [(16, 3), (32, 3), (16, 12)]
CASES += [(32, 4), (48, 4), (80, 4), (96, 4), (64, 5), (128, 5), (64, 7), (64, 8), (128, 6)]
CASES += [(32, 13), (48, 13), (80, 13), (96, 13)]


@pytest.mark.parametrize("n,variant", CASES)
def test_variant_matches_oracle(cuda, monkeypatch, n, variant):
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", str(variant))
    batch = 3 if n <= 64 else 2
    x = torch.from_numpy(synth.uniform_grids(n, batch, seed=30 + n + variant)).cuda()
    for inverse, norm in ((False, "none"), (True, "by_n")):
        p = Plan(n, n, n, batch, inverse=inverse, norm=norm)
        assert p.variant == variant
        y = torch.empty_like(x)
        p.execute(x, y)
        assert p.device_status() == 0
        ref = oracle.dft3d(x.cpu().numpy().astype(np.complex128), 1 if inverse else -1)
        if norm == "by_n":
            ref /= float(n) ** 3
        yc = y.cpu().numpy()
        for b in range(batch):
            assert oracle.rel_l2(yc[b], ref[b]) <= FP32_TOL


@pytest.mark.parametrize("n,variant", [(16, 3), (32, 3), (16, 12), (64, 7), (64, 8), (128, 6),
                                       (32, 13), (48, 13), (80, 13), (96, 13)])
def test_variant_in_place_and_many_grids(cuda, monkeypatch, n, variant):
    """More grids than blocks or clusters (every block goes many times round
    its tiles or loops over grids) and in == out."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", str(variant))
    batch = {48: 300, 64: 200, 80: 100, 96: 60, 128: 40}.get(n, 700)
    x = torch.from_numpy(synth.uniform_grids(n, 1, seed=n)).cuda().repeat(batch, 1, 1, 1)
    x = (x * torch.arange(1, batch + 1, device="cuda").view(-1, 1, 1, 1)).contiguous()
    ref0 = oracle.dft3d(x[0].cpu().numpy().astype(np.complex128), -1)
    p = Plan(n, n, n, batch)
    p.execute(x, x)
    assert p.device_status() == 0
    for b in (0, batch // 2, batch - 1):
        assert oracle.rel_l2(x[b].cpu().numpy(), (b + 1) * ref0) <= FP32_TOL


@pytest.mark.parametrize("variant", [7, 8])
def test_tensor_kernels_schedule_beyond_shared_table(cuda, monkeypatch, variant):
    """More schedule blocks (2 per grid) than the tensor-TMA kernels keep in
    shared memory (8192): the producer reads the schedule from global
    memory instead.  4100 grids of 64^3 (8.6 GB each way); three of them are
    checked against the oracle."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", str(variant))
    n, batch = 64, 4100
    base = torch.from_numpy(synth.uniform_grids(n, 1, seed=77)).cuda()
    x = base.repeat(batch, 1, 1, 1)
    x.mul_(torch.arange(1, batch + 1, device="cuda", dtype=torch.float32).view(-1, 1, 1, 1))
    y = torch.empty_like(x)
    p = Plan(n, n, n, batch)
    assert p.variant == variant
    p.execute(x, y)
    assert p.device_status() == 0
    ref0 = oracle.dft3d(base[0].cpu().numpy().astype(np.complex128), -1)
    for b in (0, 2049, batch - 1):
        assert oracle.rel_l2(y[b].cpu().numpy(), (b + 1) * ref0) <= FP32_TOL
    del x, y
    torch.cuda.empty_cache()


def test_thread_pair_kernel_schedule_beyond_shared_table(cuda, monkeypatch):
    """More schedule blocks (2 per grid) than the thread-pair kernel keeps in
    shared memory (4096): 2100 grids of 32^3 (four-plane items), the
    producer reads the schedule from global memory; three grids against the
    oracle."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", "13")
    n, batch = 32, 2100
    base = torch.from_numpy(synth.uniform_grids(n, 1, seed=78)).cuda()
    x = base.repeat(batch, 1, 1, 1)
    x.mul_(torch.arange(1, batch + 1, device="cuda", dtype=torch.float32).view(-1, 1, 1, 1))
    y = torch.empty_like(x)
    p = Plan(n, n, n, batch)
    assert p.variant == 13
    p.execute(x, y)
    assert p.device_status() == 0
    ref0 = oracle.dft3d(base[0].cpu().numpy().astype(np.complex128), -1)
    for b in (0, 1049, batch - 1):
        assert oracle.rel_l2(y[b].cpu().numpy(), (b + 1) * ref0) <= FP32_TOL


@pytest.mark.parametrize("n,variant,precision,batch",
                         [(64, 8, "fp32", 64), (128, 6, "fp32", 8), (96, 13, "fp32", 8),
                          (80, 13, "fp32", 8), (64, 9, "split_fp16", 64),
                          (128, 9, "split_fp16", 8)])
def test_back_to_back_launches_stay_live(cuda, monkeypatch, n, variant, precision, batch):
    """Thousands of launches in a row of the kernels whose three tiles serve
    two compute groups in turn (a tile barrier per group and tile): no
    bounded wait may time out, and the last result equals the first."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", str(variant))
    x = torch.from_numpy(synth.uniform_grids(n, batch, seed=41)).cuda()
    y = torch.empty_like(x)
    p = Plan(n, n, n, batch, precision=precision)
    assert p.variant == variant
    p.execute(x, y)
    first = y.clone()
    for _ in range(2000):
        p.execute(x, y)
    assert p.device_status() == 0
    assert torch.equal(y, first)
