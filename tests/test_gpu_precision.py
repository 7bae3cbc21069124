"""Tensor-core precision kinds of the radix-16 stage against the FP64
oracle and the plain FP32 path (Gaussian-sum grids).

Gate: split FP16 <= 1e-5 relative L2 against the oracle and against FP32 on
the same GPU.  Split BF16 and plain FP16 are reported (printed) and only
checked against loose sanity bounds."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

SPLIT_FP16_TOL = 1e-5


def _run(x, precision, inverse=False):
    from paper_2006_08435_gb300 import fft3d
    return fft3d(x, inverse=inverse, precision=precision)


@pytest.mark.parametrize("n,batch", [(64, 2), (128, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_split_fp16_gate_and_report(cuda, n, batch, inverse):
    x = synth.gaussian_sum_grids(n, batch, seed=7)
    xd = torch.from_numpy(x).cuda()
    sign = 1 if inverse else -1
    ref = oracle.dft3d(x.astype(np.complex128), sign)
    f32 = _run(xd, "fp32", inverse).cpu().numpy()
    report = {}
    for prec in ("split_fp16", "split_bf16", "fp16"):
        y = _run(xd, prec, inverse).cpu().numpy()
        report[prec] = max(oracle.rel_l2(y[b], ref[b]) for b in range(batch))
        report[prec + "_vs_fp32"] = max(oracle.rel_l2(y[b], f32[b]) for b in range(batch))
    report["fp32"] = max(oracle.rel_l2(f32[b], ref[b]) for b in range(batch))
    print(f"\nrel-L2 n={n} inverse={inverse}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in report.items()))
    assert report["split_fp16"] <= SPLIT_FP16_TOL
    assert report["split_fp16_vs_fp32"] <= SPLIT_FP16_TOL
    assert report["split_bf16"] < 1e-3
    assert report["fp16"] < 1e-2


def test_split_fp16_closed_forms(cuda):
    from paper_2006_08435_gb300 import fft3d
    n = 64
    d = torch.zeros((1, n, n, n), dtype=torch.complex64, device="cuda")
    d[0, 0, 0, 0] = 1.0
    y = fft3d(d, precision="split_fp16").cpu().numpy()
    assert np.abs(y - 1.0).max() < 1e-6
    c = torch.full((1, n, n, n), 3.0 - 1.0j, dtype=torch.complex64, device="cuda")
    y = fft3d(c, precision="split_fp16").cpu().numpy()
    expect = np.zeros((1, n, n, n), np.complex128)
    expect[0, 0, 0, 0] = (3.0 - 1.0j) * n ** 3
    assert oracle.rel_l2(y, expect) <= SPLIT_FP16_TOL


def test_split_fp16_round_trip_large_values(cuda):
    """Values up to n^3 max|f| (the forward result) go back through the
    inverse without FP16 overflow thanks to the per-vector scale."""
    from paper_2006_08435_gb300 import fft3d
    n = 128
    # a mean of 1 puts ~n^3 = 2.1e6 into the k = 0 bin
    x = torch.from_numpy(synth.uniform_grids(n, 1, seed=9) + 1.0).cuda()
    f = fft3d(x, precision="split_fp16")
    assert float(f.abs().max()) > 65504.0
    back = fft3d(f, inverse=True, norm="by_n", precision="split_fp16")
    assert oracle.rel_l2(back.cpu().numpy(), x.cpu().numpy()) <= 2 * SPLIT_FP16_TOL


def test_precision_unsupported_size_is_refused(cuda):
    from paper_2006_08435_gb300 import Plan, FFT3DError
    with pytest.raises(FFT3DError):
        Plan(48, 48, 48, 1, precision="split_fp16")


@pytest.mark.parametrize("variant", [0, 9])
@pytest.mark.parametrize("inverse", [False, True])
def test_precision_kinds_per_variant_64(cuda, monkeypatch, variant, inverse):
    """Each 64^3 tensor-core kernel (0 plain persistent, 9 two-plane
    tcgen05) for every precision kind, three grids (a ragged tail of
    plane-pair items), forward and normalised inverse."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", str(variant))
    n, batch = 64, 3
    x = torch.from_numpy(synth.gaussian_sum_grids(n, batch, seed=11 + variant)).cuda()
    ref = oracle.dft3d(x.cpu().numpy().astype(np.complex128), 1 if inverse else -1)
    norm = "by_n" if inverse else "none"
    if inverse:
        ref /= float(n) ** 3
    for prec, tol in (("split_fp16", SPLIT_FP16_TOL), ("split_bf16", 1e-3), ("fp16", 1e-2)):
        p = Plan(n, n, n, batch, precision=prec, inverse=inverse, norm=norm)
        assert p.variant == variant
        y = torch.empty_like(x)
        p.execute(x, y)
        assert p.device_status() == 0
        err = max(oracle.rel_l2(y[b].cpu().numpy(), ref[b]) for b in range(batch))
        print(f"\nvariant {variant} {prec} inverse={inverse}: rel-L2 {err:.2e}")
        assert err <= tol


def test_split_fp16_two_plane_in_place_many_grids(cuda, monkeypatch):
    """40 grids in place (every block goes several times round its tiles),
    each a multiple of the first, so one oracle transform checks three."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", "9")
    n, batch = 64, 40
    base = torch.from_numpy(synth.gaussian_sum_grids(n, 1, seed=5)).cuda()
    x = (base.repeat(batch, 1, 1, 1) *
         torch.arange(1, batch + 1, device="cuda", dtype=torch.float32).view(-1, 1, 1, 1)).contiguous()
    p = Plan(n, n, n, batch, precision="split_fp16")
    assert p.variant == 9
    p.execute(x, x)
    assert p.device_status() == 0
    ref0 = oracle.dft3d(base[0].cpu().numpy().astype(np.complex128), -1)
    for b in (0, batch // 2, batch - 1):
        assert oracle.rel_l2(x[b].cpu().numpy(), (b + 1) * ref0) <= SPLIT_FP16_TOL


def test_split_fp16_two_plane_closed_forms_and_range(cuda, monkeypatch):
    """The two-plane tcgen05 kernel on a delta (all-ones result), a
    constant (one bin), zero planes, and a round trip through values far
    above the FP16 range."""
    from paper_2006_08435_gb300 import fft3d
    monkeypatch.setenv("FFT3D_VARIANT", "9")
    n = 64
    d = torch.zeros((1, n, n, n), dtype=torch.complex64, device="cuda")
    d[0, 0, 0, 0] = 1.0
    y = fft3d(d, precision="split_fp16").cpu().numpy()
    assert np.abs(y - 1.0).max() < 1e-6
    c = torch.full((1, n, n, n), 3.0 - 1.0j, dtype=torch.complex64, device="cuda")
    y = fft3d(c, precision="split_fp16").cpu().numpy()
    expect = np.zeros((1, n, n, n), np.complex128)
    expect[0, 0, 0, 0] = (3.0 - 1.0j) * n ** 3
    assert oracle.rel_l2(y, expect) <= SPLIT_FP16_TOL
    x = torch.from_numpy(synth.uniform_grids(n, 1, seed=9) * 1e6 + 3e6).cuda()
    f = fft3d(x, precision="split_fp16")
    assert float(f.abs().max()) > 1e11
    back = fft3d(f, inverse=True, norm="by_n", precision="split_fp16")
    assert oracle.rel_l2(back.cpu().numpy(), x.cpu().numpy()) <= 2 * SPLIT_FP16_TOL


@pytest.mark.parametrize("n_grids", [1, 3, 40])
def test_tcgen05_kernel_all_kinds(cuda, monkeypatch, n_grids):
    """The tcgen05 two-plane 64^3 kernel (variant 9) for every precision kind,
    forward and normalised inverse: one grid, a ragged three, and 40 grids
    in place (each block goes several times round its tiles; the grids are
    multiples of the first, so one oracle transform checks them)."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", "9")
    n = 64
    base = torch.from_numpy(synth.gaussian_sum_grids(n, 1, seed=21)).cuda()
    x = (base.repeat(n_grids, 1, 1, 1) *
         torch.arange(1, n_grids + 1, device="cuda", dtype=torch.float32).view(-1, 1, 1, 1)).contiguous()
    ref0 = {s: oracle.dft3d(base[0].cpu().numpy().astype(np.complex128), s) for s in (-1, 1)}
    check = sorted({0, n_grids // 2, n_grids - 1})
    for prec, tol in (("split_fp16", SPLIT_FP16_TOL), ("split_bf16", 1e-3), ("fp16", 1e-2)):
        for inverse in (False, True):
            p = Plan(n, n, n, n_grids, precision=prec, inverse=inverse,
                     norm="by_n" if inverse else "none")
            assert p.variant == 9
            y = x.clone()
            p.execute(y, y)
            assert p.device_status() == 0
            ref = ref0[1] / float(n) ** 3 if inverse else ref0[-1]
            err = max(oracle.rel_l2(y[b].cpu().numpy(), (b + 1) * ref) for b in check)
            print(f"\ntcgen05 {prec} grids={n_grids} inverse={inverse}: rel-L2 {err:.2e}")
            assert err <= tol


@pytest.mark.parametrize("n_grids", [1, 5])
def test_tcgen05_128_kernel_all_kinds(cuda, monkeypatch, n_grids):
    """The tcgen05 split-y 128^3 kernel (variant 9) for every precision kind,
    forward and normalised inverse, in place; grids are multiples of the
    first, so one oracle transform checks them."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", "9")
    n = 128
    base = torch.from_numpy(synth.gaussian_sum_grids(n, 1, seed=23)).cuda()
    x = (base.repeat(n_grids, 1, 1, 1) *
         torch.arange(1, n_grids + 1, device="cuda", dtype=torch.float32).view(-1, 1, 1, 1)).contiguous()
    ref0 = {s: oracle.dft3d(base[0].cpu().numpy().astype(np.complex128), s) for s in (-1, 1)}
    check = sorted({0, n_grids - 1})
    for prec, tol in (("split_fp16", SPLIT_FP16_TOL), ("split_bf16", 1e-3), ("fp16", 1e-2)):
        for inverse in (False, True):
            p = Plan(n, n, n, n_grids, precision=prec, inverse=inverse,
                     norm="by_n" if inverse else "none")
            assert p.variant == 9
            y = x.clone()
            p.execute(y, y)
            assert p.device_status() == 0
            ref = ref0[1] / float(n) ** 3 if inverse else ref0[-1]
            err = max(oracle.rel_l2(y[b].cpu().numpy(), (b + 1) * ref) for b in check)
            print(f"\ntcgen05 128^3 {prec} grids={n_grids} inverse={inverse}: rel-L2 {err:.2e}")
            assert err <= tol
