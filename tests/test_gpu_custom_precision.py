"""Custom operand precisions of the tensor-core kernels (the paper names
custom-precision floating-point units as future work, section "Results"):
block floating point FP16 (one exponent per 64-point pencil, 11-bit
fixed-point mantissas), split FP8 (E4M3 hi + lo) and FP8, next to the
gated split FP16, split BF16, FP16 and FP32, on Gaussian-sum grids (the
precision workload's inputs) against the FP64 oracle.

The error study: relative L2 error per transform of every kind, printed
(run with -s), with the bounds asserted here; the orderings the formats'
resolutions predict are checked too (FP32 < split FP16 < split BF16 <
FP16, split FP16 < block floating point, split FP8 < FP8)."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

KINDS = ["fp32", "split_fp16", "split_bf16", "fp16", "bfp16", "split_fp8", "fp8"]
# generous bounds around the measured errors (the study reports the values)
BOUND = {"fp32": 5e-6, "split_fp16": 1e-5, "split_bf16": 1e-3, "fp16": 1e-2, "bfp16": 1e-2,
         "split_fp8": 3e-2, "fp8": 2e-1}


@pytest.mark.parametrize("n,batch", [(64, 16), (128, 4)])
@pytest.mark.parametrize("inverse", [False, True])
def test_error_study(cuda, n, batch, inverse):
    from paper_2006_08435_gb300 import Plan
    x = torch.from_numpy(synth.gaussian_sum_grids(n, batch, seed=60 + n)).cuda()
    ref = oracle.dft3d(x.cpu().numpy().astype(np.complex128), 1 if inverse else -1)
    norm = "by_n" if inverse else "none"
    if inverse:
        ref /= float(n) ** 3
    errs = {}
    for kind in KINDS:
        p = Plan(n, n, n, batch, precision=kind, inverse=inverse, norm=norm)
        if kind not in ("fp32",):
            assert p.variant == 9
        y = torch.empty_like(x)
        p.execute(x, y)
        assert p.device_status() == 0
        yc = y.cpu().numpy()
        errs[kind] = [oracle.rel_l2(yc[b], ref[b]) for b in range(batch)]
        print(f"\n{n}^3 x {batch} inverse={inverse} {kind:>10}: rel-L2 per transform "
              + " ".join(f"{e:.2e}" for e in errs[kind]))
    for kind in KINDS:
        assert max(errs[kind]) <= BOUND[kind], (kind, max(errs[kind]))
    worst = {k: max(v) for k, v in errs.items()}
    assert worst["fp32"] < worst["split_fp16"] < worst["split_bf16"] < worst["fp16"]
    assert worst["split_fp16"] < worst["bfp16"]
    assert worst["split_fp8"] < worst["fp8"]


@pytest.mark.parametrize("kind,tol", [("bfp16", 1e-2), ("split_fp8", 3e-2), ("fp8", 2e-1)])
def test_custom_kinds_closed_forms_and_round_trip(cuda, kind, tol):
    """A delta gives all ones and a constant one bin (both exact in every
    format after the per-pencil exponent); a round trip of a grid with a
    large mean goes through values far above the FP8 range."""
    from paper_2006_08435_gb300 import fft3d
    n = 64
    d = torch.zeros((1, n, n, n), dtype=torch.complex64, device="cuda")
    d[0, 0, 0, 0] = 1.0
    y = fft3d(d, precision=kind).cpu().numpy()
    assert np.abs(y - 1.0).max() <= tol
    c = torch.full((1, n, n, n), 3.0 - 1.0j, dtype=torch.complex64, device="cuda")
    y = fft3d(c, precision=kind).cpu().numpy()
    expect = np.zeros((1, n, n, n), np.complex128)
    expect[0, 0, 0, 0] = (3.0 - 1.0j) * n ** 3
    assert oracle.rel_l2(y, expect) <= tol
    x = torch.from_numpy(synth.uniform_grids(n, 2, seed=9) + 1.0).cuda()
    f = fft3d(x, precision=kind)
    assert float(f.abs().max()) > 448.0
    back = fft3d(f, inverse=True, norm="by_n", precision=kind)
    assert oracle.rel_l2(back.cpu().numpy(), x.cpu().numpy()) <= 2 * tol


@pytest.mark.parametrize("kind", ["bfp16", "split_fp8", "fp8"])
def test_custom_kinds_in_place_128_many_grids(cuda, kind):
    """The 128^3 tcgen05 kernel with the custom kinds, in place, 12 distinct
    grids: the in-place result equals the out-of-place one bit for bit."""
    from paper_2006_08435_gb300 import Plan
    n, batch = 128, 12
    x = torch.from_numpy(synth.uniform_grids(n, batch, seed=77)).cuda()
    p = Plan(n, n, n, batch, precision=kind)
    y = torch.empty_like(x)
    p.execute(x, y)
    z = x.clone()
    p.execute(z, z)
    assert p.device_status() == 0
    assert torch.equal(y, z)
    ref = oracle.dft3d(x[batch - 1].cpu().numpy().astype(np.complex128), -1)
    assert oracle.rel_l2(y[batch - 1].cpu().numpy(), ref) <= BOUND[kind]


def test_custom_kinds_refused_elsewhere(cuda):
    from paper_2006_08435_gb300 import FFT3DError, Plan
    for kind in ("bfp16", "split_fp8", "fp8"):
        with pytest.raises(FFT3DError):
            Plan(32, 32, 32, 2, precision=kind)
        with pytest.raises(FFT3DError):
            Plan(64, 128, 96, 1, precision=kind)
