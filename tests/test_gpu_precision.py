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
