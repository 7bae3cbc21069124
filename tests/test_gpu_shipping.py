"""The kernels the library ships as defaults, at the benchmark's sizes.

* In place on the 128^3 split-y kernels (FP32 variant 6, tensor-core variant
  9): a plane's two half-plane items read and write overlapping rows, so
  the in-place result must equal the out-of-place one bit for bit on every
  grid (same kernel, same arithmetic), and match the FP64 oracle on sampled
  grids.  Grids are distinct iid draws, so a slip between grids cannot hide
  behind a common structure.
* The split-FP16 gate (<= 1e-5 relative L2 against the oracle AND against
  plain FP32 on the same GPU) on the tcgen05 kernels at 64^3 x 16 and
  128^3 x 32, Gaussian-sum grids; split BF16 and plain FP16 reported.
* Two streams transforming the same shape at once through fft3d().
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6
SPLIT_FP16_TOL = 1e-5


def _sample(batch, k=8):
    return sorted({int(round(i * (batch - 1) / (k - 1))) for i in range(k)})


@pytest.mark.parametrize("variant,precision,tol", [(6, "fp32", FP32_TOL),
                                                   (9, "split_fp16", SPLIT_FP16_TOL)])
@pytest.mark.parametrize("inverse", [False, True])
def test_in_place_128_split_y_full_batch(cuda, monkeypatch, variant, precision, tol, inverse):
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", str(variant))
    n, batch = 128, 32
    x = torch.from_numpy(synth.uniform_grids(n, batch, seed=300 + variant)).cuda()
    norm = "by_n" if inverse else "none"
    p = Plan(n, n, n, batch, precision=precision, inverse=inverse, norm=norm)
    assert p.variant == variant
    out_of_place = torch.empty_like(x)
    p.execute(x, out_of_place)
    y = x.clone()
    for _ in range(2):  # the second round goes through the transform again in place
        y.copy_(x)
        p.execute(y, y)
        assert p.device_status() == 0
        assert torch.equal(y, out_of_place)
    sample = _sample(batch)
    ref = oracle.dft3d(x[sample].cpu().numpy().astype(np.complex128), 1 if inverse else -1)
    if inverse:
        ref /= float(n) ** 3
    got = y[sample].cpu().numpy()
    errs = [oracle.rel_l2(got[i], ref[i]) for i in range(len(sample))]
    print(f"\nin place variant {variant} {precision} inverse={inverse}: max rel-L2 {max(errs):.2e}")
    assert max(errs) <= tol


@pytest.mark.parametrize("n,batch", [(64, 16), (128, 32)])
def test_split_fp16_gate_on_tcgen05_kernels(cuda, monkeypatch, n, batch):
    from paper_2006_08435_gb300 import Plan
    x = torch.from_numpy(synth.gaussian_sum_grids(n, batch, seed=40 + n)).cuda()
    sample = _sample(batch)
    ref = oracle.dft3d(x[sample].cpu().numpy().astype(np.complex128), -1)
    f32 = torch.empty_like(x)
    Plan(n, n, n, batch).execute(x, f32)
    f32s = f32[sample].cpu().numpy()
    report = {"fp32": max(oracle.rel_l2(f32s[i], ref[i]) for i in range(len(sample)))}
    monkeypatch.setenv("FFT3D_VARIANT", "9")
    for prec in ("split_fp16", "split_bf16", "fp16"):
        p = Plan(n, n, n, batch, precision=prec)
        assert p.variant == 9
        y = torch.empty_like(x)
        p.execute(x, y)
        assert p.device_status() == 0
        ys = y[sample].cpu().numpy()
        per = [oracle.rel_l2(ys[i], ref[i]) for i in range(len(sample))]
        report[prec] = max(per)
        report[prec + "_vs_fp32"] = max(oracle.rel_l2(ys[i], f32s[i]) for i in range(len(sample)))
        print(f"\n{n}^3 x {batch} {prec} rel-L2 per sampled transform: " +
              " ".join(f"{e:.2e}" for e in per))
    print(f"\n{n}^3 x {batch}: " + ", ".join(f"{k} {v:.2e}" for k, v in report.items()))
    assert report["fp32"] <= FP32_TOL
    assert report["split_fp16"] <= SPLIT_FP16_TOL
    assert report["split_fp16_vs_fp32"] <= SPLIT_FP16_TOL
    assert report["split_bf16"] < 1e-3
    assert report["fp16"] < 1e-2


def test_two_streams_same_shape(cuda):
    """fft3d() keeps one plan per stream, so two streams transforming the
    same shape at the same time do not share work counters."""
    from paper_2006_08435_gb300 import Plan, fft3d
    n, batch = 64, 24
    xs = [torch.from_numpy(synth.uniform_grids(n, batch, seed=500 + i)).cuda() for i in range(2)]
    want = []
    for x in xs:
        w = torch.empty_like(x)
        Plan(n, n, n, batch).execute(x, w)
        want.append(w)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.empty_like(xs[0]), torch.empty_like(xs[1])]
    for _ in range(20):
        for s, x, o in zip(streams, xs, outs):
            with torch.cuda.stream(s):
                fft3d(x, out=o)
    torch.cuda.synchronize()
    for o, w in zip(outs, want):
        assert torch.equal(o, w)
