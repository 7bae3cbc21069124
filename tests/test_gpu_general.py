"""The general path (variant 10): non-cubic grids and edges without a fused
kernel, up to 512 -- one pencil pass per axis -- against the FP64 oracle.

Small and medium shapes are checked on every output; 256^3 on whole grids;
512^3 on single outputs computed one by one from the definition
(oracle.dft3d_points), a plane wave's closed form and a round trip."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6


def _grids(shape, batch, seed):
    return torch.from_numpy(synth.uniform_grids(shape, batch, seed=seed)).cuda()


def _check_all(x, y, sign, norm_pts=None):
    ref = oracle.dft3d(x.cpu().numpy().astype(np.complex128), sign)
    if norm_pts:
        ref /= norm_pts
    yc = y.cpu().numpy()
    errs = [oracle.rel_l2(yc[b], ref[b]) for b in range(x.shape[0])]
    return max(errs)


# (nz, ny, nx): non-cubic mixes of radices 2, 3, 5, odd edges, tiny edges,
# an x extent that is not a multiple of the 16-pencil tile
SHAPES = [(96, 128, 64), (2, 3, 5), (5, 6, 8), (27, 10, 12), (16, 48, 250), (9, 25, 45),
          (40, 40, 40), (100, 4, 3), (3, 512, 2), (81, 2, 18)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("inverse", [False, True])
def test_non_cubic_against_oracle(cuda, shape, inverse):
    from paper_2006_08435_gb300 import Plan
    nz, ny, nx = shape
    batch = 3
    x = _grids(shape, batch, seed=sum(shape))
    norm = "by_n" if inverse else "none"
    p = Plan(nx, ny, nz, batch, inverse=inverse, norm=norm)
    assert p.variant == 10
    y = torch.empty_like(x)
    p.execute(x, y)
    err = _check_all(x, y, 1 if inverse else -1, nx * ny * nz if inverse else None)
    assert err <= FP32_TOL, err
    # in place gives the same bits
    z = x.clone()
    p.execute(z, z)
    assert torch.equal(z, y)


def test_chunks_and_tail(cuda):
    """Enough grids for several L2-sized chunks and a shorter last one;
    sampled grids (first, a middle one, the last) against the oracle, ortho
    normalisation."""
    from paper_2006_08435_gb300 import Plan
    nz, ny, nx = 96, 128, 64
    batch = 19
    x = _grids((nz, ny, nx), batch, seed=7)
    p = Plan(nx, ny, nz, batch, norm="ortho")
    y = torch.empty_like(x)
    p.execute(x, y)
    sample = [0, 9, batch - 1]
    ref = oracle.dft3d(x[sample].cpu().numpy().astype(np.complex128), -1) / np.sqrt(nx * ny * nz)
    yc = y[sample].cpu().numpy()
    for i in range(len(sample)):
        assert oracle.rel_l2(yc[i], ref[i]) <= FP32_TOL


@pytest.mark.parametrize("n,batch", [(64, 3), (128, 2), (48, 2), (16, 5)])
def test_general_variant_on_fused_sizes(cuda, monkeypatch, n, batch):
    """The general path forced on cubic edges that have fused kernels
    agrees with the oracle (and so with the fused kernels)."""
    from paper_2006_08435_gb300 import Plan
    monkeypatch.setenv("FFT3D_VARIANT", "10")
    x = _grids(n, batch, seed=n)
    p = Plan(n, n, n, batch)
    assert p.variant == 10
    y = torch.empty_like(x)
    p.execute(x, y)
    assert _check_all(x, y, -1) <= FP32_TOL


@pytest.mark.parametrize("n", [100, 243])
def test_cubic_edges_without_fused_kernel(cuda, n):
    from paper_2006_08435_gb300 import fft3d
    x = _grids(n, 1, seed=n)
    y = fft3d(x)
    assert _check_all(x, y, -1) <= FP32_TOL


def test_256_cubed_full_grids(cuda):
    from paper_2006_08435_gb300 import fft3d
    n = 256
    x = torch.from_numpy(synth.gaussian_sum_grids(n, 2, seed=256)).cuda()
    y = fft3d(x)
    assert _check_all(x, y, -1) <= FP32_TOL
    back = fft3d(y, inverse=True, norm="by_n")
    assert oracle.rel_l2(back.cpu().numpy(), x.cpu().numpy()) <= 2 * FP32_TOL


def test_512_cubed_sampled_outputs_closed_form_round_trip(cuda):
    from paper_2006_08435_gb300 import fft3d
    n = 512
    x = _grids(n, 1, seed=512)
    y = fft3d(x)
    rng = np.random.default_rng(5)
    pts = np.stack([rng.integers(0, n, 12) for _ in range(3)], axis=1)
    pts[0] = (0, 0, 0)
    pts[1] = (n - 1, n // 2, 1)
    want = oracle.dft3d_points(x[0].cpu().numpy(), pts, -1)
    yc = y[0].cpu().numpy()
    got = yc[pts[:, 0], pts[:, 1], pts[:, 2]]
    # per output, relative to the transform's RMS magnitude (sqrt(n^3) for
    # unit-variance entries)
    rms = float(np.sqrt(np.mean(np.abs(yc.astype(np.complex128)) ** 2)))
    assert np.max(np.abs(got - want)) <= 2e-5 * rms
    back = fft3d(y, inverse=True, norm="by_n")
    assert oracle.rel_l2(back.cpu().numpy(), x.cpu().numpy()) <= 2 * FP32_TOL
    del back, y
    # a plane wave: n^3 at k0, zero elsewhere
    k0 = (3, 500, 17)
    ar = torch.arange(n, device="cuda", dtype=torch.float64)
    ph = (2 * np.pi * (k0[0] * ar.view(-1, 1, 1) + k0[1] * ar.view(1, -1, 1)
                       + k0[2] * ar.view(1, 1, -1)) / n)
    f = torch.polar(torch.ones_like(ph), ph).to(torch.complex64).unsqueeze(0)
    del ph
    F = fft3d(f)
    peak = F[0, k0[0], k0[1], k0[2]].item()
    assert abs(peak - n ** 3) <= 1e-5 * n ** 3
    F[0, k0[0], k0[1], k0[2]] = 0
    assert float(F.abs().max()) <= 1e-5 * n ** 3


@pytest.mark.parametrize("n", [256])
def test_real_grids_on_the_general_path(cuda, n):
    """Real grids of an edge without a fused kernel: the half spectra of a
    pair through the general path, against the oracle's real transform."""
    from paper_2006_08435_gb300 import irfft3d, rfft3d
    r = np.ascontiguousarray(synth.uniform_grids(n, 2, seed=9).real.astype(np.float32))
    rd = torch.from_numpy(r).cuda()
    h = rfft3d(rd)
    ref = oracle.rdft3d(r[:1].astype(np.float64))
    assert oracle.rel_l2(h[0].cpu().numpy(), ref[0]) <= FP32_TOL
    back = irfft3d(h, norm="by_n")
    assert oracle.rel_l2(back.cpu().numpy(), r.astype(np.float64)) <= 2 * FP32_TOL


def test_general_path_in_a_graph(cuda):
    """The general path's launches (three per chunk) are captured and
    replayed."""
    from paper_2006_08435_gb300 import Plan
    nz, ny, nx = 20, 36, 30
    p = Plan(nx, ny, nz, 4)
    x = torch.zeros((4, nz, ny, nx), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.execute(x, y)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p.execute(x, y)
    x.copy_(_grids((nz, ny, nx), 4, seed=3))
    g.replay()
    torch.cuda.synchronize()
    assert _check_all(x, y, -1) <= FP32_TOL
