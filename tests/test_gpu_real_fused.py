"""Parity of the dedicated real-grid kernels (16^3 .. 128^3, FP32:
half-length row transforms, no pairing) with the FP64 oracle, element by
element.

Bar: relative L2 error <= 5e-6 per grid, the FP32 tolerance of the complex
path.  Grids are independent draws (not scaled copies of one grid), so a
slip between grids shows as a wrong grid, not a wrong magnitude.  The pair
scheme, forced through FFT3D_REAL_PATH=pairs, is checked against the same
oracle on the same inputs."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6
EDGES = [16, 32, 64, 128]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel(got, ref):
    return oracle.rel_l2(np.asarray(got, dtype=np.complex128), ref)


def real_grids(N, batch, seed):
    return np.ascontiguousarray(synth.uniform_grids(N, batch, seed=seed).real.astype(np.float32))


def half_spectra(N, batch, seed):
    """Arbitrary half spectra: not Hermitian in the planes kx = 0 and n/2."""
    return np.ascontiguousarray(synth.uniform_grids((N, N, N // 2 + 1), batch, seed=seed))


def run(x, inverse=False, norm="none"):
    from paper_2006_08435_gb300 import RealPlan
    b, N = x.shape[0], x.shape[1]
    p = RealPlan(N, b, inverse=inverse, norm=norm)
    if inverse:
        out = torch.empty((b, N, N, N), dtype=torch.float32, device="cuda")
    else:
        out = torch.empty((b, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    p.execute(x, out)
    assert p.device_status() == 0
    p.close()
    return out


@pytest.mark.parametrize("N", EDGES)
@pytest.mark.parametrize("path", ["dedicated", "pairs"])
@pytest.mark.parametrize("batch", [1, 3])
def test_forward_against_oracle(cuda, monkeypatch, N, path, batch):
    if path == "pairs":
        monkeypatch.setenv("FFT3D_REAL_PATH", "pairs")
    r = real_grids(N, batch, seed=400 + batch)
    got = run(to_dev(r)).cpu().numpy()
    ref = oracle.rdft3d(r.astype(np.float64))
    errs = [rel(got[b], ref[b]) for b in range(batch)]
    assert max(errs) <= FP32_TOL, errs


@pytest.mark.parametrize("N", EDGES)
@pytest.mark.parametrize("path", ["dedicated", "pairs"])
def test_inverse_non_hermitian_against_oracle(cuda, monkeypatch, N, path):
    """Columns kx = 0 and n/2 not Hermitian: the oracle's Re of the inverse
    of the Hermitian extension; the input is left unchanged."""
    if path == "pairs":
        monkeypatch.setenv("FFT3D_REAL_PATH", "pairs")
    h = half_spectra(N, 3, seed=77)
    hd = to_dev(h)
    keep = hd.clone()
    got = run(hd, inverse=True).cpu().numpy()
    assert torch.equal(hd, keep)
    ref = oracle.irdft3d(h.astype(np.complex128), N)
    errs = [rel(got[b], ref[b]) for b in range(3)]
    assert max(errs) <= FP32_TOL, errs


@pytest.mark.parametrize("N", EDGES)
def test_special_inputs(cuda, N):
    """Closed forms through the dedicated kernels: a delta at the origin
    has a flat spectrum; a cosine along x with m cycles has n^3/2 at kx = m
    (ky = kz = 0) and nothing else; the Nyquist cosine (-1)^(x+y+z) has n^3
    at (n/2, n/2, n/2) -- the bin the packed Nyquist pencil carries."""
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    delta = np.zeros((N, N, N), np.float32)
    delta[0, 0, 0] = 1.0
    cosx = np.cos(2 * np.pi * 5 * x / N).astype(np.float32)
    nyq = ((-1.0) ** (x + y + z)).astype(np.float32)
    got = run(to_dev(np.stack([delta, cosx, nyq]))).cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got[0] - 1.0)) <= 1e-6
    e = np.zeros((N, N, N // 2 + 1), np.complex128)
    e[0, 0, 5] = N ** 3 / 2
    assert np.max(np.abs(got[1] - e)) <= 1e-6 * N ** 3
    e = np.zeros((N, N, N // 2 + 1), np.complex128)
    e[N // 2, N // 2, N // 2] = N ** 3
    assert np.max(np.abs(got[2] - e)) <= 1e-6 * N ** 3


@pytest.mark.parametrize("N", EDGES)
def test_norms_and_round_trip(cuda, N):
    r = real_grids(N, 2, seed=91)
    rd = to_dev(r)
    ref = oracle.rdft3d(r.astype(np.float64))
    fo = run(rd, norm="ortho").cpu().numpy()
    assert max(rel(fo[b], ref[b] / N ** 1.5) for b in range(2)) <= FP32_TOL
    fb = run(rd, norm="by_n")
    assert max(rel(fb[b].cpu().numpy(), ref[b] / N ** 3) for b in range(2)) <= FP32_TOL
    f = run(rd)
    back = run(f, inverse=True, norm="by_n").cpu().numpy()
    assert rel(back, r.astype(np.float64)) <= 2 * FP32_TOL
    bo = run(to_dev(fo.astype(np.complex64)), inverse=True, norm="ortho").cpu().numpy()
    assert rel(bo, r.astype(np.float64)) <= 2 * FP32_TOL


@pytest.mark.parametrize("N", EDGES)
def test_schedule_beyond_shared_table(cuda, N):
    """1100 grids: more schedule blocks (2200) than the kernel keeps in
    shared memory, so tickets are resolved from the global table.  Sampled
    grids against the oracle; every grid back through the inverse."""
    batch = 1100
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((batch, N, N, N), generator=gen, device="cuda", dtype=torch.float32)
    y = run(x)
    for b in (0, 517, batch - 1):
        ref = oracle.rdft3d(x[b].cpu().numpy().astype(np.float64))
        assert rel(y[b].cpu().numpy(), ref) <= FP32_TOL, b
    back = run(y, inverse=True, norm="by_n")
    err = (torch.linalg.vector_norm((back - x).reshape(batch, -1), dim=1)
           / torch.linalg.vector_norm(x.reshape(batch, -1), dim=1))
    assert float(err.max()) <= 2 * FP32_TOL


@pytest.mark.parametrize("N", EDGES)
def test_graph_capture(cuda, N):
    from paper_2006_08435_gb300 import RealPlan
    batch = 2
    fwd, inv = RealPlan(N, batch), RealPlan(N, batch, inverse=True, norm="by_n")
    xs = torch.zeros((batch, N, N, N), dtype=torch.float32, device="cuda")
    hs = torch.empty((batch, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    bs = torch.empty_like(xs)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fwd.execute(xs, hs)
        inv.execute(hs, bs)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fwd.execute(xs, hs)
        inv.execute(hs, bs)
    r = real_grids(N, batch, seed=12)
    xs.copy_(to_dev(r))
    g.replay()
    torch.cuda.synchronize()
    ref = oracle.rdft3d(r.astype(np.float64))
    assert max(rel(hs[b].cpu().numpy(), ref[b]) for b in range(batch)) <= FP32_TOL
    assert rel(bs.cpu().numpy(), r.astype(np.float64)) <= 2 * FP32_TOL
