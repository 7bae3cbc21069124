"""fft3d_execute_noalloc, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc at the moment they need a transform --
for example a solver loop whose framework hands out all device memory up
front.  fft3d_execute_noalloc serves them from a fixed device array inside
the library instead of a plan's buffers.  These tests call it through the C
ABI and check that it gives what the planned path (fft3d_plan_create +
fft3d_execute) gives and what the FP64 oracle gives, on two calls in a row
(the array keeps the previous call's contents, so the second call shows
that it starts clean), that its status word reads clean after a normal
call, and that it refuses a batch larger than the array can hold.

This file is collected last so that a failure here does not hide the other
GPU tests in a run that stops at the first failure."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import _lib as L
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6


def rel_l2(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def call_noalloc(lib, x, out, n, batch, direction, norm):
    return lib.fft3d_execute_noalloc(n, batch, direction, norm, x.data_ptr(), out.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)


# the plain persistent kernel at (64, 3), (128, 2), (48, 2); (16, 300): 600
# schedule blocks (several words of the phase bits
# the set-up kernel expands) with slab blocks interleaved among the planes
@pytest.mark.parametrize("n,batch", [(64, 3), (128, 2), (48, 2), (16, 300)])
def test_matches_planned_path_and_oracle_on_two_calls(cuda, n, batch):
    from paper_2006_08435_gb300 import Plan
    lib = L.lib()
    sample = sorted({0, batch // 2, batch - 1})
    for call, (inverse, norm) in enumerate([(False, "none"), (True, "by_n")]):
        x = torch.from_numpy(synth.uniform_grids(n, batch, seed=100 + call)).to("cuda")
        want = torch.empty_like(x)
        Plan(n, n, n, batch, inverse=inverse, norm=norm).execute(x, want)
        got = torch.full_like(x, float("nan"))
        rc = call_noalloc(lib, x, got, n, batch, L.FFT3D_INVERSE if inverse else L.FFT3D_FORWARD,
                          L.FFT3D_NORM_BY_N if norm == "by_n" else L.FFT3D_NORM_NONE)
        assert rc == L.FFT3D_SUCCESS
        stream = torch.cuda.current_stream().cuda_stream
        assert lib.fft3d_noalloc_get_device_status(stream) == L.FFT3D_SUCCESS
        assert rel_l2(got, want) <= FP32_TOL
        xs = x[sample].cpu().numpy().astype(np.complex128)
        ref = oracle.dft3d(xs, 1 if inverse else -1)
        if norm == "by_n":
            ref /= float(n) ** 3
        g = got[sample].cpu().numpy()
        for i in range(len(sample)):
            assert oracle.rel_l2(g[i], ref[i]) <= FP32_TOL


def test_rejects_batch_beyond_the_static_array(cuda):
    lib = L.lib()
    buf = torch.zeros(16 ** 3, dtype=torch.complex64, device="cuda")
    rc = call_noalloc(lib, buf, buf, 16, L.FFT3D_NOALLOC_MAX_BATCH + 1, L.FFT3D_FORWARD,
                      L.FFT3D_NORM_NONE)
    assert rc == L.FFT3D_ERR_EXCEEDS_STATIC_SCRATCH
    assert "static scratch" in lib.fft3d_error_string(rc).decode()
