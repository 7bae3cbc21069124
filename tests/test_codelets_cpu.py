"""The register DFT codelets of the kernels (csrc/codelets.cuh), compiled as
host code by nvcc and run on the CPU: every radix the kernels use, forward
and inverse, against numpy.fft on the same inputs (FP64).  The codelets'
twiddles are their own compile-time constants, so a wrong factorisation,
index or sign in any of them shows here without a GPU."""
import os
import subprocess

import numpy as np
import pytest

RADICES = [2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 24, 32, 40, 48, 64]

SRC = r"""
#include <cmath>
#include <cstdio>
#include "codelets.cuh"
using namespace fft3d;

template <int R, int DIR>
void one() {
  float2 v[R];
  for (int n = 0; n < R; ++n)
    v[n] = make_float2((float)std::cos(0.7 * n + 0.3), (float)std::sin(1.3 * n - 0.2));
  DFT<R, DIR>::run(v);
  std::printf("%d %d", R, DIR);
  for (int n = 0; n < R; ++n) std::printf(" %.9e %.9e", v[n].x, v[n].y);
  std::printf("\n");
}
template <int R>
void both() {
  one<R, -1>();
  one<R, 1>();
}
int main() {
  both<2>(); both<3>(); both<4>(); both<5>(); both<6>(); both<8>(); both<9>(); both<10>();
  both<12>(); both<15>(); both<16>(); both<24>(); both<32>(); both<40>(); both<48>(); both<64>();
  return 0;
}
"""


@pytest.fixture(scope="module")
def codelet_output(tmp_path_factory):
    from paper_2006_08435_gb300 import build as B
    cc = B.nvcc()
    if not cc or not os.path.exists(cc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("codelets")
    src = d / "codelets_host.cu"
    exe = d / "codelets_host"
    src.write_text(SRC)
    csrc = os.path.join(os.path.dirname(B.__file__), "csrc")
    subprocess.run([cc, "-std=c++17", "-O2", "-I", csrc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.strip().splitlines():
        f = line.split()
        r, sign = int(f[0]), int(f[1])
        vals = np.array([float(t) for t in f[2:]]).reshape(r, 2)
        res[(r, sign)] = vals[:, 0] + 1j * vals[:, 1]
    return res


@pytest.mark.slow
@pytest.mark.parametrize("r", RADICES)
@pytest.mark.parametrize("sign", [-1, 1])
def test_codelet_is_the_dft(codelet_output, r, sign):
    n = np.arange(r)
    x = np.cos(0.7 * n + 0.3).astype(np.float32).astype(np.float64) + \
        1j * np.sin(1.3 * n - 0.2).astype(np.float32).astype(np.float64)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * r
    got = codelet_output[(r, sign)]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
