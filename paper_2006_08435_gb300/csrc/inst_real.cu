// Real-grid kernels: forward (R2C) and inverse (C2R), whole grids per block
// at 16^3 and 32^3 (rwholegrid.cuh), two-phase kernels at 64^3 and 128^3
// (rgrid.cuh).
#include "rgrid.cuh"
#include "rwholegrid.cuh"

namespace fft3d {

KernelInfo real_kernel_info(int n, int dir) {
  if (n == 16) return dir < 0 ? rwg::info<16, -1>() : rwg::info<16, 1>();
  if (n == 32) return dir < 0 ? rwg::info<32, -1>() : rwg::info<32, 1>();
  if (n == 64) return dir < 0 ? rg::info<64, -1>() : rg::info<64, 1>();
  if (n == 128) return dir < 0 ? rg::info<128, -1>() : rg::info<128, 1>();
  return KernelInfo{};
}

}  // namespace fft3d
