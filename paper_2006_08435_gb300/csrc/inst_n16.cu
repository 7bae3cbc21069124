// Single-size persistent kernel for 16^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n16(int dir) {
  constexpr int T = fused_threads(16);
  return dir < 0 ? make_fused_info<T, -1, 16>() : make_fused_info<T, 1, 16>();
}

}  // namespace fft3d
