// Single-size persistent kernel for 64^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n64(int dir) {
  constexpr int T = fused_threads(64);
  return dir < 0 ? make_fused_info<T, -1, 64>() : make_fused_info<T, 1, 64>();
}

}  // namespace fft3d
