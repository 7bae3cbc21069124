// Single-size persistent kernel for 128^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n128(int dir) {
  constexpr int T = fused_threads(128);
  return dir < 0 ? make_fused_info<T, -1, 128>() : make_fused_info<T, 1, 128>();
}

}  // namespace fft3d
