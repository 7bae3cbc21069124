// Single-size persistent kernel for 32^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n32(int dir) {
  constexpr int T = fused_threads(32);
  return dir < 0 ? make_fused_info<T, -1, 32>() : make_fused_info<T, 1, 32>();
}

}  // namespace fft3d
