// Single-size persistent kernel for 80^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n80(int dir) {
  constexpr int T = fused_threads(80);
  return dir < 0 ? make_fused_info<T, -1, 80>() : make_fused_info<T, 1, 80>();
}

}  // namespace fft3d
