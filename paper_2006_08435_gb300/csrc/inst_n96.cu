// Single-size persistent kernel for 96^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n96(int dir) {
  constexpr int T = fused_threads(96);
  return dir < 0 ? make_fused_info<T, -1, 96>() : make_fused_info<T, 1, 96>();
}

}  // namespace fft3d
