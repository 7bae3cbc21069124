// Single-size persistent kernel for 48^3 grids (forward and inverse).
#include "persistent.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n48(int dir) {
  constexpr int T = fused_threads(48);
  return dir < 0 ? make_fused_info<T, -1, 48>() : make_fused_info<T, 1, 48>();
}

}  // namespace fft3d
