// Tensor-core (split FP16, split BF16, FP16) persistent kernels for 64^3
// grids: the radix-16 first step of each axis runs as mma.sync GEMMs.
#include "persistent.cuh"

namespace fft3d {

KernelInfo tc_kernel_info_n64(int dir, int prec) {
  constexpr int T = fused_threads(64);
  if (dir < 0) {
    if (prec == 1) return make_fused_info_prec<T, -1, 1, 64>();
    if (prec == 2) return make_fused_info_prec<T, -1, 2, 64>();
    return make_fused_info_prec<T, -1, 3, 64>();
  }
  if (prec == 1) return make_fused_info_prec<T, 1, 1, 64>();
  if (prec == 2) return make_fused_info_prec<T, 1, 2, 64>();
  return make_fused_info_prec<T, 1, 3, 64>();
}

}  // namespace fft3d
