// Tensor-core (split FP16, split BF16, FP16) persistent kernels for 128^3
// grids: the radix-16 first step of each axis runs as mma.sync GEMMs.
#include "persistent.cuh"

namespace fft3d {

KernelInfo tc_kernel_info_n128(int dir, int prec, int /*variant*/) {
  constexpr int T = fused_threads(128);
  if (dir < 0) {
    if (prec == 1) return make_fused_info_prec<T, -1, 1, 128>();
    if (prec == 2) return make_fused_info_prec<T, -1, 2, 128>();
    return make_fused_info_prec<T, -1, 3, 128>();
  }
  if (prec == 1) return make_fused_info_prec<T, 1, 1, 128>();
  if (prec == 2) return make_fused_info_prec<T, 1, 2, 128>();
  return make_fused_info_prec<T, 1, 3, 128>();
}

}  // namespace fft3d
