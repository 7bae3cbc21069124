// Single-size kernels for 128^3 grids (forward and inverse): the plain
// persistent kernel (variant 0), the warp-owned two-phase kernel (5, the
// fastest for one grid) and the split-y kernel with 64 KB items (6, the
// fastest from two grids; x and z by thread pairs in registers).
#include "splity.cuh"
#include "warpown.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n128(int dir, int variant) {
  constexpr int T = fused_threads(128);
  if (variant == 6) return dir < 0 ? sy::info<128, -1>() : sy::info<128, 1>();
  if (variant == 5) return dir < 0 ? wown::info<128, -1>() : wown::info<128, 1>();
  return dir < 0 ? make_fused_info<T, -1, 128>() : make_fused_info<T, 1, 128>();
}

}  // namespace fft3d
