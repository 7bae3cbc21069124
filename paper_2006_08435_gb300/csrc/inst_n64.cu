// Single-size kernels for 64^3 grids (forward and inverse): the plain
// persistent kernel in two block sizes (variant 0, and 1 with twice the
// threads per block: more warps to hide latency, fewer registers per
// thread), the warp-owned two-phase kernel (5), the thread-per-pencil
// kernel fed by tensor TMA (7) and the same with two-plane items and a
// register split (8).  Each is the fastest for some batch on the GB300.
#include "rowfft.cuh"
#include "rowfft2.cuh"
#include "warpown.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n64(int dir, int variant) {
  constexpr int T = fused_threads(64);
  if (variant == 8) return dir < 0 ? rowk2::info<64, -1>() : rowk2::info<64, 1>();
  if (variant == 7) return dir < 0 ? rowk::info<64, -1>() : rowk::info<64, 1>();
  if (variant == 5) return dir < 0 ? wown::info<64, -1>() : wown::info<64, 1>();
  if (variant == 1 && 2 * T <= 1024)
    return dir < 0 ? make_fused_info<2 * T, -1, 64>() : make_fused_info<2 * T, 1, 64>();
  return dir < 0 ? make_fused_info<T, -1, 64>() : make_fused_info<T, 1, 64>();
}

}  // namespace fft3d
