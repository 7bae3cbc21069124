// Single-size persistent kernels for 16^3 grids (forward and inverse),
// in two block sizes: the default and twice as many threads per block
// (more warps to hide latency, fewer registers per thread), plus the
// cluster-fused single-pass kernel (variant 3) and the whole-grid kernel
// (variant 12: a grid per block, no counters).
#include "cluster.cuh"
#include "wholegrid.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n16(int dir, int variant) {
  constexpr int T = fused_threads(16);
  if (variant == 12) return dir < 0 ? wg::info<16, -1>() : wg::info<16, 1>();
  if (variant == 3) return dir < 0 ? clus::info<16, -1>() : clus::info<16, 1>();
  if (variant == 1 && 2 * T <= 1024)
    return dir < 0 ? make_fused_info<2 * T, -1, 16>() : make_fused_info<2 * T, 1, 16>();
  return dir < 0 ? make_fused_info<T, -1, 16>() : make_fused_info<T, 1, 16>();
}

}  // namespace fft3d
