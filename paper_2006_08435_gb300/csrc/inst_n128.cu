// Single-size persistent kernels for 128^3 grids (forward and inverse),
// in two block sizes: the default and twice as many threads per block
// (more warps to hide latency, fewer registers per thread), plus the
// warp-specialised TMA-fed kernel (variant 2).
// Variant 5: warp-owned rows/columns inside the two-phase items.
// Variant 6: split-y items of 64 KB (x and z by thread pairs in registers).
#include "pipelined.cuh"
#include "splity.cuh"
#include "warpown.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n128(int dir, int variant) {
  constexpr int T = fused_threads(128);
  if (variant == 6) return dir < 0 ? sy::info<128, -1>() : sy::info<128, 1>();
  if (variant == 5) return dir < 0 ? wown::info<128, -1>() : wown::info<128, 1>();
  if (variant == 2) return dir < 0 ? piped::info<128, -1>() : piped::info<128, 1>();
  if (variant == 1 && 2 * T <= 1024)
    return dir < 0 ? make_fused_info<2 * T, -1, 128>() : make_fused_info<2 * T, 1, 128>();
  return dir < 0 ? make_fused_info<T, -1, 128>() : make_fused_info<T, 1, 128>();
}

}  // namespace fft3d
