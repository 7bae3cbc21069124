// Single-size persistent kernels for 32^3 grids (forward and inverse),
// in two block sizes: the default and twice as many threads per block
// (more warps to hide latency, fewer registers per thread), plus the
// cluster-fused single-pass kernel (variant 3).
// Variant 4: the double-buffered (cp.async prefetch) persistent kernel.
// Variant 13: the thread-pair kernel (tensor copies of four planes or slabs
// per item, pencils of 32 points in pairs of threads).
#include "cluster.cuh"
#include "pairfft.cuh"
#include "prefetch.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n32(int dir, int variant) {
  constexpr int T = fused_threads(32);
  if (variant == 13) return dir < 0 ? pf::info<32, -1>() : pf::info<32, 1>();
  if (variant == 4) return dir < 0 ? pref::info<T, -1, 32>() : pref::info<T, 1, 32>();
  if (variant == 3) return dir < 0 ? clus::info<32, -1>() : clus::info<32, 1>();
  if (variant == 1 && 2 * T <= 1024)
    return dir < 0 ? make_fused_info<2 * T, -1, 32>() : make_fused_info<2 * T, 1, 32>();
  return dir < 0 ? make_fused_info<T, -1, 32>() : make_fused_info<T, 1, 32>();
}

}  // namespace fft3d
