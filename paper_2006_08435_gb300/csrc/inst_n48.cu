// Single-size persistent kernels for 48^3 grids (forward and inverse),
// in two block sizes: the default and twice as many threads per block
// (more warps to hide latency, fewer registers per thread).
// Variant 4: the double-buffered (cp.async prefetch) persistent kernel.
// Variant 13: the thread-pair plane kernel (tensor copies, pencils of n
// points in pairs of threads).
#include "pairfft.cuh"
#include "persistent.cuh"
#include "prefetch.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n48(int dir, int variant) {
  constexpr int T = fused_threads(48);
  if (variant == 13) return dir < 0 ? pf::info<48, -1>() : pf::info<48, 1>();
  if (variant == 4) return dir < 0 ? pref::info<T, -1, 48>() : pref::info<T, 1, 48>();
  if (variant == 1 && 2 * T <= 1024)
    return dir < 0 ? make_fused_info<2 * T, -1, 48>() : make_fused_info<2 * T, 1, 48>();
  return dir < 0 ? make_fused_info<T, -1, 48>() : make_fused_info<T, 1, 48>();
}

}  // namespace fft3d
