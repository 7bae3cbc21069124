// Single-size persistent kernels for 64^3 grids (forward and inverse),
// in two block sizes: the default and twice as many threads per block
// (more warps to hide latency, fewer registers per thread), plus the
// warp-specialised TMA-fed kernel (variant 2) and the cluster-fused
// single-pass kernel (variant 3).
// Variant 4: the double-buffered (cp.async prefetch) persistent kernel.
// Variant 5: warp-owned rows/columns inside the two-phase items.
// Variant 6: double-buffered TMA-fed blocks with producer and signaller warps.
// Variant 7: thread-per-pencil register FFTs fed by tensor TMA.
// Variant 8: the same with two-plane items and a register split.
#include "cluster.cuh"
#include "dbuf.cuh"
#include "prefetch.cuh"
#include "pipelined.cuh"
#include "rowfft.cuh"
#include "rowfft2.cuh"
#include "warpown.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n64(int dir, int variant) {
  constexpr int T = fused_threads(64);
  if (variant == 8) return dir < 0 ? rowk2::info<64, -1>() : rowk2::info<64, 1>();
  if (variant == 7) return dir < 0 ? rowk::info<64, -1>() : rowk::info<64, 1>();
  if (variant == 6) return dir < 0 ? dbuf::info<64, -1>() : dbuf::info<64, 1>();
  if (variant == 5) return dir < 0 ? wown::info<64, -1>() : wown::info<64, 1>();
  if (variant == 4) return dir < 0 ? pref::info<T, -1, 64>() : pref::info<T, 1, 64>();
  if (variant == 3) return dir < 0 ? clus::info<64, -1>() : clus::info<64, 1>();
  if (variant == 2) return dir < 0 ? piped::info<64, -1>() : piped::info<64, 1>();
  if (variant == 1 && 2 * T <= 1024)
    return dir < 0 ? make_fused_info<2 * T, -1, 64>() : make_fused_info<2 * T, 1, 64>();
  return dir < 0 ? make_fused_info<T, -1, 64>() : make_fused_info<T, 1, 64>();
}

}  // namespace fft3d
