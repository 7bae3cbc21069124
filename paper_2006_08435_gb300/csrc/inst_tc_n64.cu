// Tensor-core (split FP16, split BF16, FP16; the block-floating-point and
// FP8 kinds in inst_tc_n64_f4.cu) kernels for 64^3 grids: the
// radix-16 step of each axis runs on the tensor cores.  Variant 0: the
// plain persistent kernel (mma.sync, the fastest below 16 grids); 9: the
// two-plane tensor-TMA items with tcgen05 products (tcgen.cuh).
#include "persistent.cuh"
#include "tcgen.cuh"

namespace fft3d {

template <int DIR, int PREC>
static KernelInfo tc_info_n64(int variant) {
  if (variant == 9) return tg::info<64, DIR, PREC>();
  return make_fused_info_prec<fused_threads(64), DIR, PREC, 64>();
}

KernelInfo tc_kernel_info_n64_f4(int dir, int prec);

KernelInfo tc_kernel_info_n64(int dir, int prec, int variant) {
  if (prec >= FFT3D_BFP16) return variant == 9 ? tc_kernel_info_n64_f4(dir, prec) : KernelInfo{};
  if (dir < 0) {
    if (prec == 1) return tc_info_n64<-1, 1>(variant);
    if (prec == 2) return tc_info_n64<-1, 2>(variant);
    return tc_info_n64<-1, 3>(variant);
  }
  if (prec == 1) return tc_info_n64<1, 1>(variant);
  if (prec == 2) return tc_info_n64<1, 2>(variant);
  return tc_info_n64<1, 3>(variant);
}

}  // namespace fft3d
