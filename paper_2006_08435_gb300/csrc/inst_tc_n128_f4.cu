// Block-floating-point FP16 and FP8 (E4M3) operand kinds for 128^3 grids,
// on the tcgen05 kernel only (variant 9): tcsplity.cuh.
#include "tcsplity.cuh"

namespace fft3d {

KernelInfo tc_kernel_info_n128_f4(int dir, int prec) {
  if (dir < 0) {
    if (prec == FFT3D_BFP16) return tsy::info<128, -1, FFT3D_BFP16>();
    if (prec == FFT3D_SPLIT_FP8) return tsy::info<128, -1, FFT3D_SPLIT_FP8>();
    return tsy::info<128, -1, FFT3D_FP8>();
  }
  if (prec == FFT3D_BFP16) return tsy::info<128, 1, FFT3D_BFP16>();
  if (prec == FFT3D_SPLIT_FP8) return tsy::info<128, 1, FFT3D_SPLIT_FP8>();
  return tsy::info<128, 1, FFT3D_FP8>();
}

}  // namespace fft3d
