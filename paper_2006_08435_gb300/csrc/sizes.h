// Edge lengths planned by the fused kernels and their two-factor split.
// Shared by host planning (twiddle tables) and device code (codelet
// choice); the split must agree on both sides.
//
// An edge n is transformed as n = L1 * L2 (four-step): first L1 DFTs of
// length L2 over the stride-L1 subsequences, a twiddle W_n^(n1 k2), then L2
// DFTs of length L1 (the 1D FFTs of the paper's "Approach" section).
#pragma once

namespace fft3d {

// Cubic edges with a fused persistent kernel, in the order their twiddle
// tables are concatenated.
constexpr int kFusedSizes[] = {16, 32, 48, 64, 80, 96, 128};
constexpr int kNumFusedSizes = 7;

__host__ __device__ constexpr int split_l1(int n) {
  return n == 16 ? 4 : n == 32 ? 4 : n == 48 ? 3 : n == 64 ? 8
       : n == 80 ? 5 : n == 96 ? 6 : n == 128 ? 8 : 0;
}
__host__ __device__ constexpr int split_l2(int n) {
  return split_l1(n) ? n / split_l1(n) : 0;
}
// Split used by a kernel: the FP32 kernels use split_l1; the tensor-core
// kinds (prec != 0) always make the first step radix 16, n = (n/16) * 16.
__host__ __device__ constexpr int item_l1(int n, int prec) {
  return prec ? n / 16 : split_l1(n);
}
// Threads per block of the single-size persistent kernel for edge n.
__host__ __device__ constexpr int fused_threads(int n) {
  return n == 16 ? 64 : n == 32 ? 128 : n == 48 ? 192 : n == 64 ? 256
       : n == 80 ? 320 : n == 96 ? 384 : 512;
}
// Threads per block of the mixed-size persistent kernel.
constexpr int kMixedThreads = 512;

__host__ __device__ constexpr int fused_slot(int n) {
  return n == 16 ? 0 : n == 32 ? 1 : n == 48 ? 2 : n == 64 ? 3
       : n == 80 ? 4 : n == 96 ? 5 : n == 128 ? 6 : -1;
}

}  // namespace fft3d
