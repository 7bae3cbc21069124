// Mixed-size persistent kernel (every fused edge in one launch) and the
// bounded-wait self test.
#include "persistent.cuh"

namespace fft3d {

KernelInfo mixed_kernel_info(int dir) {
  constexpr int T = kMixedThreads;
  return dir < 0 ? make_fused_info<T, -1, 16, 32, 48, 64, 80, 96, 128>()
                 : make_fused_info<T, 1, 16, 32, 48, 64, 80, 96, 128>();
}

// One thread waits, with the persistent kernel's bounded wait, on a flag
// that nothing sets.
__global__ void wait_selftest_kernel(const unsigned* flag, unsigned* status, long long timeout_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) bounded_wait_geq(flag, 1u, status, timeout_ns);
}

cudaError_t launch_wait_selftest(unsigned* flag, unsigned* status, long long timeout_ns,
                                 cudaStream_t stream) {
  wait_selftest_kernel<<<1, 32, 0, stream>>>(flag, status, timeout_ns);
  return cudaGetLastError();
}

}  // namespace fft3d
