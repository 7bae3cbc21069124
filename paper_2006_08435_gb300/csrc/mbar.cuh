// mbarrier helpers of the warp-specialised kernels (the tile rings of
// rowfft.cuh, rowfft2.cuh, splity.cuh and the tcgen05 kernels): shared-
// window addresses, initialisation, arrivals, and waits that are bounded in
// time and report a timeout through the plan's status word instead of
// hanging.
#pragma once

#include "persistent.cuh"

namespace fft3d {
namespace mb {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ unsigned mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok;
}
// As above, but the thread may sleep in hardware (up to ~hint_ns) until the
// phase completes instead of returning at once: waiting warps do not take
// issue slots from working ones.
__device__ __forceinline__ unsigned mbar_try_wait_sleep(unsigned long long* b, unsigned parity,
                                                        unsigned hint_ns) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; "
      "selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok;
}
// Wait for the phase with the given parity to complete: at most timeout_ns
// of %globaltimer and 2^20 sleeping polls.  0 on timeout (status set) or
// when another block already reported a failure.
__device__ __forceinline__ int mbar_wait_bounded(unsigned long long* b, unsigned parity,
                                                 unsigned* status, long long timeout_ns) {
  if (mbar_try_wait(b, parity)) return 1;
  const unsigned long long t0 = global_timer_ns();
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try_wait_sleep(b, parity, 100000u)) return 1;
    if (*(volatile unsigned*)status != kStatusOk) return 0;
    if ((long long)(global_timer_ns() - t0) > timeout_ns) break;
  }
  atomicCAS(status, kStatusOk, kStatusTimeout);
  return 0;
}
// Warp-level bounded wait: every lane waits (sleeping in hardware) and the
// warp proceeds only if all lanes saw the phase complete, so the warp stays
// converged and takes one decision.
__device__ __forceinline__ int warp_wait(unsigned long long* b, unsigned parity,
                                         const FusedArgs& a) {
  const int ok = mbar_wait_bounded(b, parity, a.status, a.timeout_ns);
  return __all_sync(0xffffffffu, ok);
}

}  // namespace mb
}  // namespace fft3d
