// Register and shared-memory helpers of the tcgen05 tensor-core kernels
// (tcgen.cuh, tcsplity.cuh): tile accesses by shared-window address, a
// three-way max, the radix-4 DFT, and the split of a scaled value into the
// FP16 / BF16 operand halves.
#pragma once

#include "rowfft2.cuh"
#include "tc_stage.cuh"

namespace fft3d {
namespace tco {

// Shared-memory accesses by 32-bit shared-window address; the load declares
// that it reads memory, so it stays ordered after the barrier waits and the
// stores that fill the tile.
__device__ __forceinline__ float2 lds2(uint32_t a) {
  float2 v;
  asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts4(uint32_t a, float2 v, float2 w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(w.x),
               "f"(w.y)
               : "memory");
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}


// y = x * s (s carries the conjugation), split into the A-fragment halves.
template <int PREC>
__device__ __forceinline__ void split(float2 x, float2 s, uint32_t& hi, uint32_t& lo) {
  if constexpr (PREC == 3) {
    const float2 y = mul2(x, s);
    const __half2 h = __floats2half2_rn(y.x, y.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = 0u;
  } else {
    constexpr float C = PREC == 2 ? 1610612736.0f : 201326592.0f;  // 1.5 * 2^30, 1.5 * 2^27
    const float2 c = make_float2(C, C);
    const float2 t = fma2(x, s, c);
    const float2 hf = csub(t, c);                  // x s rounded to the hi quantum
    const float2 lf = fma2(x, s, csub(c, t));      // x s - hf, exact
    if constexpr (PREC == 2) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(hf.x, hf.y);
      const __nv_bfloat162 l = __floats2bfloat162_rn(lf.x, lf.y);
      hi = *reinterpret_cast<const uint32_t*>(&h);
      lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
      const __half2 h = __floats2half2_rn(hf.x, hf.y);
      const __half2 l = __floats2half2_rn(lf.x, lf.y);
      hi = *reinterpret_cast<const uint32_t*>(&h);
      lo = *reinterpret_cast<const uint32_t*>(&l);
    }
  }
}


// Forward (DIR < 0) or inverse DFT_4 of v[0..3], natural order.
template <int DIR>
__device__ __forceinline__ void dft4(float2 (&v)[4]) {
  const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  const float2 c = cadd(v[1], v[3]), d = mul_i<DIR>(csub(v[1], v[3]));
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

}  // namespace tco
}  // namespace fft3d
