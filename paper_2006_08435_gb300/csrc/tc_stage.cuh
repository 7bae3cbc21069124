// Radix-16 DFT stage on tensor cores with split half-precision operands.
//
// Sixteen length-16 complex vectors x_v (v = row) are transformed at once as
// the real matrix product Y = X B, X: 16 x 32 (re/im interleaved inputs),
// B: 32 x 32 real form of the DFT matrix W_16^(j k) (forward root), with FP32
// accumulation (mma.sync m16n8k16, two k-steps, four n-tiles).  Precision
// kinds:
//   1  split FP16:  X B ~ Xh Bh + Xh Bl + Xl Bh   (hi = rn(x), lo = rn(x - hi))
//   2  split BF16:  same with bfloat16 halves
//   3  FP16:        Xh Bh only
// Each vector is first scaled by an exact power of two so that its largest
// component lies in [2^14, 2^15): FP16 cannot overflow (the transform's
// values grow up to n^3 max|f|) and the lo part stays in the normal range.
// The scale is undone exactly on the FP32 result.  The inverse direction
// uses conj(DFT(conj(x))).
//
// Fragment layout (PTX ISA, mma.m16n8k16, .f16/.bf16): lane = 4 g + t.
//   A regs: {row g, cols 2t,2t+1}, {row g+8, cols 2t,2t+1},
//           {row g, cols 2t+8,2t+9}, {row g+8, cols 2t+8,2t+9}
//   B regs: {rows 2t,2t+1, col g}, {rows 2t+8,2t+9, col g}
//   C regs: {row g, cols 2t,2t+1}, {row g+8, cols 2t,2t+1}
// With re/im interleaving, lane (g, t) supplies points j = 8 s + t and
// 8 s + t + 4 of vectors g and g + 8 for k-step s, and receives output
// points k = 4 u + t of the same vectors for n-tile u: complex values stay
// whole in every register pair.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "codelets.cuh"

namespace fft3d {
namespace tc {

// B fragments in the table: [term (hi, lo)][s (2)][u (4)][lane (32)][2] u32.
constexpr int kFragWords = 2 * 2 * 4 * 32 * 2;

template <int PREC>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  if constexpr (PREC == 2) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

template <int PREC>
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                    uint32_t b1) {
  if constexpr (PREC == 2)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 2^e as a float for e in [-126, 127] (exact).
__device__ __forceinline__ float pow2(int e) { return __int_as_float((127 + e) << 23); }

// Exponent ex with 2^ex <= m < 2^(ex+1) for a finite m > 0, clamped so
// that the scale 2^(14 - ex) and its inverse stay normal floats.
__device__ __forceinline__ int exponent_of(float m) {
  int ex = ((__float_as_int(m) >> 23) & 0xff) - 127;
  return ex < -100 ? -100 : (ex > 100 ? 100 : ex);
}

// One warp transforms the 16 vectors of a group.  load(vec, j) returns point
// j of vector vec (vec in [0, 16) within the group), store(vec, k, y) writes
// output point k.  frag: B fragments in shared memory.
template <int PREC, int DIR, class Load, class Store>
__device__ __forceinline__ void dft16_group(const uint32_t* __restrict__ frag, Load load,
                                            Store store) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // inputs: x[r][q] = vector g + 8 r, point t + 4 q
  float2 x[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 v = load(g + 8 * r, t + 4 * q);
      if constexpr (DIR > 0) v.y = -v.y;
      x[r][q] = v;
    }
  // per-vector power-of-two scale from the vector's max |component|
  float sc[2], inv[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    float m = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) m = fmaxf(m, fmaxf(fabsf(x[r][q].x), fabsf(x[r][q].y)));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    const int ex = m > 0.0f ? exponent_of(m) : 0;
    sc[r] = pow2(14 - ex);
    inv[r] = pow2(ex - 14);
  }
  // A fragments for k-steps s = 0, 1: regs {g, pt 8s+t}, {g+8, 8s+t},
  // {g, 8s+t+4}, {g+8, 8s+t+4}; points 8s+t -> q = 2s, 8s+t+4 -> q = 2s+1
  uint32_t ah[2][4], al[2][4];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = i & 1, q = 2 * s + (i >> 1);
      split2<PREC>(x[r][q].x * sc[r], x[r][q].y * sc[r], ah[s][i], al[s][i]);
    }
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[u][i] = 0.0f;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t* fh = frag + (((0 * 2 + s) * 4 + u) * 32 + lane) * 2;
      const uint32_t* fl = frag + (((1 * 2 + s) * 4 + u) * 32 + lane) * 2;
      mma<PREC>(acc[u], ah[s], fh[0], fh[1]);
      if constexpr (PREC != 3) {
        mma<PREC>(acc[u], ah[s], fl[0], fl[1]);
        mma<PREC>(acc[u], al[s], fh[0], fh[1]);
      }
    }
  }
  // outputs: acc[u] = {vec g: k = 4u + t (re, im)}, {vec g + 8: same k}
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float2 y = make_float2(acc[u][2 * r] * inv[r], acc[u][2 * r + 1] * inv[r]);
      if constexpr (DIR > 0) y.y = -y.y;
      store(g + 8 * r, 4 * u + t, y);
    }
}

}  // namespace tc
}  // namespace fft3d
