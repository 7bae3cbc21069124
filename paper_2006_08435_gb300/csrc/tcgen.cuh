// Split-precision two-plane kernel for 64^3 grids on the fifth-generation
// tensor cores (tcgen05): the tiles, work items, producer and publisher of
// rowfft2.cuh, one pencil per thread as in the FP32 kernel, and the
// radix-16 stage of every axis as tcgen05.mma products with the
// accumulators in tensor memory.
//
// Each 64-point transform is split as n = 16 n1 + n2, k = k1 + 4 k2:
//     R[k1][n2] = DFT_4 over n1 (registers, the transform's direction),
//     X[k1 + 4 k2] = sum_n2 R[k1][n2] W_64^(n2 (k1 + 4 k2))   (tensor cores),
// the second step a 16 x 16 complex product per k1 whose matrix carries the
// twiddles of the split (host table, FP64 rounded to hi + lo halves).  A
// pass over the 128 pencils of an item:
//   1. each thread loads its pencil, scales it by one power of two (its
//      largest component to [2^12, 2^13), so |R| < 2^15), and runs the
//      radix-4 stage;
//   2. each thread writes its four rows (k1) of the A operands into tensor
//      memory (lane = pencil, one 32-bit column per two K entries): hi = R
//      rounded to a multiple of 16 by adding and subtracting 1.5 * 2^27
//      (exact in FP16; 128 and BF16 for split BF16), stored as -hi (the
//      products with it negate A), lo = the exact remainder rounded once;
//   3. after one group barrier, one thread of warp k1 issues D_k1 = A_hi
//      B_hi + A_hi B_lo + A_lo B_hi (M = 128 pencils, N = 32, K = 32: six
//      kind::f16 products, A from tensor memory, B from shared memory, FP32
//      accumulation in 32 tensor-memory columns) and commits them to the
//      group's mbarrier (four arrivals);
//   4. each thread reads its own row of D, undoes the scale and stores X
//      (x: back into its row of the tile, 16-byte chunks; y, z: to global
//      memory, coalesced across the warp).
// Plain FP16 keeps only A_hi B_hi with A rounded to nearest.  The inverse
// feeds conj(R) to the forward matrices and conjugates the result.  The
// shared-memory traffic is the FP32 kernel's plus the small B operands; a
// tile goes back to the producer as soon as its y or z pencils are loaded.
//
// Tensor memory (512 columns): group g owns columns 256 g .. 256 g + 255,
// A_(term, k1) at + (4 term + k1) * 16 and D_k1 at + 128 + 32 k1.
// B operands (16 KB, shared memory for the kernel's life), K-major with no
// swizzle: 8-row x 16-byte core matrices, row r at byte r * 16, core
// matrices 128 bytes apart along K (the leading byte offset) and 512 bytes
// apart along N (the stride byte offset).
#pragma once

#include <cuda_fp8.h>

#include "tcops.cuh"

namespace fft3d {
namespace tg {

using mb::mbar_arrive;
using mb::mbar_init;
using mb::saddr;
using mb::warp_wait;
using rowk::Desc;
using rowk::policy_evict_last;
using rowk2::boff;
using rowk2::Cfg;
using tco::lds2;
using tco::max3;
using tco::sts4;

constexpr int kBBytes = 2 * 4 * 2048;  // B operands: term (hi, lo) x k1 x 32 x 32 halves
constexpr int kTmemCols = 512;         // 2 groups x (A: 8 x 16, D: 4 x 32 columns)

// Operand kinds (PREC, the fft3d_precision value):
//   1 split FP16, 2 split BF16: A = hi + lo (hi a fixed-point mantissa under
//     the pencil's exponent, lo the rounded remainder), B = hi + lo;
//     A_hi B_hi + A_hi B_lo + A_lo B_hi.
//   3 FP16: A = rn(x), B = hi; A B_hi.
//   4 block floating point FP16: A = the fixed-point mantissa hi alone (one
//     exponent per pencil, values multiples of 16 below 2^15: 11 bits and a
//     sign), B = hi + lo; A_hi B_hi + A_hi B_lo -- the error is the data's
//     quantisation alone.
//   5 split FP8 (E4M3): A = hi + lo, each rounded to E4M3, B = 16 b split the
//     same way; A_hi B_hi + A_hi B_lo + A_lo B_hi, kind::f8f6f4 (K = 32 per
//     product).
//   6 FP8 (E4M3): A = rn(x), B = hi; A B_hi.
template <int PREC>
struct Kind {
  static constexpr bool fp8 = PREC == 5 || PREC == 6;
  static constexpr bool a_lo = PREC == 1 || PREC == 2 || PREC == 5;  // an A_lo B_hi product
  static constexpr bool b_lo = PREC != 3 && PREC != 6;               // an A_hi B_lo product
  static constexpr bool neg_hi = PREC == 1 || PREC == 2 || PREC == 4;  // -hi stored (fixed point)
  // the pencil's largest component is scaled to [2^E, 2^(E+1)): below 2^15
  // after the radix-4 stage for the FP16 containers, below 448 (the E4M3
  // maximum) for FP8; block floating point measures it after the radix-4
  // stage, so that its largest mantissa uses all 11 bits
  static constexpr bool post = PREC == 4;
  static constexpr int E = fp8 ? 5 : (post ? 14 : 12);
  static constexpr float bscale = fp8 ? 16.0f : 1.0f;  // B table entries are bscale * b
};

// Shared-memory matrix descriptor: start address, leading byte offset 128
// (next core matrix along K), stride byte offset 512 (next eight rows),
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(512u >> 4) << 32) | (1ull << 46);
}

// Shared-memory descriptor of the FP8 B operands: 8-row x 16-byte core
// matrices (16 E4M3 entries along K per row), the next core matrix along K
// 128 bytes on, the next eight rows 256 bytes on.
__device__ __forceinline__ uint64_t sdesc8(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(256u >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 (A and B FP16, or BF16 for PREC 2) and
// of kind::f8f6f4 (A and B E4M3, format code 0): FP32 accumulator, A
// negated if NEG, both K-major, N = 32, M = 128.
template <int PREC, bool NEG = false>
constexpr uint32_t idesc() {
  constexpr uint32_t ab = PREC == 2 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((NEG ? 1u : 0u) << 13) | ((32u >> 3) << 17) |
         ((128u >> 4) << 24);
}

// Two floats to two E4M3 bytes (round to nearest even, saturating to the
// largest finite value), x.x in the low byte, and back.
__device__ __forceinline__ uint32_t to_e4m3x2(float2 v) {
  return (uint32_t)__nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float2 from_e4m3x2(uint32_t b) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)b, __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

// FP8 A operands: y = x s and the next point's, rounded to E4M3 as hi and
// (split kind) lo = rn(y - hi); one 32-bit word holds the two points
// (re, im, re, im from the low byte).
template <int PREC>
__device__ __forceinline__ void split8(float2 x0, float2 x1, float2 s, uint32_t& hi,
                                       uint32_t& lo) {
  const float2 y0 = mul2(x0, s), y1 = mul2(x1, s);
  const uint32_t h0 = to_e4m3x2(y0), h1 = to_e4m3x2(y1);
  hi = h0 | (h1 << 16);
  if constexpr (Kind<PREC>::a_lo) {
    const uint32_t l0 = to_e4m3x2(csub(y0, from_e4m3x2(h0)));
    const uint32_t l1 = to_e4m3x2(csub(y1, from_e4m3x2(h1)));
    lo = l0 | (l1 << 16);
  } else {
    lo = 0u;
  }
}

// y = x s split as hi + lo for the split kinds, returning -hi: the adding
// and subtracting of 1.5 * 2^27 (2^30 for BF16) yields -hi and the exact
// remainder with one subtraction, and the products with hi negate A.  Plain
// FP16 returns hi = rn(y) itself.
template <int PREC>
__device__ __forceinline__ void split_nhi(float2 x, float2 s, uint32_t& nhi, uint32_t& lo) {
  static_assert(!Kind<PREC>::fp8, "FP8 operands: split8");
  if constexpr (PREC == 3) {
    tco::split<3>(x, s, nhi, lo);
  } else {
    constexpr float C = PREC == 2 ? 1610612736.0f : 201326592.0f;
    const float2 c = make_float2(C, C);
    const float2 t = fma2(x, s, c);
    const float2 hn = csub(c, t);       // -(x s rounded to the hi quantum)
    const float2 lf = fma2(x, s, hn);   // x s - hi, exact
    if constexpr (PREC == 2) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(hn.x, hn.y);
      const __nv_bfloat162 l = __floats2bfloat162_rn(lf.x, lf.y);
      nhi = *reinterpret_cast<const uint32_t*>(&h);
      lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
      const __half2 h = __floats2half2_rn(hn.x, hn.y);
      const __half2 l = __floats2half2_rn(lf.x, lf.y);
      nhi = *reinterpret_cast<const uint32_t*>(&h);
      lo = *reinterpret_cast<const uint32_t*>(&l);
    }
  }
}

// D (tensor memory) (+)= A (tensor memory) B (shared memory descriptor).
__device__ __forceinline__ void umma(uint32_t d, uint32_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}
// The same for 8-bit operands (K = 32 per product).
__device__ __forceinline__ void umma8(uint32_t d, uint32_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}

// 8 consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_st8(uint32_t addr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
      : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Barrier over `count` threads that also ANDs their `ok`: every thread of a
// compute group takes the same decision after a bounded wait, so none is
// left at a later barrier that the others never reach.
__device__ __forceinline__ int group_and(int id, int count, int ok) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
      " selp.b32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(ok), "r"(id), "r"(count)
      : "memory");
  return r;
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane, loaded
// straight into float registers (a .b32 load may name them), so that nothing
// reads the registers before the wait below.
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]),
        "=f"(v[14]), "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]),
        "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]),
        "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(addr));
}
// The registers of a tcgen05.ld hold their values only after tcgen05.wait::ld.
// The values are passed through an empty asm after the wait, so that no use
// of them can be scheduled ahead of it (the wait itself names no register).
__device__ __forceinline__ void tmem_tie(float (&v)[32]) {
  asm volatile(""
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                 "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]),
                 "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]), "+f"(v[16]), "+f"(v[17]),
                 "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]), "+f"(v[22]), "+f"(v[23]),
                 "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]), "+f"(v[29]),
                 "+f"(v[30]), "+f"(v[31]));
}
__device__ __forceinline__ void tmem_wait_ld(float (&dk)[4][32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) tmem_tie(dk[k1]);
}

// Largest |component| of the 64 points.
__device__ __forceinline__ float absmax64(const float2 (&v)[64]) {
  float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < 64; i += 4)
#pragma unroll
    for (int p = 0; p < 2; ++p)
      m[p * 2] = max3(m[p * 2], fabsf(v[i + 2 * p].x), fabsf(v[i + 2 * p].y)),
      m[p * 2 + 1] = max3(m[p * 2 + 1], fabsf(v[i + 2 * p + 1].x), fabsf(v[i + 2 * p + 1].y));
  return fmaxf(max3(m[0], m[1], m[2]), m[3]);
}

// Group state of the tensor-core passes.
struct Pass {
  uint32_t bsm;            // shared address of the B operands
  uint32_t col;            // tensor-memory address of the group's first column
  uint32_t lanes;          // this warp's lane quarter (in the address's high half)
  unsigned long long* bar; // the group's product-completion mbarrier
  int g, gt;
};

// One tensor-core pass over the pencils of the group's tile: v holds this
// thread's pencil (natural order); store(kp, k2, y0, y1) receives output
// points 2 kp + 4 k2 and 2 kp + 1 + 4 k2, multiplied by out_scale.
// Returns false if a wait gave up (the status word is set).
template <int DIR, int PREC, class Store>
__device__ __forceinline__ bool pass(float2 (&v)[64], const Pass& P, unsigned& phase,
                                     const FusedArgs& a, float out_scale, Store store) {
  using KD = Kind<PREC>;
  int ex = 0;
  if constexpr (!KD::post) {
    const float m = absmax64(v);
    ex = m > 0.0f ? tc::exponent_of(m) : 0;
  }
  const float cj = DIR > 0 ? -1.0f : 1.0f;
  // radix-4 over n1: v[16 k1 + n2] = R[k1][n2]
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) {
    float2 q[4] = {v[n2], v[16 + n2], v[32 + n2], v[48 + n2]};
    tco::dft4<DIR>(q);
    v[n2] = q[0];
    v[16 + n2] = q[1];
    v[32 + n2] = q[2];
    v[48 + n2] = q[3];
  }
  if constexpr (KD::post) {
    const float m = absmax64(v);
    ex = m > 0.0f ? tc::exponent_of(m) : 0;
  }
  const float sc = tc::pow2(KD::E - ex);
  // A rows: lane gt of matrix (term, k1), column n2 = (re, im) of point n2
  const float2 s2 = make_float2(sc, cj * sc);
  if constexpr (KD::fp8) {
    // 16 points of a row: 32 E4M3 entries, 8 columns
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      uint32_t h[8], l[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        split8<PREC>(v[16 * k1 + 2 * i], v[16 * k1 + 2 * i + 1], s2, h[i], l[i]);
      tmem_st8(P.col + P.lanes + 16 * k1, h);
      if constexpr (KD::a_lo) tmem_st8(P.col + P.lanes + 16 * (4 + k1), l);
    }
  } else {
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_nhi<PREC>(v[16 * k1 + 8 * e + i], s2, h[i], l[i]);
        tmem_st8(P.col + P.lanes + 16 * k1 + 8 * e, h);
        if constexpr (KD::a_lo) tmem_st8(P.col + P.lanes + 16 * (4 + k1) + 8 * e, l);
      }
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  tc_fence_before();
  named_bar(1 + P.g, Cfg<64>::GT);  // every A row is written, every D row read
  if ((P.gt & 31) == 0) {
    // warp k1 of the group issues the products of k1: four issuing threads
    // keep the tensor cores busier than one (each instruction costs its
    // issuing thread some tens of cycles)
    tc_fence_after();
    // the A_hi columns hold -hi for the fixed-point kinds: those products
    // negate A
    constexpr uint32_t idh = idesc<PREC, KD::neg_hi>(), idl = idesc<PREC>();
    const int k1 = P.gt >> 5;
    const uint32_t d = P.col + 128 + 32 * k1;
    const uint32_t ahi = P.col + 16 * k1, alo = P.col + 16 * (4 + k1);
    if constexpr (KD::fp8) {
      // one product per term (K = 32); B blocks of 1 KB
      const uint32_t bhi = P.bsm + k1 * 1024, blo = P.bsm + (4 + k1) * 1024;
      umma8(d, ahi, sdesc8(bhi), idh, 0);
      if constexpr (KD::b_lo) umma8(d, ahi, sdesc8(blo), idh, 1);
      if constexpr (KD::a_lo) umma8(d, alo, sdesc8(bhi), idl, 1);
    } else {
      const uint32_t bhi = P.bsm + k1 * 2048, blo = P.bsm + (4 + k1) * 2048;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) umma(d, ahi + 8 * ks, sdesc(bhi + 256 * ks), idh, ks);
      if constexpr (KD::b_lo) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) umma(d, ahi + 8 * ks, sdesc(blo + 256 * ks), idh, 1);
      }
      if constexpr (KD::a_lo) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) umma(d, alo + 8 * ks, sdesc(bhi + 256 * ks), idl, 1);
      }
    }
    umma_commit(P.bar);
  }
  if (!group_and(1 + P.g, Cfg<64>::GT, warp_wait(P.bar, phase & 1, a))) return false;
  ++phase;
  tc_fence_after();
  const float inv = tc::pow2(ex - KD::E) * (out_scale / KD::bscale);
  const float2 o = make_float2(inv, cj * inv);
  float dk[4][32];  // the four D rows of this pencil, read before one wait
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) tmem_ld32(P.col + P.lanes + 128 + 32 * k1, dk[k1]);
  tmem_wait_ld(dk);
#pragma unroll
  for (int kp = 0; kp < 2; ++kp)
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2)
      store(kp, k2, mul2(make_float2(dk[2 * kp][2 * k2], dk[2 * kp][2 * k2 + 1]), o),
            mul2(make_float2(dk[2 * kp + 1][2 * k2], dk[2 * kp + 1][2 * k2 + 1]), o));
  tc_fence_before();  // these reads precede the group's next products
  return true;
}

template <int N>
constexpr size_t kSmem = Cfg<N>::smem + 128 + kBBytes + 2 * sizeof(unsigned long long) + 16;

template <int N, int DIR, int PREC>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    tcgen_fft3d_kernel(const FusedArgs a, const __grid_constant__ CUtensorMap tin,
                       const __grid_constant__ CUtensorMap tout) {
  using K = Cfg<N>;
  static_assert(N == 64 && K::GT == 128, "one pencil per thread of a 128-thread group");
  constexpr int NT = K::NTILE;
  constexpr long long NN = (long long)N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const uint32_t tiles = saddr(base);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(base + (size_t)NT * K::TILE);
  unsigned long long* empty = full + K::NFULL;
  unsigned long long* tr = empty + NT;
  unsigned long long* done = tr + K::GROUPS;
  Desc* desc = reinterpret_cast<Desc*>(done + K::DQ);
  int* pubq = reinterpret_cast<int*>(desc + NT);
  volatile int* pub_done = pubq + K::DQ;
  unsigned short* sched = reinterpret_cast<unsigned short*>(pubq + K::DQ + 1);
  unsigned char* bsm_p = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(sched + K::SCHED) + 127) & ~(uintptr_t)127);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(bsm_p + kBBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int w = threadIdx.x >> 5;
  if (a.nblocks <= K::SCHED)
    for (int b = threadIdx.x; b < a.nblocks; b += K::T)
      sched[b] = (unsigned short)(a.blocks[b].grid * 2 + a.blocks[b].phase);
  for (int i = threadIdx.x; i < kBBytes / 16; i += K::T)
    reinterpret_cast<uint4*>(bsm_p)[i] = reinterpret_cast<const uint4*>(a.mma_frag)[i];
  if (threadIdx.x == 0) {
    for (int i = 0; i < K::NFULL; ++i) mbar_init(&full[i], 1);
    for (int s = 0; s < NT; ++s) mbar_init(&empty[s], K::GW);
    for (int g = 0; g < K::GROUPS; ++g) mbar_init(&tr[g], K::GW);
    for (int q = 0; q < K::DQ; ++q) mbar_init(&done[q], K::GW);
    mbar_init(&mbar[0], 4);  // one commit per issuing warp of the group
    mbar_init(&mbar[1], 4);
    *pub_done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 4) {  // the first compute warp owns the tensor-memory allocation
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "n"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B operands, for the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (w < 4) {  // control warpgroup
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(K::REG_CTRL));
    if (w == 0)
      rowk2::producer<N>(a, &tin, &tout, tiles, full, empty, done, pubq, pub_done, desc, sched);
    if (w == 1) rowk::publisher<N>(a, done, pubq, pub_done);
    return;
  }
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(K::REG_COMP));

  // compute group g (warpgroup g + 1), thread gt of 128: pencil gt of a pass
  const int g = (w - 4) / K::GW, gt = threadIdx.x - 128 - g * K::GT, lane = threadIdx.x & 31;
  const int j = gt >> 6, u = gt & (N - 1);
  Pass P;
  P.bsm = saddr(bsm_p);
  P.col = *tslot + (uint32_t)(256 * g);
  P.lanes = (uint32_t)(32 * (gt >> 5)) << 16;
  P.bar = &mbar[g];
  P.g = g;
  P.gt = gt;
  unsigned phase = 0;  // completed product batches of this group
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!group_and(1 + g, K::GT,
                   warp_wait(&full[rowk::full_idx<NT, K::GROUPS>(k)],
                             rowk::full_par<NT, K::GROUPS>(k), a)))
      break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    const uint32_t tl = tiles + (uint32_t)(s * K::TILE);
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2 v[N];
    if (d.phase == 0) {
      // x: row gt of the pair (row y = u of plane j), 16-byte chunks
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const float4 q = *reinterpret_cast<const float4*>(base + (size_t)s * K::TILE + boff<N>(gt, 2 * i));
        v[2 * i] = make_float2(q.x, q.y);
        v[2 * i + 1] = make_float2(q.z, q.w);
      }
      if (!pass<DIR, PREC>(v, P, phase, a, 1.0f, [&](int kp, int k2, float2 y0, float2 y1) {
            sts4(tl + boff<N>(gt, 2 * kp + 4 * k2), y0, y1);
          }))
        break;
      named_bar(1 + g, K::GT);  // the x results are in the tile
      // y: column x = u of plane j, output rows straight to global memory
#pragma unroll
      for (int r = 0; r < N; ++r) v[r] = lds2(tl + boff<N>(64 * j + r, u));
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // the tile is read: back to the producer
      float2* dst = gout + (long long)(2 * d.idx + j) * NN + u;
      const unsigned long long keep = policy_evict_last();  // until its slabs read it
      if (!pass<DIR, PREC>(v, P, phase, a, 1.0f, [&](int kp, int k2, float2 y0, float2 y1) {
            float2* p = dst + (long long)(2 * kp + 4 * k2) * N;
            asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p),
                         "f"(y0.x), "f"(y0.y), "l"(keep));
            asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p + N),
                         "f"(y1.x), "f"(y1.y), "l"(keep));
          }))
        break;
    } else {
      // z: column x = u of slab y = 2 idx + j
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = lds2(tl + boff<N>(2 * z + j, u));
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // the tile is read: back to the producer
      float2* dst = gout + (long long)(2 * d.idx + j) * N + u;
      if (!pass<DIR, PREC>(v, P, phase, a, a.do_scale ? a.scale : 1.0f,
                           [&](int kp, int k2, float2 y0, float2 y1) {
                             float2* p = dst + (long long)(2 * kp + 4 * k2) * NN;
                             st_stream(p, y0);
                             st_stream(p + NN, y1);
                           }))
        break;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[k % K::DQ]);  // the stores are done, for the publisher
  }
  // every compute warp is out of its loop: no product or tensor-memory read
  // is in flight
  tc_fence_before();
  named_bar(3, 2 * K::GT);
  tc_fence_after();
  if (w == 4)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot),
                 "n"(kTmemCols));
}

// Uniform batches only (packed buffers, grids in plan order).
template <int N, int DIR, int PREC>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off || !a.mma_frag) return cudaErrorInvalidValue;
  CUtensorMap tin, tout;
  if (!rowk::encode_map(&tin, a.in, N, a.ngrids, N, 2) ||
      !rowk::encode_map(&tout, a.out, N, a.ngrids, 2, N))
    return cudaErrorInvalidValue;
  tcgen_fft3d_kernel<N, DIR, PREC><<<grid, Cfg<N>::T, kSmem<N>, stream>>>(a, tin, tout);
  return cudaGetLastError();
}

template <int N, int DIR, int PREC>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR, PREC>;
  k.func = (const void*)&tcgen_fft3d_kernel<N, DIR, PREC>;
  k.threads = Cfg<N>::T;
  k.smem = kSmem<N>;
  k.twiddle_entries = N;  // (the B operands carry the twiddles; a table is uploaded anyway)
  k.tw_l1 = 4;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;
  k.phase_items = Cfg<N>::ITEMS;
  k.prec = PREC;
  k.umma_b = 1;
  return k;
}

}  // namespace tg
}  // namespace fft3d
