// Split-precision two-plane kernel for 64^3 grids: the tiles, work items,
// producer and publisher of rowfft2.cuh, with every 64-point transform
// split as 64 = 16 x 4 and its radix-16 stage on the tensor cores.
//
// One warp transforms 16 pencils at a time.  Lane (g, t) = (lane / 4,
// lane % 4) holds pencils g and g + 8 of the set, points t + 4 q (q < 4) of
// each length-16 vector, as the mma.m16n8k16 A fragment wants them
// (tc_stage.cuh).  Each pencil is split as n = 16 n1 + n2, k = k1 + 4 k2
// (decimation in frequency):
//     Z[k1][n2] = DFT_4 over n1 (registers),  Z *= W_64^(n2 k1),
//     X[k1 + 4 k2] = DFT_16 over n2 (tensor cores),
// so the radix-4 stage stays inside the thread, and the four vectors of a
// pencil (k1 = 0..3) go through four products with the same DFT_16 matrix,
// whose B fragments stay in registers.
//
// The pencil-to-lane maps are chosen for shared-memory banks.  With the
// tile's 128-byte swizzle an 8-byte access of a half-warp (16-byte access
// of a quarter-warp) meets no conflict when its lanes hit distinct
// (16-byte slot, half) pairs of the 128-byte row pattern:
//   x rows: lane group gl takes row rho(gl) of each eight, rho =
//     0 3 4 7 1 2 5 6, so that the rows of a half-warp differ in the slot
//     bits that the points' 8-byte loads and the k1-pairs' 16-byte stores
//     leave free;
//   y columns: columns whose bits 3 and 0 differ within a half-warp (the
//     points t of a lane quad fill the slot's low bits);
//   z columns of a slab: consecutive columns.
//
// Operands: each pencil is scaled by one power of two so that its largest
// component (after the radix-4 stage for DIF) stays below 2^15, then split
// as hi + lo, hi = the value rounded to a multiple of 16 (128 for BF16) by
// adding and subtracting 1.5 * 2^27 (1.5 * 2^30), lo the exact remainder;
// hi is exact in FP16 (BF16) and lo rounds once.  Products: hi B_hi +
// hi B_lo + lo B_hi, FP32 accumulation (plain FP16: hi B_hi with hi the
// rounded value).  The inverse transform runs the forward stages on the
// conjugate, the conjugations folded into the scale factors.
#pragma once

#include "rowfft2.cuh"
#include "tc_stage.cuh"

namespace fft3d {
namespace tcr {

using piped::mbar_arrive;
using piped::mbar_init;
using piped::saddr;
using piped::warp_wait;
using rowk::Desc;
using rowk::policy_evict_last;
using rowk2::boff;
using rowk2::Cfg;

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

// B fragments of the DFT_16 matrix, hi and lo terms, in registers.
struct Frag {
  uint32_t h[2][4][2], l[2][4][2];
};

template <int PREC>
__device__ __forceinline__ void load_frag(const uint32_t* __restrict__ f, Frag& b) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        b.h[s][u][r] = f[(((0 * 2 + s) * 4 + u) * 32 + lane) * 2 + r];
        b.l[s][u][r] = PREC == 3 ? 0u : f[(((1 * 2 + s) * 4 + u) * 32 + lane) * 2 + r];
      }
}

// The pencil's scale: sc = 2^(E - e), inv = 2^(e - E), e the exponent of
// the largest component m over the four lanes of the quad.
template <int E>
__device__ __forceinline__ void pencil_scale(float m, float& sc, float& inv) {
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
  const int ex = m > 0.0f ? tc::exponent_of(m) : 0;
  sc = tc::pow2(E - ex);
  inv = tc::pow2(ex - E);
}

// Largest |component| of 16 complex values.
__device__ __forceinline__ float absmax16(const float2 (&x)[4][4]) {
  float m = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 4; i += 2)
      m = max3(m, max3(fabsf(x[q][i].x), fabsf(x[q][i].y), fabsf(x[q][i + 1].x)),
               fabsf(x[q][i + 1].y));
  return m;
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

// acc[u] = 16 vectors x DFT_16, output points 4 u + t (tc_stage.cuh layout).
// The four n-tiles are innermost, so consecutive products are independent.
template <int PREC>
__device__ __forceinline__ void dft16_mma(const Frag& b, const uint32_t (&ah)[2][4],
                                          const uint32_t (&al)[2][4], float (&acc)[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[u][i] = 0.0f;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int u = 0; u < 4; ++u) tc::mma<PREC>(acc[u], ah[s], b.h[s][u][0], b.h[s][u][1]);
  if constexpr (PREC != 3) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int u = 0; u < 4; ++u) tc::mma<PREC>(acc[u], ah[s], b.l[s][u][0], b.l[s][u][1]);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int u = 0; u < 4; ++u) tc::mma<PREC>(acc[u], al[s], b.h[s][u][0], b.h[s][u][1]);
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

// The per-lane twiddles W_64^(a (4 b + t)), a = 1..3, b = 0..3 (forward),
// read from the shared copy of the table tw[k2 * 4 + n1] = W_64^(n1 k2)
// at the start of each set.
struct Tw {
  float2 w[3][4];
};

__device__ __forceinline__ void load_tw(uint32_t table, Tw& tw) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) tw.w[a - 1][b] = lds2(table + (uint32_t)((4 * b + t) * 4 + a) * 8u);
}

// One set of 16 pencils: load(r, q, n1) returns point 16 n1 + t + 4 q of
// pencil r; store(r, u, kp, y0, y1) takes output points k1 + 4 (4 u + t)
// for k1 = 2 kp, 2 kp + 1, already multiplied by `out_scale`.
template <int DIR, int PREC, class Load, class Store>
__device__ __forceinline__ void dif_set(const Frag& b, uint32_t twtab, float out_scale, Load load,
                                        Store store) {
  float2 x[2][4][4];  // [r][q][n1], then [r][q][k1]
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) x[r][q][n1] = load(r, q, n1);
  float sc[2], inv[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) pencil_scale<11>(absmax16(x[r]), sc[r], inv[r]);
  // radix-4 in the transform's own direction and twiddles W^(DIR n2 k1);
  // the tensor-core stage then runs forward on the conjugate (inverse)
  Tw tw;
  load_tw(twtab, tw);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dft4<DIR>(x[r][q]);
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) x[r][q][k1] = cmul_tw<DIR>(x[r][q][k1], tw.w[k1 - 1][q]);
    }
  const float cj = DIR > 0 ? -1.0f : 1.0f;
#pragma unroll
  for (int kp = 0; kp < 2; ++kp) {
    float acc[2][4][4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = i & 1, q = 2 * s + (i >> 1);
          split<PREC>(x[r][q][2 * kp + e], make_float2(sc[r], cj * sc[r]), ah[s][i], al[s][i]);
        }
      dft16_mma<PREC>(b, ah, al, acc[e]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const float2 o = make_float2(inv[r] * out_scale, cj * inv[r] * out_scale);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        store(r, u, kp, mul2(make_float2(acc[0][u][2 * r], acc[0][u][2 * r + 1]), o),
              mul2(make_float2(acc[1][u][2 * r], acc[1][u][2 * r + 1]), o));
    }
  }
}

// The two-plane kernel's shared memory plus the twiddle table.
template <int N>
constexpr size_t kSmem = Cfg<N>::smem + 16 + N * sizeof(float2);

template <int N, int DIR, int PREC>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    tcrow_fft3d_kernel(const FusedArgs a, const __grid_constant__ CUtensorMap tin,
                       const __grid_constant__ CUtensorMap tout) {
  using K = Cfg<N>;
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
  float2* twt = reinterpret_cast<float2*>(
      (reinterpret_cast<uintptr_t>(sched + K::SCHED) + 15) & ~(uintptr_t)15);
  const int w = threadIdx.x >> 5;
  if (a.nblocks <= K::SCHED)
    for (int b = threadIdx.x; b < a.nblocks; b += K::T)
      sched[b] = (unsigned short)(a.blocks[b].grid * 2 + a.blocks[b].phase);
  if (threadIdx.x < N) twt[threadIdx.x] = a.twiddles[threadIdx.x];
  if (threadIdx.x == 0) {
    for (int i = 0; i < K::NFULL; ++i) mbar_init(&full[i], 1);
    for (int s = 0; s < NT; ++s) mbar_init(&empty[s], K::GW);
    for (int g = 0; g < K::GROUPS; ++g) mbar_init(&tr[g], K::GW);
    for (int q = 0; q < K::DQ; ++q) mbar_init(&done[q], K::GW);
    *pub_done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (w < 4) {  // control warpgroup
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(K::REG_CTRL));
    if (w == 0)
      rowk2::producer<N>(a, &tin, &tout, tiles, full, empty, done, pubq, pub_done, desc, sched);
    if (w == 1) rowk::publisher<N>(a, done, pubq, pub_done);
    return;
  }
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(K::REG_COMP));

  // compute group g (warpgroup g + 1), warp wl of its four; lane = 4 gl + t
  const int g = (w - 4) / K::GW, wl = (w - 4) % K::GW, lane = threadIdx.x & 31;
  const int gl = lane >> 2, t = lane & 3;
  Frag fb;
  load_frag<PREC>(a.mma_frag, fb);
  const uint32_t tw = saddr(twt);
  unsigned pairs = 0;  // plane-pair items of this group (parity of its barrier)
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!warp_wait(&full[rowk::full_idx<NT, K::GROUPS>(k)], rowk::full_par<NT, K::GROUPS>(k), a))
      break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    const uint32_t tl = tiles + (uint32_t)(s * K::TILE);
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    if (d.phase == 0) {
      // x: rows R = 32 wl + 16 h + rho(gl) + 8 r of the pair (R = 64 j + y)
      const int rho = (4 * ((gl >> 1) & 1) + 3 * (gl & 1)) ^ (gl >> 2);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int R0 = 32 * wl + 16 * h + rho;
        dif_set<DIR, PREC>(
            fb, tw, 1.0f,
            [&](int r, int q, int n1) { return lds2(tl + boff<N>(R0 + 8 * r, 16 * n1 + t + 4 * q)); },
            [&](int r, int u, int kp, float2 y0, float2 y1) {
              sts4(tl + boff<N>(R0 + 8 * r, 2 * kp + 16 * u + 4 * t), y0, y1);
            });
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&tr[g]);
      if (!warp_wait(&tr[g], pairs & 1, a)) break;
      ++pairs;
      // y: columns c of plane j = wl / 2, c = 32 (wl % 2) + 16 h + gamma(gl)
      // + 2 r, gamma = 0 1 8 9 4 5 12 13
      const int j = wl >> 1;
      float2* dst = gout + (long long)(2 * d.idx + j) * NN;
      const unsigned long long keep = policy_evict_last();  // until its slabs read it
      const int gamma = (gl & 1) + 8 * ((gl >> 1) & 1) + 4 * (gl >> 2);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int c0 = 32 * (wl & 1) + 16 * h + gamma;
        dif_set<DIR, PREC>(
            fb, tw, 1.0f,
            [&](int r, int q, int n1) {
              return lds2(tl + boff<N>(64 * j + 16 * n1 + t + 4 * q, c0 + 2 * r));
            },
            [&](int r, int u, int kp, float2 y0, float2 y1) {
              float2* p = dst + (long long)(2 * kp + 16 * u + 4 * t) * N + c0 + 2 * r;
              asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p),
                           "f"(y0.x), "f"(y0.y), "l"(keep));
              asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p + N),
                           "f"(y1.x), "f"(y1.y), "l"(keep));
            });
      }
    } else {
      // z: columns c of slab y = 2 idx + j, j = wl / 2, c as for y
      const int j = wl >> 1;
      float2* dst = gout + (long long)(2 * d.idx + j) * N;
      const float os = a.do_scale ? a.scale : 1.0f;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int c0 = 32 * (wl & 1) + 16 * h + gl;
        dif_set<DIR, PREC>(
            fb, tw, os,
            [&](int r, int q, int n1) {
              return lds2(tl + boff<N>(2 * (16 * n1 + t + 4 * q) + j, c0 + 8 * r));
            },
            [&](int r, int u, int kp, float2 y0, float2 y1) {
              float2* p = dst + (long long)(2 * kp + 16 * u + 4 * t) * NN + c0 + 8 * r;
              st_stream(p, y0);
              st_stream(p + NN, y1);
            });
      }
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[s]);         // the tile is free
      mbar_arrive(&done[k % K::DQ]);  // and the stores done, for the publisher
    }
  }
}

// Uniform batches only (packed buffers, grids in plan order).
template <int N, int DIR, int PREC>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off || !a.mma_frag) return cudaErrorInvalidValue;
  CUtensorMap tin, tout;
  if (!rowk::encode_map(&tin, a.in, N, a.ngrids, N, 2) ||
      !rowk::encode_map(&tout, a.out, N, a.ngrids, 2, N))
    return cudaErrorInvalidValue;
  tcrow_fft3d_kernel<N, DIR, PREC><<<grid, Cfg<N>::T, kSmem<N>, stream>>>(a, tin, tout);
  return cudaGetLastError();
}

template <int N, int DIR, int PREC>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR, PREC>;
  k.func = (const void*)&tcrow_fft3d_kernel<N, DIR, PREC>;
  k.threads = Cfg<N>::T;
  k.smem = kSmem<N>;
  k.twiddle_entries = N;  // W_64^(n1 k2), n1 < 4, k2 < 16
  k.tw_l1 = 4;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;
  k.phase_items = Cfg<N>::ITEMS;
  k.prec = PREC;
  return k;
}

}  // namespace tcr
}  // namespace fft3d
