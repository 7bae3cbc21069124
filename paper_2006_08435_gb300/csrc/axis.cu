// Pencil passes of the general path: any edge 2 <= n <= 512 whose prime
// factors are 2, 3 and 5, on every axis independently (non-cubic grids),
// as three passes over the grid, one per axis -- the 1D FFTs along x, then
// y, then z of the paper's section "Approach", each a batched 1D transform
// of all pencils along one axis.
//
// A block takes a tile of W pencils at a time into shared memory, laid out
// [i][q] (element i of pencil q at i * (W + 1) + q; the odd pitch keeps the
// column accesses of the x pass free of bank conflicts):
//   x pass (contiguous pencils): W consecutive rows, read row by row;
//   y and z passes (strided): the 16 pencils at x0 .. x0 + 15 of W / 16
//     consecutive (grid, z) or (grid, y) slices, element i of the 16 of a
//     slice being one 128-byte run in memory.
// A tile holds about 8192 points (4096 per buffer when two buffers let the
// next tile's copies run during this one's transform).
// The L-point transform of each pencil runs in place in the tile as
// decimation in frequency over the radices R_0, R_1, ... (product L):
// stage t splits each block of N_t = L / (R_0 ... R_{t-1}) points into R_t
// sub-blocks of M = N_t / R_t points, y_k = sum_r x[j + r M] W_R^(r k) times
// W_(N_t)^(j k) going to position j + k M, so that sub-block k holds the
// sequence whose M-point DFT is X[k + R m].  After the last stage output K
// = k_0 + R_0 (k_1 + R_1 (k_2 + ...)) sits at position
// sum_t k_t L / (R_0 ... R_t) (the mixed-radix digit reversal, a host
// table); the stores read it from there, in natural order.  Twiddles are a
// host table of W_L^m, m < L, in FP64 rounded to FP32 (the inverse uses the
// conjugates); the radix-R butterflies are the register codelets.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fft3d.h"
#include "codelets.cuh"
#include "internal.h"

namespace fft3d {
namespace ax {

constexpr int kThreads = 256;

using Args = AxisArgs;

// n / d for n < 2^32 with the multiplier and shift of FastDiv (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994:
// m = floor(2^32 (2^l - d) / d) + 1 with l = ceil(log2 d), q = (hi(n m) + n) >> l).
__device__ __forceinline__ unsigned fdiv(unsigned n, FastDiv d) {
  return (unsigned)(((unsigned long long)__umulhi(n, d.mul) + n) >> d.shift);
}

// Tile slot of element i of pencil c.  In the x pass of a power-of-two
// span S = L / R_0, the digit-reversed positions that consecutive outputs
// read are S apart, so without a rotation every lane of a warp would hit
// the same bank (16-way conflicts at L = 256); the pencil index is XORed
// with bits of i / S (a permutation of each aligned group of 16 pencils, so
// the butterflies, whose lanes share i, stay conflict-free).
__device__ __forceinline__ int tix(const Args& a, int i, int c, int P) {
  return i * P + (c ^ ((i >> a.swsh) & a.swmask));
}

template <int R, int DIR>
__device__ __forceinline__ void stage(float2* tile, const float2* tw, const Args& a, int t, int P) {
  const int N = a.span[t], M = a.sub[t], stw = a.twst[t];
  const int nb = (a.L / R) << a.lw;  // butterflies in the tile
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    const int q = b & (a.W - 1);
    const unsigned jb = (unsigned)b >> a.lw;
    const unsigned blk = fdiv(jb, a.divsub[t]);
    const int j = (int)(jb - blk * (unsigned)M);
    const int i0 = (int)blk * N + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[tix(a, i0 + r * M, q, P)];
    DFT<R, DIR>::run(v);
    const int st = j * stw;  // W_N^(j k) = W_L^(j k L / N); j k L / N < L
    if (st) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul_tw<DIR>(v[k], tw[k * st]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) tile[tix(a, i0 + k * M, q, P)] = v[k];
  }
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Where tile t lives.  x pass: W consecutive rows from base (nv of them
// exist; the last tile can be partial).  y and z passes: the 16 pencils at
// x0 .. x0 + 15 (nvx < 16 at the x edge) of G = W / 16 consecutive slices
// o0 .. o0 + G - 1 (ng of them exist); pencil c of the tile is (g, q) =
// (c / 16, c % 16).
struct TileRef {
  long long base;  // x pass
  int nv;          // x pass: rows
  unsigned o0;     // strided: first slice
  int x0, nvx, ng;
};
__device__ __forceinline__ TileRef tile_of(const Args& a, unsigned t) {
  TileRef r;
  if (a.contiguous) {
    const long long r0 = (long long)t << a.lw;
    r.nv = (int)min((long long)a.W, a.rows - r0);
    r.base = r0 * a.L;
  } else {
    const unsigned ot = fdiv(t, a.divx);
    r.x0 = (int)(t - ot * (unsigned)a.xtiles) << 4;
    r.nvx = min(16, a.nx - r.x0);
    r.o0 = ot << (a.lw - 4);
    r.ng = (int)min((long long)(a.W >> 4), a.outer - (long long)r.o0);
  }
  return r;
}
// First element of slice o: (o / d1) s1 + (o % d1) s0.
__device__ __forceinline__ long long slice_base(const Args& a, unsigned o) {
  const unsigned o1 = fdiv(o, a.divd1);
  return (long long)o1 * a.s1 + (long long)(o - o1 * (unsigned)a.d1) * a.s0;
}

// Asynchronous copies of tile t into buf ([i][c], pitch P), 8 bytes each:
// every copy of a thread is in flight at once.
__device__ __forceinline__ void load_tile(const Args& a, unsigned t, float2* buf, int P) {
  const TileRef r = tile_of(a, t);
  const uint32_t sb = (uint32_t)__cvta_generic_to_shared(buf);
  if (a.contiguous) {
    const float2* src = a.in + r.base;
    for (int e = threadIdx.x; e < r.nv * a.L; e += kThreads) {
      const unsigned q = fdiv((unsigned)e, a.divL);
      cp_async8(sb + 8u * (uint32_t)tix(a, e - (int)q * a.L, (int)q, P), src + e);
    }
  } else {
    // W <= kThreads: a thread's pencil c is the same in every step
    const int c = threadIdx.x & (a.W - 1), q = c & 15, g = c >> 4;
    if (q < r.nvx && g < r.ng) {
      const float2* src = a.in + slice_base(a, r.o0 + g) + r.x0 + q;
      for (int i = threadIdx.x >> a.lw; i < a.L; i += kThreads >> a.lw)
        cp_async8(sb + 8u * (uint32_t)tix(a, i, c, P), src + (long long)i * a.pi);
    }
  }
}

// NBUF = 2: the next tile's copies are issued before the current tile is
// transformed (two tile buffers); NBUF = 1: one buffer, the copies of a
// tile all in flight at once, other blocks on the multiprocessor overlap.
template <int DIR, int NBUF>
__global__ void __launch_bounds__(kThreads, NBUF == 2 ? 3 : 2) axis_pass_kernel(const Args a) {
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.W + 1;
  const size_t bstride = (size_t)a.L * P;  // buffer b at sm + b * bstride
  float2* tw = sm + NBUF * bstride;
  unsigned short* pos = reinterpret_cast<unsigned short*>(tw + a.L);
  for (int i = threadIdx.x; i < a.L; i += kThreads) {
    tw[i] = a.tw[i];
    pos[i] = a.pos[i];
  }
  unsigned t = blockIdx.x;
  if (NBUF == 2 && t < a.ntiles) {
    load_tile(a, t, sm, P);
    cp_async_commit();
  }
  for (int it = 0; t < a.ntiles; t += gridDim.x, ++it) {
    float2* tile = sm + (NBUF == 2 ? (it & 1) : 0) * bstride;
    if (NBUF == 2) {
      if (t + gridDim.x < a.ntiles) load_tile(a, t + gridDim.x, sm + ((it & 1) ^ 1) * bstride, P);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      load_tile(a, t, tile, P);
      cp_async_commit();
      cp_async_wait<0>();
    }
    __syncthreads();
    for (int s = 0; s < a.nst; ++s) {
      switch (a.radix[s]) {
        case 16: stage<16, DIR>(tile, tw, a, s, P); break;
        case 15: stage<15, DIR>(tile, tw, a, s, P); break;
        case 12: stage<12, DIR>(tile, tw, a, s, P); break;
        case 10: stage<10, DIR>(tile, tw, a, s, P); break;
        case 9: stage<9, DIR>(tile, tw, a, s, P); break;
        case 8: stage<8, DIR>(tile, tw, a, s, P); break;
        case 6: stage<6, DIR>(tile, tw, a, s, P); break;
        case 5: stage<5, DIR>(tile, tw, a, s, P); break;
        case 4: stage<4, DIR>(tile, tw, a, s, P); break;
        case 3: stage<3, DIR>(tile, tw, a, s, P); break;
        default: stage<2, DIR>(tile, tw, a, s, P); break;
      }
      __syncthreads();
    }
    const float sc = a.do_scale ? a.scale : 1.0f;
    const TileRef r = tile_of(a, t);
    if (a.contiguous) {
      float2* dst = a.out + r.base;
#pragma unroll 4
      for (int e = threadIdx.x; e < r.nv * a.L; e += kThreads) {
        const unsigned q = fdiv((unsigned)e, a.divL);
        dst[e] = cscale(tile[tix(a, pos[e - (int)q * a.L], (int)q, P)], sc);
      }
    } else {
      const int c = threadIdx.x & (a.W - 1), q = c & 15, g = c >> 4;
      if (q < r.nvx && g < r.ng) {
        float2* dst = a.out + slice_base(a, r.o0 + g) + r.x0 + q;
#pragma unroll 4
        for (int k = threadIdx.x >> a.lw; k < a.L; k += kThreads >> a.lw)
          dst[(long long)k * a.pi] = cscale(tile[tix(a, pos[k], c, P)], sc);
      }
    }
    __syncthreads();  // this buffer is reloaded next
  }
}

// ------------------------------------------------------------ plane pass
constexpr int kPlaneThreads = 256;

// One stage over `np` pencils of the plane (pencil c fastest across the
// threads), element i of pencil c at addr(c, i).
template <int R, int DIR, class Addr>
__device__ __forceinline__ void plane_stage(float2* pl, const float2* tw, const AxisStages& st,
                                            int t, int np, FastDiv divnp, Addr addr) {
  const int N = st.span[t], M = st.sub[t], stw = st.twst[t];
  const int nb = (st.L / R) * np;
  for (int b = threadIdx.x; b < nb; b += kPlaneThreads) {
    const unsigned jb = fdiv((unsigned)b, divnp);
    const int c = b - (int)jb * np;
    const unsigned blk = fdiv(jb, st.divsub[t]);
    const int j = (int)(jb - blk * (unsigned)M);
    const int i0 = (int)blk * N + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = pl[addr(c, i0 + r * M)];
    DFT<R, DIR>::run(v);
    const int sk = j * stw;
    if (sk) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul_tw<DIR>(v[k], tw[k * sk]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) pl[addr(c, i0 + k * M)] = v[k];
  }
}

template <int DIR, class Addr>
__device__ __forceinline__ void plane_axis(float2* pl, const float2* tw, const AxisStages& st,
                                           int np, FastDiv divnp, Addr addr) {
  for (int s = 0; s < st.nst; ++s) {
    switch (st.radix[s]) {
      case 16: plane_stage<16, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 15: plane_stage<15, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 12: plane_stage<12, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 10: plane_stage<10, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 9: plane_stage<9, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 8: plane_stage<8, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 6: plane_stage<6, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 5: plane_stage<5, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 4: plane_stage<4, DIR>(pl, tw, st, s, np, divnp, addr); break;
      case 3: plane_stage<3, DIR>(pl, tw, st, s, np, divnp, addr); break;
      default: plane_stage<2, DIR>(pl, tw, st, s, np, divnp, addr); break;
    }
    __syncthreads();
  }
}

// Planes of nx x ny points (rows of nx contiguous in memory), one per block
// at a time: the plane is copied in (cp.async, rows contiguous), the x
// stages run over its ny rows, the y stages over its nx columns, and the
// stores read the digit-reversed result of both axes in natural order.
// Shared layout: element (x, y) at y * px + rot(x), px odd (the x stages'
// lanes are rows: stride px; the y stages' lanes are columns: consecutive),
// rot(x) = x ^ ((x >> rsh) & rmask) a permutation of each aligned group of
// 16 that keeps the stores' digit-reversed reads (consecutive outputs S =
// nx / R_0 apart) off a single bank.
template <int DIR>
__global__ void __launch_bounds__(kPlaneThreads, 2) plane_pass_kernel(const PlaneArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const int nx = a.nx, ny = a.ny, px = a.px;
  float2* pl = sm;
  float2* twx = pl + (size_t)ny * px;
  float2* twy = twx + nx;
  unsigned short* posx = reinterpret_cast<unsigned short*>(twy + ny);
  unsigned short* posy = posx + nx;
  for (int i = threadIdx.x; i < nx; i += kPlaneThreads) {
    twx[i] = a.twx[i];
    posx[i] = a.posx[i];
  }
  for (int i = threadIdx.x; i < ny; i += kPlaneThreads) {
    twy[i] = a.twy[i];
    posy[i] = a.posy[i];
  }
  auto rot = [&](int x) { return x ^ ((x >> a.rsh) & a.rmask); };
  const uint32_t sb = (uint32_t)__cvta_generic_to_shared(pl);
  const int pts = nx * ny;
  for (unsigned p = blockIdx.x; p < a.nplanes; p += gridDim.x) {
    const float2* src = a.in + (size_t)p * pts;
    for (int e = threadIdx.x; e < pts; e += kPlaneThreads) {
      const int y = (int)fdiv((unsigned)e, a.divnx), x = e - y * nx;
      cp_async8(sb + 8u * (uint32_t)(y * px + rot(x)), src + e);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // x: pencils are the rows (c = y), elements x
    plane_axis<DIR>(pl, twx, a.sx, ny, a.divny, [&](int c, int i) { return c * px + rot(i); });
    // y: pencils are the columns (c = x), elements y
    plane_axis<DIR>(pl, twy, a.sy, nx, a.divnx, [&](int c, int i) { return i * px + rot(c); });
    float2* dst = a.out + (size_t)p * pts;
#pragma unroll 4
    for (int e = threadIdx.x; e < pts; e += kPlaneThreads) {
      const int ky = (int)fdiv((unsigned)e, a.divnx), kx = e - ky * nx;
      dst[e] = pl[posy[ky] * px + rot(posx[kx])];
    }
    __syncthreads();  // the plane is reloaded next
  }
}

constexpr int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

size_t smem_bytes(int L, int W, int nbuf) {
  return ((size_t)nbuf * L * (W + 1) + L) * sizeof(float2) + (size_t)L * sizeof(unsigned short);
}
// The largest smem_bytes of any pass (L W <= 8192 pencil points, L <= 512,
// two buffers): the kernels' dynamic shared-memory limit is set once to
// this, since the passes of one plan (different L and W) share a kernel.
constexpr size_t kSmemLimit =
    (2 * (8192 + 512) + 512) * sizeof(float2) + 512 * sizeof(unsigned short);

}  // namespace ax

FastDiv make_fastdiv(unsigned d) {
  FastDiv f{1u, 0};
  if (d <= 1) {
    f.mul = 1u;  // hi(n * 1) = 0: q = n
    return f;
  }
  int l = 0;
  while ((1ull << l) < d) ++l;
  f.shift = l;
  f.mul = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  return f;
}

int axis_stages(int L, int* radix) {
  if (L < 2 || L > kAxisMaxLen) return 0;
  int n = 0, rem = L;
  while (rem > 1) {
    int r = 0;
    for (int c : ax::kRadices)
      if (rem % c == 0) {
        r = c;
        break;
      }
    if (!r || n == kAxisMaxStages) return 0;
    radix[n++] = r;
    rem /= r;
  }
  return n;
}

void axis_positions(int L, int nst, const int* radix, int* pos) {
  for (int K = 0; K < L; ++K) {
    int rem = K, span = L, p = 0;
    for (int t = 0; t < nst; ++t) {
      span /= radix[t];
      p += (rem % radix[t]) * span;
      rem /= radix[t];
    }
    pos[K] = p;
  }
}

int prepare_axis_pass(const AxisTable& tab, int dir, const AxisGeom& g, int sms, AxisLaunch* out) {
  ax::Args a{};
  a.tw = tab.d_tw;
  a.pos = tab.d_pos;
  a.L = tab.L;
  a.nst = tab.nst;
  a.contiguous = g.contiguous;
  // two tile buffers (the next tile's copies in flight during this one's
  // transform) unless they would leave one block per multiprocessor (the
  // 512-point strided passes, measured faster with one buffer and three
  // blocks)
  // (x pass: at least 16 rows, about 8192 points per tile, 4096 with two
  // buffers; y and z passes: 16 adjacent pencils, one 128-byte run per
  // element)
  // x pass: W consecutive rows; y and z passes: 16 adjacent pencils of
  // W / 16 consecutive slices (at most as many slices as there are, and W
  // at most the block's threads)
  auto tile_lw = [&](int nb) {
    int lw = 4;
    while (lw < (g.contiguous ? 9 : 8) && (tab.L << (lw + 1)) <= (nb == 2 ? 4096 : 8192) &&
           (g.contiguous || (1LL << (lw + 1 - 4)) <= g.outer))
      ++lw;
    return lw;
  };
  const int nbuf = ax::smem_bytes(tab.L, 1 << tile_lw(2), 2) <= 110 * 1024 ? 2 : 1;
  a.lw = tile_lw(nbuf);
  a.W = 1 << a.lw;
  int span = tab.L;
  for (int t = 0; t < tab.nst; ++t) {
    a.radix[t] = tab.radix[t];
    a.span[t] = span;
    a.sub[t] = span / tab.radix[t];
    a.twst[t] = tab.L / span;
    a.divsub[t] = make_fastdiv((unsigned)a.sub[t]);
    span = a.sub[t];
  }
  a.divL = make_fastdiv((unsigned)tab.L);
  // x pass: rotate pencils by bits of i / S for a power-of-two S = L / R_0
  // of at least 8 (the rotation turns the copies' conflict-free writes
  // into 2-way ones; it pays where the reads were 8- or 16-way: measured
  // 256^3 0.160 -> 0.187, slower at S = 4)
  a.swsh = 0;
  a.swmask = 0;
  const int S0 = tab.L / tab.radix[0];
  if (g.contiguous && S0 >= 8 && (S0 & (S0 - 1)) == 0) {
    while ((1 << a.swsh) < S0) ++a.swsh;
    a.swmask = 15;
  }
  long long ntiles;
  if (g.contiguous) {
    a.rows = g.rows;
    ntiles = (g.rows + a.W - 1) >> a.lw;
  } else {
    a.nx = g.nx;
    a.xtiles = (g.nx + 15) >> 4;
    a.outer = g.outer;
    a.d1 = g.d1;
    a.divx = make_fastdiv((unsigned)a.xtiles);
    a.divd1 = make_fastdiv((unsigned)g.d1);
    a.s1 = g.s1;
    a.s0 = g.s0;
    a.pi = g.pi;
    const long long G = a.W >> 4;
    ntiles = ((g.outer + G - 1) / G) * a.xtiles;
  }
  if (ntiles <= 0 || ntiles >= (1ll << 31)) return FFT3D_ERR_INVALID_ARG;
  a.ntiles = (unsigned)ntiles;
  a.scale = g.scale;
  a.do_scale = g.do_scale;
  const size_t smem = ax::smem_bytes(tab.L, a.W, nbuf);
  const void* fn = nbuf == 2 ? (dir < 0 ? (const void*)&ax::axis_pass_kernel<-1, 2>
                                        : (const void*)&ax::axis_pass_kernel<1, 2>)
                             : (dir < 0 ? (const void*)&ax::axis_pass_kernel<-1, 1>
                                        : (const void*)&ax::axis_pass_kernel<1, 1>);
  int per_sm = 0;
  if (smem > ax::kSmemLimit) return FFT3D_ERR_INVALID_ARG;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ax::kSmemLimit) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ax::kThreads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  out->args = a;
  out->dir = dir;
  out->nbuf = nbuf;
  out->smem = smem;
  out->grid = (int)std::min<long long>(ntiles, (long long)per_sm * sms);
  return FFT3D_SUCCESS;
}

cudaError_t launch_axis_pass(const AxisLaunch& l, const float2* in, float2* out,
                             cudaStream_t stream) {
  ax::Args a = l.args;
  a.in = in;
  a.out = out;
  if (l.nbuf == 2) {
    if (l.dir < 0)
      ax::axis_pass_kernel<-1, 2><<<l.grid, ax::kThreads, l.smem, stream>>>(a);
    else
      ax::axis_pass_kernel<1, 2><<<l.grid, ax::kThreads, l.smem, stream>>>(a);
  } else {
    if (l.dir < 0)
      ax::axis_pass_kernel<-1, 1><<<l.grid, ax::kThreads, l.smem, stream>>>(a);
    else
      ax::axis_pass_kernel<1, 1><<<l.grid, ax::kThreads, l.smem, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace fft3d

namespace fft3d {

static void fill_stages(const AxisTable& tab, AxisStages& st) {
  st.L = tab.L;
  st.nst = tab.nst;
  int span = tab.L;
  for (int t = 0; t < tab.nst; ++t) {
    st.radix[t] = tab.radix[t];
    st.span[t] = span;
    st.sub[t] = span / tab.radix[t];
    st.twst[t] = tab.L / span;
    st.divsub[t] = make_fastdiv((unsigned)st.sub[t]);
    span = st.sub[t];
  }
}

// One block per multiprocessor at most when the plane uses more than half
// of the shared memory; planes above 200 KB take the separate passes.
size_t plane_pass_smem(int nx, int ny) {
  const int px = nx | 1;
  const size_t b = ((size_t)ny * px + nx + ny) * sizeof(float2) + (size_t)(nx + ny) * sizeof(unsigned short);
  return b <= 200 * 1024 ? b : 0;
}

int prepare_plane_pass(const AxisTable& tx, const AxisTable& ty, int dir, long long planes, int sms,
                       PlaneLaunch* out) {
  const size_t smem = plane_pass_smem(tx.L, ty.L);
  if (!smem || planes <= 0 || planes >= (1ll << 31)) return FFT3D_ERR_INVALID_ARG;
  PlaneArgs a{};
  a.twx = tx.d_tw;
  a.posx = tx.d_pos;
  a.twy = ty.d_tw;
  a.posy = ty.d_pos;
  fill_stages(tx, a.sx);
  fill_stages(ty, a.sy);
  a.nx = tx.L;
  a.ny = ty.L;
  a.px = tx.L | 1;
  // rotation: S = nx / R_0 a power of two, nx a multiple of 16
  const int S0 = tx.L / tx.radix[0];
  a.rsh = 0;
  a.rmask = 0;
  if (tx.L % 16 == 0 && S0 >= 2 && (S0 & (S0 - 1)) == 0) {
    while ((1 << a.rsh) < S0) ++a.rsh;
    a.rmask = 15;
  }
  a.divnx = make_fastdiv((unsigned)tx.L);
  a.divny = make_fastdiv((unsigned)ty.L);
  a.nplanes = (unsigned)planes;
  const void* fn = dir < 0 ? (const void*)&ax::plane_pass_kernel<-1> : (const void*)&ax::plane_pass_kernel<1>;
  int per_sm = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ax::kPlaneThreads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  out->args = a;
  out->dir = dir;
  out->smem = smem;
  out->threads = ax::kPlaneThreads;
  out->grid = (int)std::min<long long>(planes, (long long)per_sm * sms);
  return FFT3D_SUCCESS;
}

cudaError_t launch_plane_pass(const PlaneLaunch& l, const float2* in, float2* out,
                              cudaStream_t stream) {
  PlaneArgs a = l.args;
  a.in = in;
  a.out = out;
  if (l.dir < 0)
    ax::plane_pass_kernel<-1><<<l.grid, ax::kPlaneThreads, l.smem, stream>>>(a);
  else
    ax::plane_pass_kernel<1><<<l.grid, ax::kPlaneThreads, l.smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace fft3d

extern "C" int fft3d_axis_digit_map(int n, int* nstages, int* radix, int* pos) {
  if (!nstages || !radix || !pos) return FFT3D_ERR_NULL_PTR;
  int r[fft3d::kAxisMaxStages];
  const int s = fft3d::axis_stages(n, r);
  if (!s) return FFT3D_ERR_UNSUPPORTED_SIZE;
  for (int t = 0; t < s; ++t) radix[t] = r[t];
  *nstages = s;
  fft3d::axis_positions(n, s, r, pos);
  return FFT3D_SUCCESS;
}
