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
//   y and z passes (strided): the W = 16 pencils at x0 .. x0 + 15 of one
//     (grid, z) or (grid, y) slice, element i of all 16 being one 128-byte
//     run in memory.
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

#include "../../include/fft3d.h"
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
    for (int r = 0; r < R; ++r) v[r] = tile[(i0 + r * M) * P + q];
    DFT<R, DIR>::run(v);
    const int st = j * stw;  // W_N^(j k) = W_L^(j k L / N); j k L / N < L
    if (st) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul_tw<DIR>(v[k], tw[k * st]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) tile[(i0 + k * M) * P + q] = v[k];
  }
}

template <int DIR>
__global__ void __launch_bounds__(kThreads) axis_pass_kernel(const Args a) {
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.W + 1;
  float2* tile = sm;
  float2* tw = sm + (size_t)a.L * P;
  unsigned short* pos = reinterpret_cast<unsigned short*>(tw + a.L);
  for (int i = threadIdx.x; i < a.L; i += kThreads) {
    tw[i] = a.tw[i];
    pos[i] = a.pos[i];
  }
  const int pts = a.L << a.lw;
  for (unsigned t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    long long base;
    int nv;
    if (a.contiguous) {
      const long long r0 = (long long)t << a.lw;
      nv = (int)min((long long)a.W, a.rows - r0);
      base = r0 * a.L;
      const float2* src = a.in + base;
      for (int e = threadIdx.x; e < nv * a.L; e += kThreads) {
        const unsigned q = fdiv((unsigned)e, a.divL);
        tile[(e - (int)q * a.L) * P + (int)q] = src[e];
      }
    } else {
      const unsigned outer = fdiv(t, a.divx);
      const int x0 = (int)(t - outer * (unsigned)a.xtiles) << a.lw;
      nv = min(a.W, a.nx - x0);
      const unsigned o1 = fdiv(outer, a.divd1);
      base = (long long)o1 * a.s1 + (long long)(outer - o1 * (unsigned)a.d1) * a.s0 + x0;
      for (int e = threadIdx.x; e < pts; e += kThreads) {
        const int q = e & (a.W - 1), i = e >> a.lw;
        if (q < nv) tile[i * P + q] = a.in[base + q + i * a.pi];
      }
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
    if (a.contiguous) {
      float2* dst = a.out + base;
      for (int e = threadIdx.x; e < nv * a.L; e += kThreads) {
        const unsigned q = fdiv((unsigned)e, a.divL);
        dst[e] = cscale(tile[pos[e - (int)q * a.L] * P + (int)q], sc);
      }
    } else {
      for (int e = threadIdx.x; e < pts; e += kThreads) {
        const int q = e & (a.W - 1), k = e >> a.lw;
        if (q < nv) a.out[base + q + k * a.pi] = cscale(tile[pos[k] * P + q], sc);
      }
    }
    __syncthreads();  // the tile is reloaded next
  }
}

constexpr int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

size_t smem_bytes(int L, int W) {
  return ((size_t)L * (W + 1) + L) * sizeof(float2) + (size_t)L * sizeof(unsigned short);
}
// The largest smem_bytes of any pass (L W <= 8192 pencil points, L <= 512):
// the kernel's dynamic shared-memory limit is set once to this, since the
// passes of one plan (different L and W) share the kernel.
constexpr size_t kSmemLimit = (8192 + 2 * 512) * sizeof(float2) + 512 * sizeof(unsigned short);

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
  if (g.contiguous) {
    int lw = 4;  // at least 16 rows, about 8192 points per tile
    while (lw < 9 && (tab.L << (lw + 1)) <= 8192) ++lw;
    a.lw = lw;
  } else {
    a.lw = 4;  // 16 adjacent pencils: one 128-byte run per element
  }
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
  long long ntiles;
  if (g.contiguous) {
    a.rows = g.rows;
    ntiles = (g.rows + a.W - 1) >> a.lw;
  } else {
    a.nx = g.nx;
    a.xtiles = (g.nx + a.W - 1) >> a.lw;
    a.d1 = g.d1;
    a.divx = make_fastdiv((unsigned)a.xtiles);
    a.divd1 = make_fastdiv((unsigned)g.d1);
    a.s1 = g.s1;
    a.s0 = g.s0;
    a.pi = g.pi;
    ntiles = g.outer * a.xtiles;
  }
  if (ntiles <= 0 || ntiles >= (1ll << 31)) return FFT3D_ERR_INVALID_ARG;
  a.ntiles = (unsigned)ntiles;
  a.scale = g.scale;
  a.do_scale = g.do_scale;
  const size_t smem = ax::smem_bytes(tab.L, a.W);
  const void* fn =
      dir < 0 ? (const void*)&ax::axis_pass_kernel<-1> : (const void*)&ax::axis_pass_kernel<1>;
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
  out->smem = smem;
  out->grid = (int)std::min<long long>(ntiles, (long long)per_sm * sms);
  return FFT3D_SUCCESS;
}

cudaError_t launch_axis_pass(const AxisLaunch& l, const float2* in, float2* out,
                             cudaStream_t stream) {
  ax::Args a = l.args;
  a.in = in;
  a.out = out;
  if (l.dir < 0)
    ax::axis_pass_kernel<-1><<<l.grid, ax::kThreads, l.smem, stream>>>(a);
  else
    ax::axis_pass_kernel<1><<<l.grid, ax::kThreads, l.smem, stream>>>(a);
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
