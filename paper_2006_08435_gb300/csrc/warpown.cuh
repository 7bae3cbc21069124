// Persistent two-phase 3D FFT kernel with warp-owned work inside an item
// (64^3 and 128^3, split n = 8 * L2).
//
// Same items, tickets and schedule as the persistent kernel, but each warp
// owns 8 rows in the x step and 8 columns in the y and z steps, and moves
// its data between global memory and registers itself: the first step of an
// axis loads straight into registers (four 64-byte row segments per
// instruction), the second step stores straight from registers.  Shared
// memory only carries the in-axis exchange and the x -> y transpose, so a
// plane item has one block-wide barrier (the transpose) and a slab item none
// besides the ticket hand-off.
//
// Shared-memory layout: rows of pitch n + 8 complex, with the column index of
// row r XORed with 8 * ((r >> 3) & 1); between the two x steps a row is held
// transposed as [n1][k2 ^ n1].  With this every access of every step is free
// of bank conflicts (two rows of a half-warp always land in different
// 8-bank halves, and the XOR separates rows 8 apart).
#pragma once

#include "persistent.cuh"

namespace fft3d {
namespace wown {

template <int N>
struct Cfg {
  static constexpr int L1 = split_l1(N), L2 = split_l2(N);
  static_assert(L1 == 8 && (N == 64 || N == 128), "warp-owned kernel covers 64 and 128");
  static constexpr int P = N + 8;
  static constexpr int T = 4 * N;  // N / 8 warps
  static constexpr int TILE = N * P;
  static constexpr int MINB = N == 64 ? 3 : 1;  // blocks per SM the registers must allow
};

// physical index of (row, col) in the tile
template <int N>
__device__ __forceinline__ int at(int row, int col) {
  return row * Cfg<N>::P + (col ^ (((row >> 3) & 1) << 3));
}

template <int N, int DIR>
__device__ __forceinline__ void plane(const float2* __restrict__ src, float2* __restrict__ dst,
                                      float2* tile, const float2* tw) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r0 = 8 * w;
  // x, first step: global -> registers; rows r0 + (lane >> 3) + 4 i
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int n1 = lane & 7, row = r0 + (lane >> 3) + 4 * i;
    const float2* rp = src + (long long)row * N + n1;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = ld_stream(rp + L1 * n2);
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) tile[at<N>(row, n1 * L2 + (k2 ^ n1))] = v[k2];
  }
  __syncwarp();
  // x, second step on the warp's rows
  constexpr int RPI = 32 / L2;  // rows per lane iteration
  float2 w2[8 / RPI][L1];
#pragma unroll
  for (int i = 0; i < 8 / RPI; ++i) {
    const int k2 = lane % L2, row = r0 + lane / L2 + RPI * i;
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) w2[i][n1] = tile[at<N>(row, n1 * L2 + (k2 ^ n1))];
    DFT<L1, DIR>::run(w2[i]);
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8 / RPI; ++i) {
    const int k2 = lane % L2, row = r0 + lane / L2 + RPI * i;
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) tile[at<N>(row, k2 + L2 * k1)] = w2[i][k1];
  }
  __syncthreads();  // the transpose: every row before any column
  // y, first step on columns c0 .. c0 + 7, in place
  const int col = 8 * w + (lane & 7);
#pragma unroll
  for (int i = 0; i < L1 / 4; ++i) {
    const int n1 = (lane >> 3) + 4 * i;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = tile[at<N>(n1 + L1 * n2, col)];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) tile[at<N>(n1 + L1 * k2, col)] = v[k2];
  }
  __syncwarp();
  // y, second step: registers -> global
#pragma unroll
  for (int i = 0; i < L2 / 4; ++i) {
    const int k2 = (lane >> 3) + 4 * i;
    float2 v[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) v[n1] = tile[at<N>(L1 * k2 + n1, col)];
    DFT<L1, DIR>::run(v);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) dst[(long long)(k2 + L2 * k1) * N + col] = v[k1];
  }
}

// src/dst at (x = 0, y, z = 0) of the grid; columns x = 8 w .. 8 w + 7.
template <int N, int DIR>
__device__ __forceinline__ void slab(const float2* src, float2* dst, float2* tile,
                                     const float2* tw, float scale, int do_scale) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2;
  constexpr long long NN = (long long)N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x = 8 * w + (lane & 7);
#pragma unroll
  for (int i = 0; i < L1 / 4; ++i) {
    const int n1 = (lane >> 3) + 4 * i;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = ld_l2(src + (n1 + L1 * n2) * NN + x);
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) tile[at<N>(n1 + L1 * k2, x)] = v[k2];
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < L2 / 4; ++i) {
    const int k2 = (lane >> 3) + 4 * i;
    float2 v[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) v[n1] = tile[at<N>(L1 * k2 + n1, x)];
    DFT<L1, DIR>::run(v);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) {
      float2 o = v[k1];
      if (do_scale) o = cscale(o, scale);
      st_stream(dst + (k2 + L2 * k1) * NN + x, o);
    }
  }
}

template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::T, Cfg<N>::MINB) wown_fft3d_kernel(const FusedArgs a) {
  using K = Cfg<N>;
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int s_item, s_blk;
  float2* tw = smem;
  float2* tile = smem + N;
  for (int i = threadIdx.x; i < N; i += K::T) tw[i] = a.twiddles[i];
  for (;;) {
    if (threadIdx.x == 0) {
      int item = -1, b = -1;
      if (*(volatile unsigned*)a.status == kStatusOk) item = (int)atomicAdd(a.work, 1u);
      if (item >= a.total_items) item = -1;
      if (item >= 0) {
        b = find_block(a.blocks, a.nblocks, item);
        const SchedBlock blk = a.blocks[b];
        if (blk.phase == 1 &&
            !bounded_wait_geq(a.work + 1 + blk.grid, (unsigned)N, a.status, a.timeout_ns))
          item = -1;
      }
      s_item = item;
      s_blk = b;
    }
    __syncthreads();
    const int item = s_item;
    if (item < 0) break;
    const SchedBlock blk = a.blocks[s_blk];
    const int i = item - blk.start;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, blk.grid, N, gin, gout);
    if (blk.phase == 0) {
      const long long o = (long long)i * N * N;
      plane<N, DIR>(gin + o, gout + o, tile, tw);
    } else {
      slab<N, DIR>(gout + (long long)i * N, gout + (long long)i * N, tile, tw, a.scale,
                   a.do_scale);
    }
    __syncthreads();  // stores issued, tile and s_* free
    if (blk.phase == 0 && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.work + 1 + blk.grid, 1u);
    }
  }
}

template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  wown_fft3d_kernel<N, DIR><<<grid, Cfg<N>::T, sizeof(float2) * (N + Cfg<N>::TILE), stream>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&wown_fft3d_kernel<N, DIR>;
  k.threads = Cfg<N>::T;
  k.smem = sizeof(float2) * (N + Cfg<N>::TILE);
  k.twiddle_entries = N;
  k.sizes[0] = N;
  k.nsizes = 1;
  return k;
}

}  // namespace wown
}  // namespace fft3d
