// Whole-grid kernel for 16^3 grids: one block holds a grid in shared memory
// (32 KB) and runs the three passes of the paper's decomposition (x, then
// y, then z) with one thread per pencil -- 256 pencils of 16 points per
// pass, each a 16-point DFT in registers (compile-time twiddles) -- then
// writes the grid.  Blocks loop over the grids of the batch; no block waits
// for another, so there are no work counters, no schedule and no memset
// before the launch: one grid costs one short kernel, the latency the
// paper's non-batched setting measures.
//
// Shared layout: point (z, y, x) at z * 272 + y * 17 + x (row pitch 17, odd,
// so that the x pass -- lanes on consecutive rows -- is free of bank
// conflicts; the y and z passes put lanes on consecutive x).
#pragma once

#include "persistent.cuh"

namespace fft3d {
namespace wg {

template <int N>
struct Cfg {
  static_assert(N == 16, "the whole-grid kernel covers 16^3");
  static constexpr int T = N * N;            // one thread per pencil
  static constexpr int SY = N + 1, SZ = N * SY;
  static constexpr size_t smem = sizeof(float2) * (size_t)N * SZ;
};

template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::T) wholegrid_fft3d_kernel(const FusedArgs a) {
  using K = Cfg<N>;
  extern __shared__ __align__(16) float2 g[];
  const int t = threadIdx.x;
  for (int grid = blockIdx.x; grid < a.ngrids; grid += gridDim.x) {
    const float2* gin;
    float2* gout;
    grid_ptrs(a, grid, N, gin, gout);
    // load: thread t takes the points t + T i (consecutive threads,
    // consecutive points)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int e = t + K::T * i, z = e / (N * N), y = (e / N) % N, x = e % N;
      g[z * K::SZ + y * K::SY + x] = gin[e];
    }
    __syncthreads();
    float2 v[N];
    // x: row (z, y) = t
    {
      float2* row = g + (t / N) * K::SZ + (t % N) * K::SY;
#pragma unroll
      for (int x = 0; x < N; ++x) v[x] = row[x];
      DFT<N, DIR>::run(v);
#pragma unroll
      for (int x = 0; x < N; ++x) row[x] = v[x];
    }
    __syncthreads();
    // y: column (z, x) = t
    {
      float2* col = g + (t / N) * K::SZ + (t % N);
#pragma unroll
      for (int y = 0; y < N; ++y) v[y] = col[y * K::SY];
      DFT<N, DIR>::run(v);
#pragma unroll
      for (int y = 0; y < N; ++y) col[y * K::SY] = v[y];
    }
    __syncthreads();
    // z: pencil (y, x) = t, straight to global memory (lanes on consecutive x)
    {
      const float2* pen = g + (t / N) * K::SY + (t % N);
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = pen[z * K::SZ];
      DFT<N, DIR>::run(v);
      const float s = a.do_scale ? a.scale : 1.0f;
#pragma unroll
      for (int z = 0; z < N; ++z) st_stream(gout + z * N * N + t, cscale(v[z], s));
    }
    __syncthreads();  // the grid's shared copy is rewritten next
  }
}

template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  grid = grid < a.ngrids ? grid : a.ngrids;  // one block per grid at most
  wholegrid_fft3d_kernel<N, DIR><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&wholegrid_fft3d_kernel<N, DIR>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.twiddle_entries = N;  // (the codelets need no table; one is uploaded anyway)
  k.sizes[0] = N;
  k.nsizes = 1;
  k.uses_work = 0;  // no tickets: no counters to clear before a launch
  return k;
}

}  // namespace wg
}  // namespace fft3d
