// Cluster-fused single-pass 3D FFT for small cubic grids (16^3, 32^3).
//
// The paper's design keeps the whole 3D FFT in the FPGA's local memory when
// it fits, so the 3D transpose happens on chip (section "Approach").  Here a
// thread-block cluster of C blocks plays that role: block r of the cluster
// holds planes z in [r n/C, (r+1) n/C) of one grid in shared memory, does
// their x and y transforms locally, and after a cluster barrier reads the z
// pencils of its slabs y in [r n/C, (r+1) n/C) from all blocks' shared
// memory (distributed shared memory), transforms them and writes the result.
// The grid crosses HBM once in and once out; no block ever waits for
// another cluster.  Clusters loop over the grids of the batch.
//
// Shapes: 16^3 over 8 blocks, 32^3 over 16 (a non-portable cluster size),
// two planes per block: for the few grids this kernel serves (it is the
// default below 128 grids at 16^3 and 32^3), spreading a grid
// over more multiprocessors cuts the x-y and z steps to a fraction, and
// the cluster barrier between them costs less than the counters, memset
// and inter-block waits of the persistent kernels (one grid with L2
// flushed: 8.9 us at 16^3 against 11.9 us; 10.9 us at 32^3 against 11.9).
// Narrower clusters (16^3 in one block, 32^3 over 4) were slower at every
// batch; from 128 grids the whole-grid (16^3) and thread-pair (32^3)
// kernels take over.
#pragma once

#include <cooperative_groups.h>

#include "persistent.cuh"

namespace fft3d {
namespace clus {

namespace cg = cooperative_groups;

template <int N>
constexpr int cluster_size() {
  static_assert(N == 16 || N == 32, "cluster-fused kernel covers 16^3 and 32^3");
  return N == 16 ? 8 : 16;
}

template <int N, int CS = cluster_size<N>()>
struct Cfg {
  static constexpr int C = CS;
  static constexpr int PL = N / C;        // planes (and slabs) per block
  static constexpr int P = N + 1;         // plane row pitch (complex)
  static constexpr int L1 = split_l1(N), L2 = split_l2(N);
  static constexpr int T = 256;
  static constexpr size_t smem = sizeof(float2) * ((size_t)PL * N * P + (size_t)N * N + N);
};

// In-place x then y transform of one n x n plane with row pitch P.
template <int N, int DIR>
__device__ __forceinline__ void plane_xy(float2* pl, const float2* tw) {
  using K = Cfg<N>;  // (the pitch and the split do not depend on C)
  constexpr int L1 = K::L1, L2 = K::L2, P = K::P, T = K::T;
  const int tid = threadIdx.x;
  // x, first step (lanes walk rows; each item reads and writes its own points)
  for (int item = tid; item < N * L1; item += T) {
    const int row = item % N, n1 = item / N;
    float2* base = pl + row * P + n1;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = base[L1 * n2];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) base[L1 * k2] = v[k2];
  }
  __syncthreads();
  // x, second step: all reads, then all writes
  {
    constexpr int IB = N * L2, PB = (IB + T - 1) / T;
    float2 w[PB][L1];
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        const float2* base = pl + (item % N) * P + L1 * (item / N);
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) w[i][n1] = base[n1];
        DFT<L1, DIR>::run(w[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        float2* base = pl + (item % N) * P + item / N;
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) base[L2 * k1] = w[i][k1];
      }
    }
  }
  __syncthreads();
  // y, first step (lanes walk columns)
  for (int item = tid; item < N * L1; item += T) {
    const int col = item % N, n1 = item / N;
    float2* base = pl + n1 * P + col;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = base[L1 * n2 * P];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) base[L1 * k2 * P] = v[k2];
  }
  __syncthreads();
  // y, second step: all reads, then all writes
  {
    constexpr int IB = N * L2, PB = (IB + T - 1) / T;
    float2 w[PB][L1];
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        const float2* base = pl + (L1 * (item / N)) * P + item % N;
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) w[i][n1] = base[n1 * P];
        DFT<L1, DIR>::run(w[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        float2* base = pl + (item / N) * P + item % N;
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) base[L2 * k1 * P] = w[i][k1];
      }
    }
  }
  __syncthreads();
}

template <int N, int DIR, int CS>
__global__ void __launch_bounds__(Cfg<N, CS>::T) cluster_fft3d_kernel(const FusedArgs a) {
  using K = Cfg<N, CS>;
  constexpr int L1 = K::L1, L2 = K::L2, P = K::P, T = K::T, PL = K::PL;
  constexpr long long NN = (long long)N * N;
  extern __shared__ __align__(16) float2 smem[];
  float2* tw = smem;
  float2* planes = smem + N;                    // [PL][N][P]
  float2* scratch = planes + (size_t)PL * N * P;  // [N z][N x]
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / K::C, ncl = gridDim.x / K::C;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += T) tw[i] = a.twiddles[i];
  __syncthreads();
  for (int g = cid; g < a.ngrids; g += ncl) {
    const float2* gin;
    float2* gout;
    grid_ptrs(a, g, N, gin, gout);
    // this block's planes: contiguous in HBM
    const float2* src = gin + (long long)rank * PL * NN;
    for (long long i = tid; i < PL * NN; i += T) {
      const int pz = (int)(i / NN), rem = (int)(i % NN);
      planes[(size_t)pz * N * P + (rem / N) * P + rem % N] = ld_stream(src + i);
    }
    __syncthreads();
    for (int pz = 0; pz < PL; ++pz) plane_xy<N, DIR>(planes + (size_t)pz * N * P, tw);
    cluster.sync();  // every block's planes hold their x-y transforms
    for (int sy = 0; sy < PL; ++sy) {
      const int y = rank * PL + sy;
      // z, first step: point z = n1 + L1 n2 lives in block z / PL, plane z % PL
      for (int item = tid; item < N * L1; item += T) {
        const int x = item % N, n1 = item / N;
        float2 v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) {
          const int z = n1 + L1 * n2;
          v[n2] = *cluster.map_shared_rank(planes + (size_t)(z % PL) * N * P + y * P + x, z / PL);
        }
        DFT<L2, DIR>::run(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) scratch[(n1 + L1 * k2) * N + x] = v[k2];
      }
      __syncthreads();
      for (int item = tid; item < N * L2; item += T) {
        const int x = item % N, k2 = item / N;
        float2 w[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) w[n1] = scratch[(L1 * k2 + n1) * N + x];
        DFT<L1, DIR>::run(w);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
          float2 o = w[k1];
          if (a.do_scale) o = cscale(o, a.scale);
          st_stream(gout + (k2 + L2 * k1) * NN + (long long)y * N + x, o);
        }
      }
      __syncthreads();
    }
    cluster.sync();  // no block reloads its planes while others still read them
  }
}

template <int N, int DIR, int CS>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  using K = Cfg<N, CS>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = K::C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(K::T, 1, 1);
  cfg.dynamicSmemBytes = K::smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cluster_fft3d_kernel<N, DIR, CS>, a);
}

template <int N, int DIR, int CS = cluster_size<N>()>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR, CS>;
  k.func = (const void*)&cluster_fft3d_kernel<N, DIR, CS>;
  k.threads = Cfg<N, CS>::T;
  k.smem = Cfg<N, CS>::smem;
  k.twiddle_entries = N;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.cluster = Cfg<N, CS>::C;
  return k;
}

}  // namespace clus
}  // namespace fft3d
