// Persistent two-phase 3D FFT kernel for cubic n^3 grids (n in the fused
// size list), FP32 arithmetic.
//
// The paper (section "Approach") computes Eq. 1 as 1D FFTs along x, then y,
// then z, with a 2D transpose between x and y and a 3D transpose between y
// and z, the latter named as its bottleneck (section "Results").  Here the
// transposes are replaced by two kinds of work items that each hold a full
// n x n tile in shared memory:
//
//   plane item (g, z): load plane z of grid g (contiguous n*n points), 1D
//       FFTs along x (rows) and along y (columns) in shared memory, store the
//       plane to `out`.
//   slab item (g, y): load the n x n slab {(x, y, z)} of grid g at fixed y
//       from `out` (n rows of n contiguous points, stride n*n), 1D FFTs
//       along z, store it back to `out` (scaled).
//
// A slab item of grid g needs every plane item of grid g.  Blocks pull
// items from a global ticket counter in a fixed order that runs the plane
// items of grid g+1 before the slab items of grid g, so the intermediate of
// a grid is still in L2 when its slab items read it and each grid crosses
// HBM once in and once out.  A ticket holder only waits on smaller tickets,
// which running blocks already hold, so the scheme cannot deadlock whatever
// the number of resident blocks; each wait is still bounded in time and
// reports a timeout through the plan's status word instead of hanging.
#pragma once

#include "codelets.cuh"
#include "internal.h"
#include "sizes.h"
#include "tc_stage.cuh"

namespace fft3d {

// ------------------------------------------------------------ memory access
__device__ __forceinline__ float2 ld_stream(const float2* p) {  // read once
  float2 v;
  asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_l2(const float2* p) {  // bypass L1
  float2 v;
  asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_stream(float2* p, float2 v) {  // written once, final
  asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until *p >= target, at most timeout_ns of wall time and at most
// 2^24 polls.  Returns 1 when seen; 0 when it gave up (status set to
// kStatusTimeout) or another block already reported a failure.
static __device__ __noinline__ int bounded_wait_geq(const unsigned* p, unsigned target, unsigned* status,
                                             long long timeout_ns) {
  if (ld_acquire(p) >= target) return 1;
  const unsigned long long t0 = global_timer_ns();
  unsigned sleep_ns = 32;
  for (int iter = 0; iter < (1 << 24); ++iter) {
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns *= 2;
    if (ld_acquire(p) >= target) return 1;
    if (*(volatile unsigned*)status != kStatusOk) return 0;
    if ((long long)(global_timer_ns() - t0) > timeout_ns) break;
  }
  atomicCAS(status, kStatusOk, kStatusTimeout);
  return 0;
}

// ---------------------------------------------------------- tile transforms
// Plane item: n x n tile, rows padded to P = n + 1 complex so that lanes
// walking down a column or across rows hit distinct banks.
template <int N>
constexpr int plane_pitch() { return N + 1; }
template <int N>
constexpr int tile_elems() { return N * (N + 1); }

// STAGED: the plane is already in `tile` (row pitch N + 1) and visible to
// all threads; otherwise it is loaded from src first.
template <int N, int T, int DIR, int PREC = 0, bool STAGED = false>
__device__ __forceinline__ void plane_item(const float2* __restrict__ src, float2* __restrict__ dst,
                                           float2* tile, const float2* tw, const uint32_t* frag) {
  constexpr int L1 = item_l1(N, PREC), L2 = N / L1, P = plane_pitch<N>();
  const int tid = threadIdx.x;

  // (1) plane -> shared memory
  if constexpr (!STAGED) {
    constexpr int NE = N * N, PL = (NE + T - 1) / T;
    float2 r[PL];
#pragma unroll
    for (int i = 0; i < PL; ++i) {
      const int idx = tid + i * T;
      if (NE % T == 0 || idx < NE) r[i] = ld_stream(src + idx);
    }
#pragma unroll
    for (int i = 0; i < PL; ++i) {
      const int idx = tid + i * T;
      if (NE % T == 0 || idx < NE) tile[(idx / N) * P + idx % N] = r[i];
    }
    __syncthreads();
  }

  // (2) x, first step: per row, L1 DFTs of length L2 on stride-L1 points,
  //     times W_N^(n1 k2), in place.  Lanes walk rows.
  if constexpr (PREC != 0) {
    // 16 rows with the same n1 per warp and group, on tensor cores
    for (int grp = tid >> 5; grp < N * L1 / 16; grp += T / 32) {
      const int n1 = (grp * 16) / N, row0 = (grp * 16) % N;
      tc::dft16_group<PREC, DIR>(
          frag, [&](int v, int j) { return tile[(row0 + v) * P + n1 + L1 * j]; },
          [&](int v, int k, float2 y) {
            tile[(row0 + v) * P + n1 + L1 * k] = cmul_tw<DIR>(y, tw[k * L1 + n1]);
          });
    }
  } else {
    constexpr int IA = N * L1, PA = (IA + T - 1) / T;
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int item = tid + i * T;
      if (IA % T == 0 || item < IA) {
        const int row = item % N, n1 = item / N;
        float2* base = tile + row * P + n1;
        float2 v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[n2] = base[L1 * n2];
        DFT<L2, DIR>::run(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) base[L1 * k2] = v[k2];
      }
    }
  }
  __syncthreads();

  // (3) x, second step: L2 DFTs of length L1 on contiguous runs, output
  //     index k2 + L2 k1.  All reads land before any write.
  {
    constexpr int IB = N * L2, PB = (IB + T - 1) / T;
    float2 w[PB][L1];
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        const int row = item % N, k2 = item / N;
        const float2* base = tile + row * P + L1 * k2;
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
        const int row = item % N, k2 = item / N;
        float2* base = tile + row * P + k2;
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) base[L2 * k1] = w[i][k1];
      }
    }
  }
  __syncthreads();

  // (4) y, first step, lanes walk columns.
  if constexpr (PREC != 0) {
    for (int grp = tid >> 5; grp < N * L1 / 16; grp += T / 32) {
      const int n1 = (grp * 16) / N, col0 = (grp * 16) % N;
      tc::dft16_group<PREC, DIR>(
          frag, [&](int v, int j) { return tile[(n1 + L1 * j) * P + col0 + v]; },
          [&](int v, int k, float2 y) {
            tile[(n1 + L1 * k) * P + col0 + v] = cmul_tw<DIR>(y, tw[k * L1 + n1]);
          });
    }
  } else {
    constexpr int IA = N * L1, PA = (IA + T - 1) / T;
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int item = tid + i * T;
      if (IA % T == 0 || item < IA) {
        const int col = item % N, n1 = item / N;
        float2* base = tile + n1 * P + col;
        float2 v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[n2] = base[L1 * n2 * P];
        DFT<L2, DIR>::run(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) base[L1 * k2 * P] = v[k2];
      }
    }
  }
  __syncthreads();

  // (5) y, second step, straight to global memory (coalesced along x).
  {
    constexpr int IB = N * L2, PB = (IB + T - 1) / T;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        const int col = item % N, k2 = item / N;
        const float2* base = tile + (L1 * k2) * P + col;
        float2 w[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) w[n1] = base[n1 * P];
        DFT<L1, DIR>::run(w);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) dst[(k2 + L2 * k1) * N + col] = w[k1];
      }
    }
  }
}

// Slab item: src/dst point at (x = 0, y, z = 0) of a grid; element (x, z)
// of the slab is at x + z * N * N.
// STAGED: the slab is already in `tile` as [z][x] (pitch N) and visible to
// all threads; otherwise its first step reads it from src (L2).
template <int N, int T, int DIR, int PREC = 0, bool STAGED = false>
__device__ __forceinline__ void slab_item(const float2* src, float2* dst, float2* tile,
                                          const float2* tw, const uint32_t* frag, float scale,
                                          int do_scale) {
  constexpr int L1 = item_l1(N, PREC), L2 = N / L1;
  constexpr long long NN = (long long)N * N;
  const int tid = threadIdx.x;
  if constexpr (PREC != 0) {
    for (int grp = tid >> 5; grp < N * L1 / 16; grp += T / 32) {
      const int n1 = (grp * 16) / N, x0 = (grp * 16) % N;
      tc::dft16_group<PREC, DIR>(
          frag,
          [&](int v, int j) {
            if constexpr (STAGED) return tile[(n1 + L1 * j) * N + x0 + v];
            else return ld_l2(src + (n1 + L1 * j) * NN + x0 + v);
          },
          [&](int v, int k, float2 y) {
            tile[(n1 + L1 * k) * N + x0 + v] = cmul_tw<DIR>(y, tw[k * L1 + n1]);
          });
    }
  } else if constexpr (STAGED) {
    // each item reads and writes its own points of the tile
    constexpr int IA = N * L1, PA = (IA + T - 1) / T;
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int item = tid + i * T;
      if (IA % T == 0 || item < IA) {
        const int x = item % N, n1 = item / N;
        float2* base = tile + n1 * N + x;
        float2 v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[n2] = base[L1 * n2 * N];
        DFT<L2, DIR>::run(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) base[L1 * k2 * N] = v[k2];
      }
    }
  } else {
    constexpr int IA = N * L1, PA = (IA + T - 1) / T;
    float2 v[PA][L2];
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int item = tid + i * T;
      if (IA % T == 0 || item < IA) {
        const int x = item % N, n1 = item / N;
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[i][n2] = ld_l2(src + (n1 + L1 * n2) * NN + x);
      }
    }
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int item = tid + i * T;
      if (IA % T == 0 || item < IA) {
        const int x = item % N, n1 = item / N;
        DFT<L2, DIR>::run(v[i]);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) v[i][k2] = cmul_tw<DIR>(v[i][k2], tw[k2 * L1 + n1]);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) tile[(n1 + L1 * k2) * N + x] = v[i][k2];
      }
    }
  }
  __syncthreads();
  {
    constexpr int IB = N * L2, PB = (IB + T - 1) / T;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int item = tid + i * T;
      if (IB % T == 0 || item < IB) {
        const int x = item % N, k2 = item / N;
        float2 w[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) w[n1] = tile[(L1 * k2 + n1) * N + x];
        DFT<L1, DIR>::run(w);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
          float2 o = w[k1];
          if (do_scale) o = cscale(o, scale);
          st_stream(dst + (k2 + L2 * k1) * NN + x, o);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ kernel
template <int... Ns>
struct SizeList {
  static constexpr int count = sizeof...(Ns);
  static constexpr int tw_total = (0 + ... + Ns);
  static constexpr int max_tile = [] {
    int m = 0;
    ((m = tile_elems<Ns>() > m ? tile_elems<Ns>() : m), ...);
    return m;
  }();
  // twiddles, tensor-core B fragments (when used), tile
  static constexpr size_t smem_bytes(int prec) {
    return sizeof(float2) * (size_t)(tw_total + max_tile) +
           (prec ? sizeof(uint32_t) * tc::kFragWords : 0);
  }
};

// Offset of edge n's table inside the concatenation of the list's tables.
template <int... Ns>
__host__ __device__ constexpr int tw_offset(int n) {
  int off = 0, found = -1;
  ((found < 0 && Ns == n ? (found = off) : (off += Ns)), ...);
  return found;
}

// Input and output base of grid g (edge n) for either addressing mode.
__device__ __forceinline__ void grid_ptrs(const FusedArgs& a, int g, int n, const float2*& gin,
                                          float2*& gout) {
  if (a.grid_map) g = a.grid_map[g];
  if (a.in_ptrs) {
    gin = a.in_ptrs[g];
    gout = a.out_ptrs[g];
  } else {
    const long long off = a.grid_off ? a.grid_off[g] : (long long)g * n * n * n;
    gin = a.in + off;
    gout = a.out + off;
  }
}

template <int N, int T, int DIR, int PREC>
__device__ __forceinline__ void run_item(const FusedArgs& a, const SchedBlock& blk, int i,
                                         float2* tile, const float2* tw, const uint32_t* frag) {
  const float2* gin;
  float2* gout;
  grid_ptrs(a, blk.grid, N, gin, gout);
  if (blk.phase == 0) {
    const long long o = (long long)i * N * N;
    plane_item<N, T, DIR, PREC>(gin + o, gout + o, tile, tw, frag);
  } else {
    slab_item<N, T, DIR, PREC>(gout + (long long)i * N, gout + (long long)i * N, tile, tw, frag,
                               a.scale, a.do_scale);
  }
}

__device__ __forceinline__ int find_block(const SchedBlock* blocks, int nblocks, int item) {
  int lo = 0, hi = nblocks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blocks[mid].start <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int T, int DIR, int PREC, int... Ns>
__global__ void __launch_bounds__(T) fused_fft3d_kernel(const FusedArgs a) {
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int s_item, s_blk;
  using L = SizeList<Ns...>;
  float2* tws = smem;
  uint32_t* frag = reinterpret_cast<uint32_t*>(smem + L::tw_total);
  float2* tile = smem + L::tw_total + (PREC ? tc::kFragWords / 2 : 0);
  for (int i = threadIdx.x; i < L::tw_total; i += T) tws[i] = a.twiddles[i];
  if constexpr (PREC != 0)
    for (int i = threadIdx.x; i < tc::kFragWords; i += T) frag[i] = a.mma_frag[i];

  for (;;) {
    if (threadIdx.x == 0) {
      int item = -1, b = -1;
      if (*(volatile unsigned*)a.status == kStatusOk) item = (int)atomicAdd(a.work, 1u);
      if (item >= a.total_items) item = -1;
      if (item >= 0) {
        b = find_block(a.blocks, a.nblocks, item);
        const SchedBlock blk = a.blocks[b];
        if (blk.phase == 1 &&
            !bounded_wait_geq(a.work + 1 + blk.grid, (unsigned)blk.n, a.status, a.timeout_ns))
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
    ((blk.n == Ns ? (run_item<Ns, T, DIR, PREC>(a, blk, i, tile, tws + tw_offset<Ns...>(Ns), frag), 0)
                  : 0),
     ...);
    __syncthreads();
    if (blk.phase == 0 && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.work + 1 + blk.grid, 1u);
    }
  }
}

template <int T, int DIR, int PREC, int... Ns>
cudaError_t launch_fused(const FusedArgs& a, int grid, cudaStream_t stream) {
  fused_fft3d_kernel<T, DIR, PREC, Ns...>
      <<<grid, T, SizeList<Ns...>::smem_bytes(PREC), stream>>>(a);
  return cudaGetLastError();
}

template <int T, int DIR, int PREC, int... Ns>
KernelInfo make_fused_info_prec() {
  KernelInfo k;
  k.launch = &launch_fused<T, DIR, PREC, Ns...>;
  k.func = (const void*)&fused_fft3d_kernel<T, DIR, PREC, Ns...>;
  k.threads = T;
  k.smem = SizeList<Ns...>::smem_bytes(PREC);
  k.prec = PREC;
  k.twiddle_entries = SizeList<Ns...>::tw_total;
  const int sizes[] = {Ns...};
  k.nsizes = (int)sizeof...(Ns);
  for (int i = 0; i < k.nsizes; ++i) k.sizes[i] = sizes[i];
  return k;
}

template <int T, int DIR, int... Ns>
KernelInfo make_fused_info() {
  return make_fused_info_prec<T, DIR, 0, Ns...>();
}

}  // namespace fft3d
