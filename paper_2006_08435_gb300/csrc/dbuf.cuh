// Double-buffered, TMA-fed persistent 3D FFT kernel for 64^3 grids.
//
// Same plane and slab items and the same ticket schedule as the persistent
// kernel, with two blocks per SM, each holding three item tiles in shared
// memory: while its eight compute warps transform the item in one tile, a
// producer warp has already streamed the next two items into the others with
// 1D bulk copies (cp.async.bulk, the TMA engine), one per row of 64 points,
// completing on an mbarrier per tile.  The producer takes the tickets (one
// ahead) and waits for slab dependencies; a signaller warp publishes finished
// plane items and hands tiles back to the producer.  None of those round
// trips sits on the compute warps' path.
//
// Compute warps own rows (x step) and columns (y, z steps) as in the
// warp-owned kernel: a plane item has one barrier among the compute warps
// (the x -> y transpose), a slab item none.  Tile layout: row r at
// r * (n + 8) + 8 * ((r >> 3) & 1) complex -- rows 16-byte aligned for the
// bulk copies, and rows 8 apart shifted by 8 banks -- and between the two x
// steps a row is held as [n1][k2 ^ n1].  Every shared-memory access of every
// step is then free of bank conflicts, and in the y and z steps each lane
// reads and writes only its own points.
//
// Liveness: a block's started items finish and are published without the
// producer, so the producer's wait for a slab's planes is a wait on smaller
// tickets only, as in the persistent kernel.
// Every wait is bounded; on expiry the status word records a timeout and
// the warps leave their loops.
#pragma once

#include "pipelined.cuh"

namespace fft3d {
namespace dbuf {

using piped::bulk_g2s;
using piped::mbar_arrive;
using piped::mbar_arrive_tx;
using piped::mbar_init;
using piped::mbar_wait_bounded;
using piped::warp_wait;

template <int N>
struct Cfg {
  static constexpr int L1 = split_l1(N), L2 = split_l2(N);
  static_assert(N == 64 && L1 == 8 && L2 == 8, "double-buffered kernel covers 64");
  static constexpr int P = N + 8;
  static constexpr int TILE = N * P;
  static constexpr int NCW = N / 8;          // compute warps
  static constexpr int T = 32 * (NCW + 2);   // plus a producer and a signaller warp
  static constexpr int NTILE = 3;            // tiles per block
  static constexpr unsigned ROW_BYTES = N * sizeof(float2);
  static constexpr size_t smem = sizeof(float2) * (N + NTILE * (size_t)TILE) +
                                 (3 * NTILE + 1) * sizeof(unsigned long long) + NTILE * sizeof(int4);
};

// tile index of (row, col)
template <int N>
__device__ __forceinline__ int pos(int r, int c) {
  return r * Cfg<N>::P + c + (((r >> 3) & 1) << 3);
}

// x and y transforms of a plane staged in `t`; output rows to dst (plane z).
// Returns 0 if the wait at the transpose gave up (the item is abandoned).
template <int N, int DIR>
__device__ __forceinline__ int plane(float2* t, float2* __restrict__ dst, const float2* tw,
                                     unsigned long long* xy, unsigned parity, const FusedArgs& a) {
  constexpr int L1 = Cfg<N>::L1, L2 = Cfg<N>::L2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // x, first step on rows 8w + (lane >> 3) + 4i, n1 = lane & 7
  {
    const int n1 = lane & 7;
    float2 v[2][L2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int row = 8 * w + (lane >> 3) + 4 * i;
#pragma unroll
      for (int n2 = 0; n2 < L2; ++n2) v[i][n2] = t[pos<N>(row, n1 + L1 * n2)];
    }
    __syncwarp();  // every lane of the row has read it
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int row = 8 * w + (lane >> 3) + 4 * i;
      DFT<L2, DIR>::run(v[i]);
#pragma unroll
      for (int k2 = 1; k2 < L2; ++k2) v[i][k2] = cmul_tw<DIR>(v[i][k2], tw[k2 * L1 + n1]);
      float2* rp = t + pos<N>(row, 0) + n1 * L2;
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) rp[k2 ^ n1] = v[i][k2];
    }
  }
  __syncwarp();
  // x, second step: rows 8w + lane / 8 + 4i, k2 = lane % 8
  {
    const int k2 = lane & 7;
    float2 u[2][L1];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float2* rp = t + pos<N>(8 * w + (lane >> 3) + 4 * i, 0);
#pragma unroll
      for (int n1 = 0; n1 < L1; ++n1) u[i][n1] = rp[n1 * L2 + (k2 ^ n1)];
      DFT<L1, DIR>::run(u[i]);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float2* rp = t + pos<N>(8 * w + (lane >> 3) + 4 * i, 0);
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1) rp[k2 + L2 * k1] = u[i][k1];
    }
  }
  // the transpose: every compute warp's rows before any column
  __syncwarp();
  if (lane == 0) mbar_arrive(xy);
  if (!warp_wait(xy, parity, a)) return 0;
  // y, first step on columns 8w .. 8w + 7, in place (each lane its own points)
  const int col = 8 * w + (lane & 7);
#pragma unroll
  for (int i = 0; i < L1 / 4; ++i) {
    const int n1 = (lane >> 3) + 4 * i;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = t[pos<N>(n1 + L1 * n2, col)];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) t[pos<N>(n1 + L1 * k2, col)] = v[k2];
  }
  __syncwarp();
  // y, second step: registers -> global
#pragma unroll
  for (int i = 0; i < L2 / 4; ++i) {
    const int k2 = (lane >> 3) + 4 * i;
    float2 u[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) u[n1] = t[pos<N>(L1 * k2 + n1, col)];
    DFT<L1, DIR>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) dst[(long long)(k2 + L2 * k1) * N + col] = u[k1];
  }
  return 1;
}

// z transform of a slab staged in `t` (row z); output rows to dst (slab y,
// rows N*N apart).
template <int N, int DIR>
__device__ __forceinline__ void slab(float2* t, float2* dst, const float2* tw, float scale,
                                     int do_scale) {
  constexpr int L1 = Cfg<N>::L1, L2 = Cfg<N>::L2;
  constexpr long long NN = (long long)N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x = 8 * w + (lane & 7);
#pragma unroll
  for (int i = 0; i < L1 / 4; ++i) {
    const int n1 = (lane >> 3) + 4 * i;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = t[pos<N>(n1 + L1 * n2, x)];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) t[pos<N>(n1 + L1 * k2, x)] = v[k2];
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < L2 / 4; ++i) {
    const int k2 = (lane >> 3) + 4 * i;
    float2 u[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) u[n1] = t[pos<N>(L1 * k2 + n1, x)];
    DFT<L1, DIR>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) {
      float2 o = u[k1];
      if (do_scale) o = cscale(o, scale);
      st_stream(dst + (k2 + L2 * k1) * NN + x, o);
    }
  }
}

// Item descriptor of a tile: ticket (-1 = stop), grid, phase, plane z / slab y.
struct Desc {
  int item, grid, phase, idx;
};

// ----------------------------------------------------- producer, signaller
__device__ __forceinline__ Desc bcast(Desc d) {
  d.item = __shfl_sync(0xffffffffu, d.item, 0);
  d.grid = __shfl_sync(0xffffffffu, d.grid, 0);
  d.phase = __shfl_sync(0xffffffffu, d.phase, 0);
  d.idx = __shfl_sync(0xffffffffu, d.idx, 0);
  return d;
}

// Producer warp: tickets in order into tiles 0, 1, .., NT-1, 0, ...  A tile
// is refilled once the signaller has recorded its previous item.  A slab
// waits (bounded) for its grid's planes before its rows are copied; the
// block's earlier items need nothing from the producer to finish, so the
// wait cannot close a cycle.
template <int N>
__device__ __forceinline__ void producer(const FusedArgs& a, float2* tiles,
                                         unsigned long long* full, unsigned long long* freed,
                                         Desc* desc) {
  constexpr int NT = Cfg<N>::NTILE;
  constexpr long long NN = (long long)N * N;
  const int lane = threadIdx.x & 31;
  auto take = [&]() -> int {
    return *(volatile unsigned*)a.status == kStatusOk ? (int)atomicAdd(a.work, 1u) : a.total_items;
  };
  unsigned live = 0;  // tiles whose copies were issued (bit s)
  int next = lane == 0 ? take() : 0;
  int k = 0;
  for (;; ++k) {
    const int s = k % NT;
    if (k >= NT && !__all_sync(0xffffffffu, mbar_wait_bounded(&freed[s], (k / NT - 1) & 1,
                                                               a.status, a.timeout_ns)))
      break;
    live &= ~(1u << s);
    int st = 0;  // 0 copy, -1 stop
    Desc d{-1, 0, 0, 0};
    if (lane == 0) {
      const int t = next;
      next = take();  // one ticket ahead: its round trip overlaps this item
      if (t >= a.total_items) {
        st = -1;
      } else {
        const SchedBlock blk = a.blocks[t / N];  // N tickets per block (one edge)
        d = Desc{t, blk.grid, blk.phase, t - blk.start};
        if (blk.phase == 1 &&
            !bounded_wait_geq(a.work + 1 + blk.grid, (unsigned)N, a.status, a.timeout_ns))
          st = -1;
      }
      desc[s] = d;
      if (st < 0) {
        mbar_arrive(&full[s]);
      } else {
        // the tile was last written by the compute warps' plain stores, a
        // slab's rows by other blocks' plain stores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (d.phase == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
        mbar_arrive_tx(&full[s], (unsigned)(N * Cfg<N>::ROW_BYTES));
      }
    }
    st = __shfl_sync(0xffffffffu, st, 0);
    if (st < 0) break;
    d = bcast(d);
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2* t = tiles + (size_t)s * Cfg<N>::TILE;
    for (int r = lane; r < N; r += 32) {
      const float2* src = d.phase == 0 ? gin + d.idx * NN + (long long)r * N
                                       : gout + r * NN + (long long)d.idx * N;
      bulk_g2s(t + pos<N>(r, 0), src, Cfg<N>::ROW_BYTES, &full[s]);
    }
    live |= 1u << s;
  }
  // no bulk copy may still be writing a tile when the block exits (only on
  // a failure can a tile be left unconsumed)
  for (int j = 1; j <= NT; ++j) {
    const int kk = k - j;
    if (kk >= 0 && (live & (1u << (kk % NT))))
      mbar_wait_bounded(&full[kk % NT], (kk / NT) & 1, a.status, a.timeout_ns);
  }
}

// Signaller warp: for each item in order, once the compute warps are done
// with it, frees its tile for the producer and, for a plane, publishes it to
// the other blocks (the GPU-scope release waits for the compute warps'
// stores, so it is kept off their path).
template <int N>
__device__ __forceinline__ void signaller(const FusedArgs& a, unsigned long long* full,
                                          unsigned long long* empty,
                                          unsigned long long* freed, Desc* desc) {
  constexpr int NT = Cfg<N>::NTILE;
  const int lane = threadIdx.x & 31;
  for (int k = 0;; ++k) {
    const int s = k % NT;
    const unsigned par = (k / NT) & 1;
    if (!warp_wait(&full[s], par, a)) return;
    const Desc d = desc[s];
    if (d.item < 0) return;
    if (!warp_wait(&empty[s], par, a)) return;
    if (lane == 0) {
      mbar_arrive(&freed[s]);
      if (d.phase == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        atomicAdd(a.work + 1 + d.grid, 1u);
      }
    }
    __syncwarp();
  }
}

template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::T, 2) dbuf_fft3d_kernel(const FusedArgs a) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE;
  extern __shared__ __align__(16) float2 smem[];
  float2* tw = smem;
  float2* tiles = smem + N;
  unsigned long long* full = reinterpret_cast<unsigned long long*>(tiles + NT * (size_t)K::TILE);
  unsigned long long* empty = full + NT;
  unsigned long long* freed = empty + NT;
  unsigned long long* xy = freed + NT;  // transpose barrier of the compute warps
  Desc* desc = reinterpret_cast<Desc*>(xy + 1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < N; i += K::T) tw[i] = a.twiddles[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < NT; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], K::NCW);
      mbar_init(&freed[s], 1);
    }
    mbar_init(xy, K::NCW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (w == K::NCW) {
    producer<N>(a, tiles, full, freed, desc);
    return;
  }
  if (w == K::NCW + 1) {
    signaller<N>(a, full, empty, freed, desc);
    return;
  }

  // compute warps
  unsigned planes = 0;  // plane items done (parity of the transpose barrier)
  for (int k = 0;; ++k) {
    const int s = k % NT;
    if (!warp_wait(&full[s], (k / NT) & 1, a)) break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    float2* t = tiles + (size_t)s * K::TILE;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    if (d.phase == 0) {
      if (!plane<N, DIR>(t, gout + (long long)d.idx * N * N, tw, xy, planes & 1, a)) break;
      ++planes;
    } else {
      slab<N, DIR>(t, gout + (long long)d.idx * N, tw, a.scale, a.do_scale);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  dbuf_fft3d_kernel<N, DIR><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&dbuf_fft3d_kernel<N, DIR>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.twiddle_entries = N;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 1;  // the tiles and one ticket held ahead
  return k;
}

}  // namespace dbuf
}  // namespace fft3d
