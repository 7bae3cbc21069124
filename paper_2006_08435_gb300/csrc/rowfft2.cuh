// Thread-per-pencil persistent 3D FFT kernel for 64^3 grids with two-plane
// work items: the kernel of rowfft.cuh with each ticket covering two
// consecutive planes (or slabs) of a grid, 64 KB, so that the producer's
// per-ticket work (ticket, schedule lookup, slab dependency, four tensor
// copies, publication) is spread over twice the data.
//
//   plane-pair item (g, z0): planes z0, z0 + 1; thread t of the group takes
//     row t % 64 of plane t / 64 (x), then column t % 64 (y).
//   slab-pair item (g, y0): slabs y0, y0 + 1; thread t takes column t % 64
//     of slab t / 64 (z).
//
// Each box of a tensor copy is 16 complex wide with 128-byte swizzling (its
// rows: y then the plane, or the slab then z), so row and column accesses
// stay free of bank conflicts.  Block: a control warpgroup (producer,
// publisher) that lowers its registers with setmaxnreg, and two compute
// warpgroups of 128 threads that take the registers of every 64-point DFT;
// a ring of three tiles.  Tiles go back to the producer as soon as their
// compute group is done; the publisher learns of finished items through an
// mbarrier ring and publishes planes in order.  Liveness and bounded waits
// as in rowfft.cuh.
#pragma once

#include "rowfft.cuh"

namespace fft3d {
namespace rowk2 {

using mb::mbar_arrive;
using mb::mbar_arrive_tx;
using mb::mbar_init;
using mb::mbar_wait_bounded;
using mb::saddr;
using mb::warp_wait;
using rowk::bcast;
using rowk::Desc;
using rowk::spin_geq;
using rowk::policy_evict_first;
using rowk::policy_evict_last;
using rowk::tma_box_hint;

template <int N>
struct Cfg {
  static_assert(N == 64, "two-plane kernel covers 64");
  static constexpr int SEG = 16;                // complex per 128-byte row segment
  static constexpr int NSEG = N / SEG;          // tensor boxes per item
  static constexpr int REGION = 2 * N * 128;    // bytes of one box (two planes)
  static constexpr int TILE = NSEG * REGION;    // bytes of one item, 64 KB
  static constexpr int NTILE = 3;
  static constexpr int GT = 2 * N;              // threads per compute group
  static constexpr int GW = GT / 32;
  static constexpr int GROUPS = 2;
  static constexpr int T = 32 * (4 + GROUPS * GW);  // control warpgroup + compute
  // registers per thread at launch (three warps per SM sub-partition), then
  // moved by setmaxnreg from the control warpgroup to the compute ones: per
  // sub-partition 48 + 2 * 224 <= 3 * 168, in total 4 * 32 * 48 + 8 * 32 *
  // 224 <= 12 * 32 * 168
  static constexpr int REG_CTRL = 48, REG_COMP = 224;
  static constexpr int ITEMS = N / 2;           // items per phase of a grid
  static constexpr int SCHED = 8192;
  static constexpr int DQ = 16;                 // finished items queued for the publisher
  static constexpr int NFULL = NTILE * GROUPS;  // full barriers, one per (group, tile)
  static constexpr size_t smem = 1024 + (size_t)NTILE * TILE +
                                 (NFULL + NTILE + GROUPS + DQ) * sizeof(unsigned long long) +
                                 NTILE * sizeof(int4) + (DQ + 1) * sizeof(int) +
                                 SCHED * sizeof(unsigned short);
};

// Byte offset of complex (box row R, column c) in a tile; R = 64 j + y for
// plane j of the pair, R = 2 z + j for slab j.
template <int N>
__device__ __forceinline__ uint32_t boff(int R, int c) {
  return (uint32_t)((c >> 4) * Cfg<N>::REGION + R * 128 + ((((c & 15) >> 1) ^ (R & 7)) << 4) +
                    ((c & 1) << 3));
}

// Producer warp: tickets (two at a time, two pairs ahead; each ticket one
// item) in order into tiles k % NTILE; lanes 0 and 1 resolve the pair after
// the current one (schedule lookup, probe of a slab pair's dependencies);
// lanes 0 .. NSEG-1 issue one tensor box each.  Every copy is marked
// evict-first in L2 (each item is read once) and the planes' outputs
// evict-last, so the intermediate stays in L2 until its slabs read it.
template <int N>
__device__ __forceinline__ void producer(const FusedArgs& a, const CUtensorMap* tin,
                                         const CUtensorMap* tout, uint32_t tiles,
                                         unsigned long long* full, unsigned long long* empty,
                                         unsigned long long* done, int* pubq,
                                         volatile int* pub_done, Desc* desc,
                                         const unsigned short* sched) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, DQ = K::DQ, IT = K::ITEMS;
  const int lane = threadIdx.x & 31;
  const bool local = a.nblocks <= K::SCHED;
  auto block_of = [&](int b, int& grid, int& phase) {
    if (local) {
      grid = sched[b] >> 1;
      phase = sched[b] & 1;
    } else {
      const SchedBlock blk = a.blocks[b];
      grid = blk.grid;
      phase = blk.phase;
    }
  };
  auto take2 = [&]() -> int { return (int)atomicAdd(a.work, 2u); };
  int ahead = 0;
  int ct = a.total_items, cg = 0, cph = 0, crd = 1;
  int nt = a.total_items, ng = 0, nph = 0, nrd = 1;
  int ready_grid = -1;
  auto resolve = [&](int base, int& t, int& grid, int& phase, int& rd) {
    t = base + lane;
    grid = 0;
    phase = 0;
    rd = 1;
    if (lane < 2 && t < a.total_items) {
      block_of(t / IT, grid, phase);
      if (phase == 1 && grid != ready_grid) {
        rd = ld_acquire(a.work + 1 + grid) >= (unsigned)IT;
        if (rd) ready_grid = grid;
      }
    }
  };
  {
    int b0 = 0, b1 = 0;
    if (lane == 0) {  // same-address atomics of one thread: b0 < b1 < ahead
      b0 = take2();
      b1 = take2();
      ahead = take2();
    }
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    b1 = __shfl_sync(0xffffffffu, b1, 0);
    resolve(b0, ct, cg, cph, crd);
    resolve(b1, nt, ng, nph, nrd);
  }
  unsigned live = 0;
  const unsigned long long once = policy_evict_first();
  int k = 0;
  for (;; ++k) {
    const int s = k % NT;
    if (k > 0 && (k & 1) == 0) {
      ct = nt, cg = ng, cph = nph, crd = nrd;
      int bn = 0;
      if (lane == 0) {
        bn = ahead;
        ahead = take2();
      }
      bn = __shfl_sync(0xffffffffu, bn, 0);
      resolve(bn, nt, ng, nph, nrd);
    }
    const int src = k & 1;
    const int t = __shfl_sync(0xffffffffu, ct, src);
    Desc d{t, __shfl_sync(0xffffffffu, cg, src), __shfl_sync(0xffffffffu, cph, src), t % IT};
    const int rd = __shfl_sync(0xffffffffu, crd, src);
    int ok = t < a.total_items;
    if (ok && !rd && lane == 0)
      ok = bounded_wait_geq(a.work + 1 + d.grid, (unsigned)IT, a.status, a.timeout_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();  // lane 0's (or 1's) acquire before the copies of every lane
    if (!ok) {
      if (lane == 0) {
        for (int j = 0; j < K::GROUPS; ++j) {
          const int kk = k + j, sj = kk % NT;
          if (kk >= NT &&
              !mbar_wait_bounded(&empty[sj], (kk / NT - 1) & 1, a.status, a.timeout_ns))
            break;
          desc[sj] = Desc{-1, 0, 0, 0};
          mbar_arrive(&full[rowk::full_idx<NT, K::GROUPS>(kk)]);
          live &= ~(1u << sj);
        }
        if (spin_geq(pub_done, k - DQ + 1, a)) {
          pubq[k % DQ] = -2;
          for (int j = 0; j < K::GW; ++j) mbar_arrive(&done[k % DQ]);
        }
      }
      live = __shfl_sync(0xffffffffu, live, 0);
      break;
    }
    int fr = 1;
    if (lane == 0) {
      if (k >= NT) fr = mbar_wait_bounded(&empty[s], (k / NT - 1) & 1, a.status, a.timeout_ns);
      if (fr) fr = spin_geq(pub_done, k - DQ + 1, a);
    }
    if (!__shfl_sync(0xffffffffu, fr, 0)) break;
    live &= ~(1u << s);
    unsigned long long* fb = &full[rowk::full_idx<NT, K::GROUPS>(k)];
    if (lane == 0) {
      desc[s] = d;
      pubq[k % DQ] = d.phase == 0 ? d.grid : -1;
      mbar_arrive_tx(fb, (unsigned)K::TILE);
    }
    __syncwarp();
    if (lane < K::NSEG) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (d.phase == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
      const uint32_t dst = tiles + (uint32_t)(s * K::TILE + lane * K::REGION);
      if (d.phase == 0)  // planes 2 idx, 2 idx + 1: box {16 x, all y, 2 z}
        tma_box_hint(dst, tin, 2 * K::SEG * lane, 0, d.grid * N + 2 * d.idx, fb, once);
      else  // slabs 2 idx, 2 idx + 1: box {16 x, 2 y, all z}
        tma_box_hint(dst, tout, 2 * K::SEG * lane, 2 * d.idx, d.grid * N, fb, once);
    }
    live |= 1u << s;
  }
  if (lane == 0)
    for (int j = 1; j <= NT; ++j) {
      const int kk = k - j;
      if (kk >= 0 && (live & (1u << (kk % NT))))
        mbar_wait_bounded(&full[rowk::full_idx<NT, K::GROUPS>(kk)],
                          rowk::full_par<NT, K::GROUPS>(kk), a.status, a.timeout_ns);
    }
}

template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    rowfft2_fft3d_kernel(const FusedArgs a, const __grid_constant__ CUtensorMap tin,
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
  const int w = threadIdx.x >> 5;
  if (a.nblocks <= K::SCHED)
    for (int b = threadIdx.x; b < a.nblocks; b += K::T)
      sched[b] = (unsigned short)(a.blocks[b].grid * 2 + a.blocks[b].phase);
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

  // compute group g (warpgroup g + 1), thread gt of 128: pair member j
  const int g = (w - 4) / K::GW, gt = threadIdx.x - 128 - g * K::GT, lane = threadIdx.x & 31;
  const int j = gt >> 6, u = gt & (N - 1);
  unsigned pairs = 0;  // plane-pair items of this group (parity of its barrier)
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!warp_wait(&full[rowk::full_idx<NT, K::GROUPS>(k)], rowk::full_par<NT, K::GROUPS>(k), a))
      break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    unsigned char* t = base + (size_t)s * K::TILE;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2 v[N];
    if (d.phase == 0) {
      // x: row y = u of plane j, 16-byte chunks
      const int R = 64 * j + u;
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const float4 q = *reinterpret_cast<const float4*>(t + boff<N>(R, 2 * i));
        v[2 * i] = make_float2(q.x, q.y);
        v[2 * i + 1] = make_float2(q.z, q.w);
      }
      DFT<N, DIR>::run(v);
#pragma unroll
      for (int i = 0; i < N / 2; ++i)
        *reinterpret_cast<float4*>(t + boff<N>(R, 2 * i)) =
            make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
      __syncwarp();
      if (lane == 0) mbar_arrive(&tr[g]);
      if (!warp_wait(&tr[g], pairs & 1, a)) break;
      ++pairs;
      // y: column x = u of plane j, output rows straight to global memory
#pragma unroll
      for (int r = 0; r < N; ++r) v[r] = *reinterpret_cast<const float2*>(t + boff<N>(64 * j + r, u));
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // the tile is read: back to the producer
      DFT<N, DIR>::run(v);
      float2* dst = gout + (long long)(2 * d.idx + j) * NN + u;
      const unsigned long long keep = policy_evict_last();  // until its slabs read it
#pragma unroll
      for (int k1 = 0; k1 < N; ++k1)
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(dst + (long long)k1 * N),
                     "f"(v[k1].x), "f"(v[k1].y), "l"(keep));
    } else {
      // z: column x = u of slab y = 2 idx + j
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = *reinterpret_cast<const float2*>(t + boff<N>(2 * z + j, u));
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // the tile is read: back to the producer
      DFT<N, DIR>::run(v);
      float2* dst = gout + (long long)(2 * d.idx + j) * N + u;
#pragma unroll
      for (int k1 = 0; k1 < N; ++k1) {
        float2 o = v[k1];
        if (a.do_scale) o = cscale(o, a.scale);
        st_stream(dst + k1 * NN, o);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[k % K::DQ]);  // the stores are done, for the publisher
  }
}

// Uniform batches only (packed buffers, grids in plan order).
template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off) return cudaErrorInvalidValue;
  CUtensorMap tin, tout;
  if (!rowk::encode_map(&tin, a.in, N, a.ngrids, N, 2) ||
      !rowk::encode_map(&tout, a.out, N, a.ngrids, 2, N))
    return cudaErrorInvalidValue;
  rowfft2_fft3d_kernel<N, DIR><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, tin, tout);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&rowfft2_fft3d_kernel<N, DIR>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.twiddle_entries = N;  // (the codelets need no table; one is uploaded anyway)
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;  // the tiles and up to four tickets held ahead
  k.phase_items = Cfg<N>::ITEMS;
  return k;
}

}  // namespace rowk2
}  // namespace fft3d
