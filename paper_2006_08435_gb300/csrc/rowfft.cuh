// Thread-per-pencil persistent 3D FFT kernel for 64^3 grids, fed by tensor
// TMA.
//
// Same plane and slab items and the same ticket schedule as the persistent
// kernel; what changes is how little shared-memory traffic an item costs.
// Each 1D FFT of 64 points runs entirely in one thread's registers (a
// radix-8 x 8 codelet), so the only shared-memory passes are the ones the
// data layout forces:
//
//   plane item: TMA writes the plane; thread t reads row t, transforms it
//     along x and writes it back in place; after a barrier of its group,
//     thread t reads column t, transforms it along y and stores it to
//     global memory straight from registers (rows of the output plane).
//   slab item: TMA writes the slab (row z = the 64 points of that z);
//     thread t reads column x = t, transforms it along z and stores it.
//
// That is 4 passes over the tile for a plane and 2 for a slab.  An item is
// loaded by four 2D tensor copies (cp.async.bulk.tensor, 16 x 64 complex
// boxes) with 128-byte swizzling: a 128-byte row segment holds 16 complex
// and its 16-byte chunks are XORed with the row index mod 8, so that both
// the row reads (16-byte accesses, eight rows per phase) and the column reads
// (8-byte accesses, sixteen columns of one row per phase) are free of bank
// conflicts.
//
// Block: three compute groups of 64 threads (each group one item at a time,
// items k = g, g + 3, ...; tile k % 6, so each tile always serves the same
// group), one producer warp (tickets, slab dependencies, tensor copies into
// a ring of six tiles) and one publisher warp (publishes
// finished planes; tiles go back to the producer straight from the compute
// groups).  One block per SM.  Liveness and bounded waits
// as in the double-buffered kernel: a block's started items finish without
// the producer, so its waits for slab dependencies are waits on smaller
// tickets only.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "mbar.cuh"

namespace fft3d {
namespace rowk {

using mb::mbar_arrive;
using mb::mbar_arrive_tx;
using mb::mbar_init;
using mb::mbar_wait_bounded;
using mb::saddr;
using mb::warp_wait;

template <int N>
struct Cfg {
  static_assert(N == 64, "thread-per-pencil kernel covers 64");
  static constexpr int SEG = 16;                   // complex per 128-byte row segment
  static constexpr int NSEG = N / SEG;             // tensor boxes per item
  static constexpr int REGION = N * 128;           // bytes of one box in shared memory
  static constexpr int TILE = NSEG * REGION;       // bytes of one item
  static constexpr int NTILE = 6;
  static constexpr int SCHED = 8192;               // schedule blocks kept in shared memory
  static constexpr int DQ = 16;                    // finished items queued for the publisher
  static constexpr int GROUPS = 3;                 // compute groups of N threads
  static constexpr int GW = N / 32;                // warps per group
  static constexpr int NCW = GROUPS * GW;          // compute warps
  static constexpr int T = 32 * (NCW + 2);         // plus producer and publisher
  static constexpr size_t smem = 1024 + (size_t)NTILE * TILE +
                                 (2 * NTILE + GROUPS + DQ) * sizeof(unsigned long long) +
                                 NTILE * sizeof(int4) + (DQ + 1) * sizeof(int) +
                                 SCHED * sizeof(unsigned short);
};

// Byte offset of complex (row r, column c) in a tile (128-byte swizzle).
template <int N>
__device__ __forceinline__ uint32_t eoff(int r, int c) {
  return (uint32_t)((c >> 4) * Cfg<N>::REGION + r * 128 + ((((c & 15) >> 1) ^ (r & 7)) << 4) +
                    ((c & 1) << 3));
}

// Full barriers of a ring of NT tiles that G compute groups take in turn
// (item k: tile k % NT, group k % G; NT and G coprime).  One barrier per
// (group, tile): the consecutive phases of each are the uses by one group.
// With one barrier per tile the uses alternate between the groups, and a
// group that reaches its next use of a tile while the other group's load
// into it is still pending would match its own previous phase (same parity)
// and take a stale tile.
template <int NT, int G>
__device__ __forceinline__ int full_idx(int k) {
  static_assert(G == 2 && NT % 2 == 1, "coprime ring and group counts");
  return (k % G) * NT + k % NT;
}
template <int NT, int G>
__device__ __forceinline__ unsigned full_par(int k) {
  return (unsigned)(k / (NT * G)) & 1u;
}

// L2 eviction policies (fraction 1.0 of the accessed lines).
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// As tma_box, with an L2 eviction policy for the lines it reads.
__device__ __forceinline__ void tma_box_hint(uint32_t dst, const CUtensorMap* map, int x, int y,
                                             int z, unsigned long long* bar,
                                             unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(bar)),
      "l"(policy)
      : "memory");
}

// 2D box (16 complex wide) of a 3D tensor map into shared memory.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
      : "memory");
}

struct Desc {
  int item, grid, phase, idx;
};

// Tensor maps passed with a launch (kernel parameter space): NM = 1 for a
// packed uniform batch, kMixMaps for the grids of a mixed-edge unit.
template <int NM>
struct TensorMaps {
  CUtensorMap in[NM];
  CUtensorMap out[NM];
};

__device__ __forceinline__ Desc bcast(Desc d) {
  d.item = __shfl_sync(0xffffffffu, d.item, 0);
  d.grid = __shfl_sync(0xffffffffu, d.grid, 0);
  d.phase = __shfl_sync(0xffffffffu, d.phase, 0);
  d.idx = __shfl_sync(0xffffffffu, d.idx, 0);
  return d;
}

// Spin (sleeping) until *p >= target, bounded in time like the other waits.
__device__ __forceinline__ int spin_geq(const volatile int* p, int target, const FusedArgs& a) {
  if (*p >= target) return 1;
  const unsigned long long t0 = global_timer_ns();
  for (int it = 0; it < (1 << 22); ++it) {
    __nanosleep(64);
    if (*p >= target) return 1;
    if ((it & 63) == 0 && ((long long)(global_timer_ns() - t0) > a.timeout_ns ||
                           *(volatile unsigned*)a.status != kStatusOk))
      break;
  }
  atomicCAS(a.status, kStatusOk, kStatusTimeout);
  return 0;
}

// Producer warp: tickets in order into tiles k % NTILE.  Lane 0 takes and
// resolves the tickets; lanes 0 .. NSEG-1 issue one tensor box each.
// Tensors are viewed as [N * batch][N][2N] floats (z of all grids, y, x
// interleaved re/im); planes come from `in`, slabs from `out`.  Schedule
// block b (tickets b*N .. b*N + N - 1) is read from `sched` (grid * 2 +
// phase) when the schedule fits there, else from global memory.  A failure
// elsewhere is seen at the next dependency wait; until then the producer
// keeps taking tickets without reading the status word.  The next item is
// resolved (and a slab's planes waited for) before its tile is free, so
// those round trips overlap the tile's previous item.
template <int N>
__device__ __forceinline__ void producer(const FusedArgs& a, const CUtensorMap* tin,
                                         const CUtensorMap* tout, uint32_t tiles,
                                         unsigned long long* full, unsigned long long* empty,
                                         unsigned long long* done, int* pubq,
                                         volatile int* pub_done, Desc* desc,
                                         const unsigned short* sched) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, DQ = K::DQ;
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
  // L2 hint for a ticket this warp will load soon: a plane item's input
  // (one contiguous plane) is fetched from HBM now, so that its tensor copies
  // later read L2.
  auto prefetch_item = [&](int t) {
    if (t >= a.total_items) return;
    int grid, phase;
    block_of(t / N, grid, phase);
    if (phase != 0) return;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, grid, N, gin, gout);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                     gin + (long long)(t % N) * N * N),
                 "r"((unsigned)(N * N * sizeof(float2)))
                 : "memory");
  };
  // Tickets two at a time (t even; N is even, so a pair never spans two
  // schedule blocks), requested two pairs ahead.  When the tickets of pair
  // p are about to be issued, those of pair p + 1 are resolved by lanes 0
  // and 1 together: schedule lookup, an L2 prefetch of a plane's input, and
  // a non-blocking probe of a slab's dependencies, so the two round trips
  // overlap each other and the copies of pair p.
  auto take2 = [&]() -> int { return (int)atomicAdd(a.work, 2u); };
  int ahead = 0;  // lane 0: base of the pair after the next
  // resolved tickets, lanes 0 and 1 (ticket base + lane): current pair, next pair
  int ct = a.total_items, cg = 0, cph = 0, crd = 1;
  int nt = a.total_items, ng = 0, nph = 0, nrd = 1;
  int ready_grid = -1;  // lanes 0, 1: a grid whose planes this lane saw all published
  auto resolve = [&](int base, int& t, int& grid, int& phase, int& rd) {
    t = base + lane;
    grid = 0;
    phase = 0;
    rd = 1;
    if (lane < 2 && t < a.total_items) {
      block_of(t / N, grid, phase);
      if (phase == 0) {
        prefetch_item(t);
      } else if (grid != ready_grid) {
        rd = ld_acquire(a.work + 1 + grid) >= (unsigned)N;
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
  unsigned live = 0;    // tiles whose copies were issued (bit s)
  int k = 0;
  for (;; ++k) {
    const int s = k % NT;
    if (k > 0 && (k & 1) == 0) {  // next pair becomes current; resolve the one after
      ct = nt, cg = ng, cph = nph, crd = nrd;
      int bn = 0;
      if (lane == 0) {
        bn = ahead;
        ahead = take2();
      }
      bn = __shfl_sync(0xffffffffu, bn, 0);
      resolve(bn, nt, ng, nph, nrd);
    }
    const int src = k & 1;  // lane holding this item's ticket
    const int t = __shfl_sync(0xffffffffu, ct, src);
    Desc d{t, __shfl_sync(0xffffffffu, cg, src), __shfl_sync(0xffffffffu, cph, src), t % N};
    const int rd = __shfl_sync(0xffffffffu, crd, src);
    int ok = t < a.total_items;
    if (ok && !rd && lane == 0)  // a slab whose planes were not all published yet
      ok = bounded_wait_geq(a.work + 1 + d.grid, (unsigned)N, a.status, a.timeout_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();  // lane 0's (or 1's) acquire before the copies of every lane
    if (!ok) {
      if (lane == 0) {
        // a stop for each compute group: items k .. k + GROUPS - 1, each tile
        // once its group is done with its earlier item
        for (int j = 0; j < K::GROUPS; ++j) {
          const int kk = k + j, sj = kk % NT;
          if (kk >= NT &&
              !mbar_wait_bounded(&empty[sj], (kk / NT - 1) & 1, a.status, a.timeout_ns))
            break;
          desc[sj] = Desc{-1, 0, 0, 0};
          mbar_arrive(&full[sj]);
          live &= ~(1u << sj);
        }
        // and one for the publisher, after item k - 1
        if (spin_geq(pub_done, k - DQ + 1, a)) {
          pubq[k % DQ] = -2;
          for (int j = 0; j < K::GW; ++j) mbar_arrive(&done[k % DQ]);
        }
      }
      live = __shfl_sync(0xffffffffu, live, 0);
      break;
    }
    // the tile: its group is done with item k - NT; the publisher's slot of
    // item k: item k - DQ published (rarely waited for)
    int fr = 1;
    if (lane == 0) {
      if (k >= NT) fr = mbar_wait_bounded(&empty[s], (k / NT - 1) & 1, a.status, a.timeout_ns);
      if (fr) fr = spin_geq(pub_done, k - DQ + 1, a);
    }
    if (!__shfl_sync(0xffffffffu, fr, 0)) break;
    live &= ~(1u << s);
    if (lane == 0) {
      desc[s] = d;
      pubq[k % DQ] = d.phase == 0 ? d.grid : -1;  // read by the publisher after item k
      mbar_arrive_tx(&full[s], (unsigned)K::TILE);
    }
    __syncwarp();
    if (lane < K::NSEG) {
      // the tile was last written by the compute threads' plain stores, a
      // slab's rows by other blocks' plain stores (seen through lane 0's
      // acquire)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (d.phase == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
      const uint32_t dst = tiles + (uint32_t)(s * K::TILE + lane * K::REGION);
      if (d.phase == 0)  // plane z = idx: box {16 x, all y} at z
        tma_box(dst, tin, 2 * K::SEG * lane, 0, d.grid * N + d.idx, &full[s]);
      else  // slab y = idx: box {16 x, all z} at y
        tma_box(dst, tout, 2 * K::SEG * lane, d.idx, d.grid * N, &full[s]);
    }
    live |= 1u << s;
  }
  // no copy may still be writing a tile when the block exits (only after a
  // failure can one be left unconsumed)
  if (lane == 0)
    for (int j = 1; j <= NT; ++j) {
      const int kk = k - j;
      if (kk >= 0 && (live & (1u << (kk % NT))))
        mbar_wait_bounded(&full[kk % NT], (kk / NT) & 1, a.status, a.timeout_ns);
    }
}

// Publisher warp (lane 0): finished items in order; a plane is published to
// the other blocks (the GPU-scope release waits for the compute group's
// stores, so it is kept off the compute and producer warps).  Item k's
// completion arrives on done[k % DQ] (both warps of its group); its grid was
// queued by the producer.  Tiles are handed back by the compute groups
// directly, so publishing never delays a refill.
template <int N>
__device__ __forceinline__ void publisher(const FusedArgs& a, unsigned long long* done,
                                          const int* pubq, volatile int* pub_done) {
  constexpr int DQ = Cfg<N>::DQ;
  if ((threadIdx.x & 31) != 0) return;
  for (int k = 0;; ++k) {
    if (!mbar_wait_bounded(&done[k % DQ], (k / DQ) & 1, a.status, a.timeout_ns)) return;
    const int grid = pubq[k % DQ];
    if (grid == -2) return;
    if (grid >= 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      atomicAdd(a.work + 1 + grid, 1u);
    }
    __threadfence_block();  // the slot is read before it is handed back
    *pub_done = k + 1;
  }
}

template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    rowfft_fft3d_kernel(const FusedArgs a, const __grid_constant__ CUtensorMap tin,
                        const __grid_constant__ CUtensorMap tout) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE;
  constexpr long long NN = (long long)N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // tiles 1024-byte aligned (the swizzle pattern follows address bits 7..9)
  unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const uint32_t tiles = saddr(base);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(base + (size_t)NT * K::TILE);
  unsigned long long* empty = full + NT;
  unsigned long long* tr = empty + NT;  // per group: rows done before columns
  unsigned long long* done = tr + K::GROUPS;  // items finished, for the publisher
  Desc* desc = reinterpret_cast<Desc*>(done + K::DQ);
  int* pubq = reinterpret_cast<int*>(desc + NT);
  volatile int* pub_done = pubq + K::DQ;
  unsigned short* sched = reinterpret_cast<unsigned short*>(pubq + K::DQ + 1);
  const int w = threadIdx.x >> 5;
  if (a.nblocks <= K::SCHED)
    for (int b = threadIdx.x; b < a.nblocks; b += K::T)
      sched[b] = (unsigned short)(a.blocks[b].grid * 2 + a.blocks[b].phase);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NT; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], K::GW);
    }
    for (int g = 0; g < K::GROUPS; ++g) mbar_init(&tr[g], K::GW);
    for (int q = 0; q < K::DQ; ++q) mbar_init(&done[q], K::GW);
    *pub_done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (w == K::NCW) {
    producer<N>(a, &tin, &tout, tiles, full, empty, done, pubq, pub_done, desc, sched);
    return;
  }
  if (w == K::NCW + 1) {
    publisher<N>(a, done, pubq, pub_done);
    return;
  }

  // compute group g, thread gt of N
  const int g = w / K::GW, gt = threadIdx.x - g * N, lane = threadIdx.x & 31;
  unsigned planes = 0;  // plane items of this group (parity of its barrier)
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!warp_wait(&full[s], (k / NT) & 1, a)) break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    unsigned char* t = base + (size_t)s * K::TILE;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2 v[N];
    if (d.phase == 0) {
      // x: row y = gt, 16-byte chunks
#pragma unroll
      for (int j = 0; j < N / 2; ++j) {
        const float4 q = *reinterpret_cast<const float4*>(t + eoff<N>(gt, 2 * j));
        v[2 * j] = make_float2(q.x, q.y);
        v[2 * j + 1] = make_float2(q.z, q.w);
      }
      DFT<N, DIR>::run(v);
#pragma unroll
      for (int j = 0; j < N / 2; ++j)
        *reinterpret_cast<float4*>(t + eoff<N>(gt, 2 * j)) =
            make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
      __syncwarp();
      if (lane == 0) mbar_arrive(&tr[g]);
      if (!warp_wait(&tr[g], planes & 1, a)) break;
      ++planes;
      // y: column x = gt, output rows straight to global memory
#pragma unroll
      for (int r = 0; r < N; ++r) v[r] = *reinterpret_cast<const float2*>(t + eoff<N>(r, gt));
      DFT<N, DIR>::run(v);
      float2* dst = gout + (long long)d.idx * NN + gt;
#pragma unroll
      for (int k1 = 0; k1 < N; ++k1) dst[(long long)k1 * N] = v[k1];
    } else {
      // z: column x = gt of slab y = idx
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = *reinterpret_cast<const float2*>(t + eoff<N>(z, gt));
      DFT<N, DIR>::run(v);
      float2* dst = gout + (long long)d.idx * N + gt;
#pragma unroll
      for (int k1 = 0; k1 < N; ++k1) {
        float2 o = v[k1];
        if (a.do_scale) o = cscale(o, a.scale);
        st_stream(dst + k1 * NN, o);
      }
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[s]);              // the tile is free
      mbar_arrive(&done[k % K::DQ]);       // and the stores done, for the publisher
    }
  }
}

// cuTensorMapEncodeTiled from the driver, looked up once.
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// [N * batch][N][2N] floats, box {32 floats (16 complex), by, bz}, 128-byte
// swizzle; along y every `ystep`-th row is taken (by = rows * ystep).
inline bool encode_map(CUtensorMap* m, const void* base, int n, int batch, unsigned by,
                       unsigned bz, unsigned ystep = 1) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * n, (cuuint64_t)n, (cuuint64_t)n * batch};
  const cuuint64_t strides[2] = {(cuuint64_t)n * 8, (cuuint64_t)n * n * 8};
  const cuuint32_t box[3] = {32, by, bz};
  const cuuint32_t estr[3] = {1, ystep, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Uniform batches only (packed buffers, grids in plan order).
template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off) return cudaErrorInvalidValue;
  CUtensorMap tin, tout;
  if (!encode_map(&tin, a.in, N, a.ngrids, N, 1) || !encode_map(&tout, a.out, N, a.ngrids, 1, N))
    return cudaErrorInvalidValue;
  rowfft_fft3d_kernel<N, DIR><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, tin, tout);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&rowfft_fft3d_kernel<N, DIR>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.twiddle_entries = N;  // (the codelets need no table; one is uploaded anyway)
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;  // the tiles and up to four tickets held ahead
  return k;
}

}  // namespace rowk
}  // namespace fft3d
