// Warp-specialised, TMA-fed persistent 3D FFT kernel for 64^3 and 128^3
// grids.
//
// Same two kinds of work items and the same ticket schedule as the plain
// persistent kernel (plane item: x and y transforms of one z plane; slab
// item: z transform of one y slab; slab items of a grid wait for all its
// plane items), but the loads no longer sit on the critical path:
//
//   * one producer warp takes tickets and streams each item's N rows of N
//     points into a ring of 64-row shared-memory slots with 1D bulk copies
//     (cp.async.bulk, the TMA engine) that complete on an mbarrier ("full");
//     a plane item's rows are contiguous in HBM, a slab item's rows (one per
//     z) are N*N points apart -- the strided pencils of the paper's 3D
//     transpose, fetched as whole rows.  An item takes N/64 slots; the ring
//     holds 3 slots at N = 128 (1.5 items) and 6 at N = 64 (6 items);
//   * sixteen consumer warps transform the item in place in its slots and
//     release them through a second mbarrier ("empty").  The warps run
//     independently: in the x step each owns N/16 rows; in the y and z steps
//     a group of 256/N warps owns 16 columns.  The only block-wide
//     synchronisation is one mbarrier between the x and y steps of a plane
//     item (the transpose); the warps of a column group meet on their own
//     mbarrier between the first and second y (or z) step;
//   * one signaller warp publishes each finished plane item to the other
//     blocks (the GPU-scope release waits for the stores to land, so it is
//     kept off the consumer warps).
//
// Staged rows use a pitch of N + 8 complex (16-byte aligned for the bulk
// copies, and 8 banks apart so that two rows of a half-warp never collide).
// Between the two x steps each row is kept transposed as [n1][k2 ^ n1] so
// that both steps access shared memory without bank conflicts.
//
// Every wait (ticket dependency, full, empty, block, group and signaller
// mbarriers) is bounded in time; on expiry the status word records a
// timeout and the warp leaves its loop, so the waits of the other warps run
// out in turn.
#pragma once

#include "persistent.cuh"

namespace fft3d {
namespace piped {

constexpr int NC = 512;      // consumer threads
constexpr int NT = NC + 64;  // plus one producer and one signaller warp
constexpr int CROWS = 64;    // rows per slot

template <int N>
struct Cfg {
  static constexpr int L1 = split_l1(N), L2 = split_l2(N);
  static_assert(L1 == 8 && (N == 64 || N == 128), "pipelined kernel covers 64 and 128");
  static constexpr int C = N / CROWS;            // slots per item
  static constexpr int PITCH = N + 8;            // complex per staged row
  static constexpr int SLOT = CROWS * PITCH;     // complex per slot
  static constexpr int NSLOT = N == 128 ? 3 : 6;
  static constexpr int RPW = N / 16;             // x rows per consumer warp
  static constexpr int G = N / 16;               // 16-column groups
  static constexpr int WPG = 16 / G;             // warps per column group
  static constexpr int N1W = L1 / WPG;           // n1 values per warp (first step)
  static constexpr int K2W = L2 / WPG;           // k2 values per warp (second step)
  static constexpr unsigned ROW_BYTES = N * sizeof(float2);
  static constexpr unsigned CHUNK_BYTES = CROWS * ROW_BYTES;
};

struct Desc {
  int item;   // ticket, or -1 = stop
  int grid;
  int phase;  // 0 plane, 1 slab
  int idx;    // z of the plane or y of the slab
};

template <int N>
constexpr size_t smem_bytes() {
  using K = Cfg<N>;
  return sizeof(float2) * (N + (size_t)K::NSLOT * K::SLOT) +
         (2 * K::NSLOT + 1 + K::G + 4) * sizeof(unsigned long long) +
         (K::NSLOT + 2) * sizeof(Desc);
}

// ---------------------------------------------------------- mbarrier, TMA
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ unsigned mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok;
}
// As above, but the thread may sleep in hardware (up to ~hint_ns) until the
// phase completes instead of returning at once: waiting warps do not take
// issue slots from working ones.
__device__ __forceinline__ unsigned mbar_try_wait_sleep(unsigned long long* b, unsigned parity,
                                                        unsigned hint_ns) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; "
      "selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok;
}
// Wait for the phase with the given parity to complete: at most timeout_ns
// of %globaltimer and 2^20 sleeping polls.  0 on timeout (status set) or
// when another block already reported a failure.
__device__ __forceinline__ int mbar_wait_bounded(unsigned long long* b, unsigned parity,
                                                 unsigned* status, long long timeout_ns) {
  if (mbar_try_wait(b, parity)) return 1;
  const unsigned long long t0 = global_timer_ns();
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try_wait_sleep(b, parity, 100000u)) return 1;
    if (*(volatile unsigned*)status != kStatusOk) return 0;
    if ((long long)(global_timer_ns() - t0) > timeout_ns) break;
  }
  atomicCAS(status, kStatusOk, kStatusTimeout);
  return 0;
}
// Warp-level bounded wait: every lane waits (sleeping in hardware) and the
// warp proceeds only if all lanes saw the phase complete, so the warp stays
// converged and takes one decision.
__device__ __forceinline__ int warp_wait(unsigned long long* b, unsigned parity,
                                         const FusedArgs& a) {
  const int ok = mbar_wait_bounded(b, parity, a.status, a.timeout_ns);
  return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}

// ------------------------------------------------------------- producer
template <int N>
__device__ __forceinline__ void producer(const FusedArgs& a, float2* slots,
                                         unsigned long long* full, unsigned long long* empty,
                                         Desc* desc) {
  using K = Cfg<N>;
  const int lane = threadIdx.x & 31;
  unsigned seq = 0;  // chunk sequence number, slot = seq % NSLOT
  for (;;) {
    int d0 = -1, d1 = 0, d2 = 0, d3 = 0;
    if (lane == 0) {
      int item = -1;
      if (*(volatile unsigned*)a.status == kStatusOk) item = (int)atomicAdd(a.work, 1u);
      if (item >= a.total_items) item = -1;
      if (item >= 0) {
        const SchedBlock blk = a.blocks[find_block(a.blocks, a.nblocks, item)];
        d0 = item;
        d1 = blk.grid;
        d2 = blk.phase;
        d3 = item - blk.start;
        if (blk.phase == 1 &&
            !bounded_wait_geq(a.work + 1 + blk.grid, (unsigned)N, a.status, a.timeout_ns))
          d0 = -1;
      }
    }
    d0 = __shfl_sync(0xffffffffu, d0, 0);
    d1 = __shfl_sync(0xffffffffu, d1, 0);
    d2 = __shfl_sync(0xffffffffu, d2, 0);
    d3 = __shfl_sync(0xffffffffu, d3, 0);
    const float2* gin = nullptr;
    float2* gout = nullptr;
    if (d0 >= 0) grid_ptrs(a, d1, N, gin, gout);
    const int nchunks = d0 < 0 ? 1 : K::C;
    for (int k = 0; k < nchunks; ++k, ++seq) {
      const unsigned s = seq % K::NSLOT;
      int ok = 1;
      if (seq >= (unsigned)K::NSLOT)
        ok = mbar_wait_bounded(&empty[s], ((seq / K::NSLOT) - 1) & 1, a.status, a.timeout_ns);
      if (!__all_sync(0xffffffffu, ok)) return;
      if (lane == 0) {
        desc[s] = Desc{d0, d1, d2, d3};
        if (d0 < 0) {
          mbar_arrive(&full[s]);
        } else {
          // rows written by other blocks' plain stores are read through the
          // async proxy next
          asm volatile("fence.proxy.async.global;" ::: "memory");
          mbar_arrive_tx(&full[s], K::CHUNK_BYTES);
        }
      }
      if (d0 < 0) return;
      __syncwarp();
      float2* slot = slots + (size_t)s * K::SLOT;
      for (int r = lane; r < CROWS; r += 32) {
        const float2* src;
        if (d2 == 0) {
          src = gin + (long long)d3 * N * N + (long long)(k * CROWS + r) * N;
        } else {
          const int n1 = k * (K::L1 / K::C) + r / K::L2, n2 = r % K::L2;
          src = gout + (long long)(n1 + K::L1 * n2) * N * N + (long long)d3 * N;
        }
        bulk_g2s(slot + r * K::PITCH, src, K::ROW_BYTES, &full[s]);
      }
    }
  }
}

// ------------------------------------------------------------- consumers
// Row r of the item (plane row y, or slab row index) in its slots.
template <int N>
__device__ __forceinline__ float2* row_ptr(float2* const* c, int r) {
  return c[r / CROWS] + (r % CROWS) * Cfg<N>::PITCH;
}

// x transform of rows rl0 .. rl0 + N/16 - 1 of one slot, one warp, in place.
template <int N, int DIR>
__device__ __forceinline__ void x_rows(float2* c, int rl0, const float2* tw) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2, P = K::PITCH;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < K::RPW * L1 / 32; ++i) {
    const int n1 = lane & 7, row = rl0 + (lane >> 3) + 4 * i;
    float2* rp = c + row * P;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = rp[n1 + L1 * n2];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) rp[n1 * L2 + (k2 ^ n1)] = v[k2];
  }
  __syncwarp();
  constexpr int RPI = 32 / L2;  // rows per lane iteration
#pragma unroll
  for (int i = 0; i < K::RPW / RPI; ++i) {
    const int k2 = lane % L2, row = rl0 + lane / L2 + RPI * i;
    float2* rp = c + row * P;
    float2 w[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) w[n1] = rp[n1 * L2 + (k2 ^ n1)];
    DFT<L1, DIR>::run(w);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) rp[k2 + L2 * k1] = w[k1];
  }
}

// First y step of the 16 columns of group cg, n1 in the warp's share; the
// plane's rows in slots c[0..C); in place.
template <int N, int DIR>
__device__ __forceinline__ void y_first(float2* const* c, int cg, int q, const float2* tw) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2;
  const int lane = threadIdx.x & 31, col = 16 * cg + (lane & 15);
#pragma unroll
  for (int i = 0; i < K::N1W / 2; ++i) {
    const int n1 = K::N1W * q + (lane >> 4) + 2 * i;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = row_ptr<N>(c, n1 + L1 * n2)[col];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) row_ptr<N>(c, n1 + L1 * k2)[col] = v[k2];
  }
}

// Second y step for the warp's share of k2: a[n1 + 8 k2] is row 8 k2 + n1.
// Result to the plane dst.
template <int N, int DIR>
__device__ __forceinline__ void y_second(float2* const* c, int cg, int q, float2* __restrict__ dst) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2;
  const int lane = threadIdx.x & 31, col = 16 * cg + (lane & 15);
#pragma unroll
  for (int i = 0; i < K::K2W / 2; ++i) {
    const int k2 = K::K2W * q + (lane >> 4) + 2 * i;
    const float2* base = row_ptr<N>(c, L1 * k2) + col;
    float2 w[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) w[n1] = base[n1 * K::PITCH];
    DFT<L1, DIR>::run(w);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) dst[(k2 + L2 * k1) * N + col] = w[k1];
  }
}

// Slab rows: z = n1 + 8 n2 is held at item row n1 * L2 + n2 (slot n1 / (L1/C)).
// First z step for the 16 columns of group cg, n1 in the warp's share.
template <int N, int DIR>
__device__ __forceinline__ void z_first(float2* const* c, int cg, int q, const float2* tw) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2;
  const int lane = threadIdx.x & 31, x = 16 * cg + (lane & 15);
#pragma unroll
  for (int i = 0; i < K::N1W / 2; ++i) {
    const int n1 = K::N1W * q + (lane >> 4) + 2 * i;
    float2* base = row_ptr<N>(c, n1 * L2) + x;
    float2 v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = base[n2 * K::PITCH];
    DFT<L2, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul_tw<DIR>(v[k2], tw[k2 * L1 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) base[k2 * K::PITCH] = v[k2];
  }
}

// Second z step for the warp's share of k2: a[n1 + 8 k2] is at item row
// n1 * L2 + k2.  dst points at (x = 0, y, z = 0) of the grid.
template <int N, int DIR>
__device__ __forceinline__ void z_second(float2* const* c, int cg, int q, float2* dst, float scale,
                                         int do_scale) {
  using K = Cfg<N>;
  constexpr int L1 = K::L1, L2 = K::L2;
  constexpr long long NN = (long long)N * N;
  const int lane = threadIdx.x & 31, x = 16 * cg + (lane & 15);
#pragma unroll
  for (int i = 0; i < K::K2W / 2; ++i) {
    const int k2 = K::K2W * q + (lane >> 4) + 2 * i;
    float2 w[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) w[n1] = row_ptr<N>(c, n1 * L2 + k2)[x];
    DFT<L1, DIR>::run(w);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) {
      float2 o = w[k1];
      if (do_scale) o = cscale(o, scale);
      st_stream(dst + (k2 + L2 * k1) * NN + x, o);
    }
  }
}

// Hands a finished item to the signaller: consumer warp 0 records the item
// (after the signaller has released the entry used two items earlier), and
// every consumer warp arrives once its own stores are issued.
__device__ __forceinline__ int hand_over(const FusedArgs& a, unsigned j, const Desc& d,
                                         unsigned long long* stored, unsigned long long* sigfree,
                                         Desc* sig) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned e = j & 1;
  if (w == 0) {
    if (j >= 2 && !warp_wait(&sigfree[e], ((j >> 1) - 1) & 1, a)) return 0;
    if (lane == 0) sig[e] = d;
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&stored[e]);
  return 1;
}

template <int N, int DIR>
__device__ __forceinline__ void consumer(const FusedArgs& a, const float2* tw, float2* slots,
                                         unsigned long long* full, unsigned long long* empty,
                                         unsigned long long* xdone, unsigned long long* grp,
                                         unsigned long long* stored, unsigned long long* sigfree,
                                         const Desc* desc, Desc* sig) {
  using K = Cfg<N>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cg = w % K::G, q = w / K::G;          // column group, share within it
  const int xs = w / (16 / K::C);                  // slot of this warp's x rows
  const int xr = (w % (16 / K::C)) * K::RPW;       // first x row within it
  unsigned seq = 0, xpar = 0, gpar = 0, j = 0;
  for (;;) {
    const unsigned s0 = seq % K::NSLOT;
    if (!warp_wait(&full[s0], (seq / K::NSLOT) & 1, a)) return;
    const Desc d = desc[s0];
    if (d.item < 0) {
      hand_over(a, j, d, stored, sigfree, sig);  // tells the signaller to stop
      return;
    }
    float2* c[K::C];
#pragma unroll
    for (int k = 0; k < K::C; ++k) c[k] = slots + (size_t)((seq + k) % K::NSLOT) * K::SLOT;
    // this warp's own slot (the first one is already complete)
    if (xs > 0 && !warp_wait(&full[(seq + xs) % K::NSLOT], ((seq + xs) / K::NSLOT) & 1, a)) return;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    if (d.phase == 0) {
      x_rows<N, DIR>(c[xs], xr, tw);
      __syncwarp();
      if (lane == 0) mbar_arrive(xdone);
      if (!warp_wait(xdone, xpar, a)) return;
      xpar ^= 1;
      y_first<N, DIR>(c, cg, q, tw);
      __syncwarp();
      if (lane == 0) mbar_arrive(&grp[cg]);
      if (!warp_wait(&grp[cg], gpar, a)) return;
      gpar ^= 1;
      y_second<N, DIR>(c, cg, q, gout + (long long)d.idx * N * N);
    } else {
      // the slab's first step reads every slot of the item
#pragma unroll
      for (int k = 1; k < K::C; ++k)
        if (k != xs && !warp_wait(&full[(seq + k) % K::NSLOT], ((seq + k) / K::NSLOT) & 1, a))
          return;
      z_first<N, DIR>(c, cg, q, tw);
      __syncwarp();
      if (lane == 0) mbar_arrive(&grp[cg]);
      if (!warp_wait(&grp[cg], gpar, a)) return;
      gpar ^= 1;
      z_second<N, DIR>(c, cg, q, gout + (long long)d.idx * N, a.scale, a.do_scale);
    }
    // the slots are rewritten by the async proxy next
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K::C; ++k) mbar_arrive(&empty[(seq + k) % K::NSLOT]);
    }
    if (!hand_over(a, j, d, stored, sigfree, sig)) return;
    ++j;
    seq += K::C;
  }
}

// Signaller warp: once all consumer warps have issued the stores of an item
// (CTA-scope release/acquire through `stored`), publish a finished plane
// item to the other blocks with one GPU-scope release.
__device__ __forceinline__ void signaller(const FusedArgs& a, unsigned long long* stored,
                                          unsigned long long* sigfree, const Desc* sig) {
  const int lane = threadIdx.x & 31;
  for (unsigned j = 0;; ++j) {
    const unsigned e = j & 1;
    if (!warp_wait(&stored[e], (j >> 1) & 1, a)) return;
    const Desc d = sig[e];
    if (d.item < 0) return;
    if (lane == 0) {
      if (d.phase == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.work + 1 + d.grid)
                     : "memory");
      mbar_arrive(&sigfree[e]);
    }
    __syncwarp();
  }
}

template <int N, int DIR>
__global__ void __launch_bounds__(NT, 1) piped_fft3d_kernel(const FusedArgs a) {
  using K = Cfg<N>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* slots = tw + N;
  unsigned long long* full =
      reinterpret_cast<unsigned long long*>(slots + (size_t)K::NSLOT * K::SLOT);
  unsigned long long* empty = full + K::NSLOT;
  unsigned long long* xdone = empty + K::NSLOT;
  unsigned long long* grp = xdone + 1;
  unsigned long long* stored = grp + K::G;
  unsigned long long* sigfree = stored + 2;
  Desc* desc = reinterpret_cast<Desc*>(sigfree + 2);
  Desc* sig = desc + K::NSLOT;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.twiddles[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < K::NSLOT; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC / 32);
    }
    mbar_init(xdone, NC / 32);
    for (int g = 0; g < K::G; ++g) mbar_init(&grp[g], K::WPG);
    for (int e = 0; e < 2; ++e) {
      mbar_init(&stored[e], NC / 32);
      mbar_init(&sigfree[e], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x >= NC + 32)
    signaller(a, stored, sigfree, sig);
  else if (threadIdx.x >= NC)
    producer<N>(a, slots, full, empty, desc);
  else
    consumer<N, DIR>(a, tw, slots, full, empty, xdone, grp, stored, sigfree, desc, sig);
}

template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  piped_fft3d_kernel<N, DIR><<<grid, NT, smem_bytes<N>(), stream>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&piped_fft3d_kernel<N, DIR>;
  k.threads = NT;
  k.smem = smem_bytes<N>();
  k.twiddle_entries = N;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NSLOT / Cfg<N>::C + 1;
  return k;
}

}  // namespace piped
}  // namespace fft3d
