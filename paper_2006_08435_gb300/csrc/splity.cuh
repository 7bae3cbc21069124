// Persistent 3D FFT kernel for 128^3 grids with the y transform split in
// two, so that every work item is 64 KB and a block can keep three of them in
// shared memory (a whole 128^3 plane, 128 KB, fits only once).
//
// With n = 128 = 2 * 64 and y = n1 + 2 n2 (n1 the parity of the row), the y
// transform of Eq. 1 is
//   Y[k2 + 64 k1] = A0[k2] + (-1)^k1 W_128^k2 A1[k2],
//   A_n1[k2] = sum over n2 of x[n1 + 2 n2] W_64^(n2 k2),
// a 64-point DFT over the rows of one parity, a twiddle, and a radix-2 step.
// The items are
//
//   half-plane (plane z, parity n1): the 64 rows y = n1 + 2 n2 of plane z
//     (one tensor copy with a row step of 2): x transform of each row, then
//     the 64-point y DFT of each column, times W_128^(n1 k2); stored to
//     rows n1 * 64 + k2 of the output plane.
//   slab (k2, x quarter q): rows y = k2 and k2 + 64 of every z, columns
//     32 q .. 32 q + 31: the radix-2 step of y (rows k2 +- W A1 -> k2, k2 +
//     64), then the z transform of each of the 64 columns, in place.
//
// Slabs of a grid wait for all 256 half-planes of that grid, as in the
// persistent kernel.  Every 128-point FFT (x and z) runs in a pair of
// threads: thread p holds the points p + 2 m (m < 64), does a 64-point DFT
// in registers, multiplies by W_128^(p k), and the pair finishes with one
// radix-2 step after exchanging half of their values with warp shuffles;
// the 64-point y DFT runs in one thread.  Tiles are tensor copies with
// 128-byte swizzling, and the lane orders are chosen so that every shared-
// memory access is free of bank conflicts.
//
// Block: two compute groups of 128 threads (items k = g, g + 2, ...), one
// producer warp (tickets, slab dependencies, tensor copies into a ring of
// three tiles; every copy marked evict-first in L2, the intermediate's stores
// evict-last, so the intermediate stays in L2 until its slabs read it) and one signaller warp (frees tiles,
// publishes finished half-planes).  Liveness and bounded waits as in the
// thread-per-pencil 64^3 kernel.
#pragma once

#include "rowfft.cuh"

namespace fft3d {
namespace sy {

using mb::mbar_arrive;
using mb::mbar_arrive_tx;
using mb::mbar_init;
using mb::mbar_wait_bounded;
using mb::saddr;
using mb::warp_wait;
using rowk::bcast;
using rowk::Desc;
using rowk::policy_evict_first;
using rowk::policy_evict_last;
using rowk::tma_box_hint;

template <int N>
struct Cfg {
  static_assert(N == 128, "split-y kernel covers 128");
  static constexpr int H = N / 2;               // points per thread
  static constexpr int TILE = 65536;            // bytes of one item
  static constexpr int NTILE = 3;
  static constexpr int GT = 128;                // threads per compute group
  static constexpr int GW = GT / 32;
  static constexpr int GROUPS = 2;
  static constexpr int NCW = GROUPS * GW;       // compute warps (warpgroups 1, 2)
  static constexpr int T = 32 * (NCW + 4);      // plus warpgroup 0: producer, signaller, 2 idle
  // registers per thread: at launch (T threads fit the register file, three
  // warps per SM sub-partition), then redistributed with setmaxnreg: the
  // control warpgroup gives up most of its share, the compute warpgroups take
  // it (per sub-partition 48 + 2 * 224 <= 3 * 168, and in total
  // 4 * 32 * 48 + 8 * 32 * 224 <= 12 * 32 * 168, the launch total)
  static constexpr int REG_LAUNCH = 168, REG_CTRL = 48, REG_COMP = 224;
  static constexpr int ITEMS = 2 * N;           // items per phase of a grid
  static constexpr int SCHED = 8192;            // schedule blocks kept in shared memory
  static constexpr int NFULL = NTILE * GROUPS;  // full barriers, one per (group, tile)
  // barriers: full (NFULL), empty, freed (NTILE each), tr (GROUPS)
  static constexpr size_t smem = 1024 + (size_t)NTILE * TILE +
                                 (NFULL + 2 * NTILE + GROUPS) * sizeof(unsigned long long) +
                                 NTILE * sizeof(int4) + SCHED * sizeof(unsigned short);
};

// Byte offsets (128-byte swizzle).  Half-plane: row r < 64, column c < 128,
// boxes of 16 columns, 8 KB each.  Slab: row r in {0, 1} (y = k2, k2 + 64),
// z < 128, local column x < 32, boxes [r][x / 16] of 16 KB.
__device__ __forceinline__ uint32_t hoff(int r, int c) {
  return (uint32_t)((c >> 4) * 8192 + r * 128 + ((((c & 15) >> 1) ^ (r & 7)) << 4) + ((c & 1) << 3));
}
__device__ __forceinline__ uint32_t soff(int r, int z, int x) {
  return (uint32_t)((r * 2 + (x >> 4)) * 16384 + z * 128 + ((((x & 15) >> 1) ^ (z & 7)) << 4) +
                    ((x & 1) << 3));
}

// Shared-memory accesses by 32-bit shared-window address.  The load is not
// volatile (an unused one may be dropped) but declares that it reads memory,
// so that it stays ordered after the barrier waits and the stores that fill
// the tile (an asm without the clobber would count as reading no memory at
// all, free to move across them or to merge with an earlier load).
__device__ __forceinline__ float2 lds2(uint32_t a) {
  float2 v;
  asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts2(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void sts4(uint32_t a, float2 v, float2 w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(w.x),
               "f"(w.y)
               : "memory");
}

// 128-point FFT finished by a thread pair: v holds this thread's 64-point
// DFT (E for p = 0, O for p = 1) of points p + 2 m.  Thread p produces
// X[k] = E[k] + W_128^k O[k] and X[k + 64] = E[k] - W_128^k O[k] for
// k = j + 32 p, j < 32: it keeps its own half k in [32 p, 32 p + 32) and
// receives the partner's values of that half (lane ^ xm), so that both
// threads multiply by the same compile-time W_128^j; the odd thread then
// applies W_128^32 = DIR i.  The outputs are handed over two at a time:
// store(j, a0, a1, b0, b1) with a_u = X[j + u + 32 p] and
// b_u = X[j + u + 32 p + 64], for even j < 32.
template <int DIR, class Store>
__device__ __forceinline__ void pair_radix2(float2* v, int p, int xm, Store store) {
  static_for<0, 16>([&](auto J) {
    constexpr int j = 2 * decltype(J)::value;
    float2 av[2], bv[2];
    static_for<0, 2>([&](auto U) {
      constexpr int jj = j + decltype(U)::value;
      const float2 send = p ? v[jj] : v[32 + jj];
      float2 recv;
      recv.x = __shfl_xor_sync(0xffffffffu, send.x, xm);
      recv.y = __shfl_xor_sync(0xffffffffu, send.y, xm);
      const float2 mine = p ? v[32 + jj] : v[jj];  // this thread's k = jj + 32 p
      const float2 e = p ? recv : mine;
      const float2 t = twc<jj, 128, DIR>(p ? mine : recv);  // W_128^jj O[k]
      const float2 o = p ? mul_i<DIR>(t) : t;              // times W_128^(32 p)
      av[decltype(U)::value] = cadd(e, o);
      bv[decltype(U)::value] = csub(e, o);
    });
    store(j, av[0], av[1], bv[0], bv[1]);
  });
}

// In place, the two half-planes of a plane overlap: the even rows' item
// writes output rows 0..63, among them the odd rows 1..63 that its partner
// (the odd rows' item) reads, and the partner writes rows 64..127, among
// them the even rows 64..126 that the first item reads.  The two are the
// consecutive tickets 2 m and 2 m + 1 of one ticket pair (a phase has an
// even number of items and starts at an even ticket), so they are the
// adjacent items k and k ^ 1 of the same block, taken by the two compute
// groups.  Before its y stores an item waits until the partner's tile has
// landed, after which the partner reads nothing more from global memory.
// The wait cannot match a stale phase: the partner's (group, tile) barrier
// is next reused by item (k ^ 1) + 6, which needs the tile freed by item
// (k ^ 1) + 3, which follows this item in its own group's order; and the
// use before it, item (k ^ 1) - 6, completed before the tile was reloaded
// for (k ^ 1) - 3 < k.  The fence orders the partner's tensor-copy reads
// (async proxy) before this item's stores (generic proxy).
template <int N>
__device__ __forceinline__ bool partner_loaded(int k, const Desc& d, unsigned long long* full,
                                               const FusedArgs& a) {
  using K = Cfg<N>;
  const int kp = (d.idx & 1) ? k - 1 : k + 1;
  if (!warp_wait(&full[rowk::full_idx<K::NTILE, K::GROUPS>(kp)],
                 rowk::full_par<K::NTILE, K::GROUPS>(kp), a))
    return false;
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return true;
}

// ------------------------------------------------------------- producer
// Lanes 0..7 issue the tensor boxes; lane 0 takes and resolves tickets
// (pairs, one pair ahead).  Tensors are [N * batch][N][2N] floats.
// Tensor maps: one pair for a packed uniform batch (planes of grid g at z =
// g N + ...), or one pair per grid (PER_GRID: a unit of a mixed-edge plan,
// whose grids sit at arbitrary offsets; z within the grid).
template <int N, bool PER_GRID>
__device__ __forceinline__ void producer(const FusedArgs& a, const CUtensorMap* tins,
                                         const CUtensorMap* touts, uint32_t tiles,
                                         unsigned long long* full, unsigned long long* freed,
                                         Desc* desc, const unsigned short* sched) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, IT = K::ITEMS;
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
  int base = 0, ahead = 0;
  if (lane == 0) {
    base = take2();
    ahead = take2();
  }
  bool second = false;
  auto next_ticket = [&]() -> int {
    if (!second) {
      second = true;
      return base;
    }
    second = false;
    const int t = base + 1;
    base = ahead;
    ahead = take2();
    return t;
  };
  // every item is read once: its lines may leave L2 first (the intermediate
  // still waiting for its slabs stays)
  const unsigned long long once = policy_evict_first();
  int ready_grid = -1;
  unsigned live = 0;
  int k = 0;
  for (;; ++k) {
    const int s = k % NT;
    Desc d{-1, 0, 0, 0};
    int ok = 0;
    if (lane == 0) {
      const int t = next_ticket();
      ok = t < a.total_items;
      if (ok) {
        const int b = t / IT;
        int grid, phase;
        block_of(b, grid, phase);
        d = Desc{t, grid, phase, t - b * IT};
        if (phase == 1 && grid != ready_grid) {
          ok = bounded_wait_geq(a.work + 1 + grid, (unsigned)IT, a.status, a.timeout_ns);
          if (ok) ready_grid = grid;
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      // a stop for each compute group: items k .. k + GROUPS - 1
      if (lane == 0)
        for (int j = 0; j < K::GROUPS; ++j) {
          const int kk = k + j, sj = kk % NT;
          if (kk >= NT &&
              !mbar_wait_bounded(&freed[sj], (kk / NT - 1) & 1, a.status, a.timeout_ns))
            break;
          desc[sj] = Desc{-1, 0, 0, 0};
          mbar_arrive(&full[rowk::full_idx<NT, K::GROUPS>(kk)]);
          live &= ~(1u << sj);
        }
      live = __shfl_sync(0xffffffffu, live, 0);
      break;
    }
    d = bcast(d);
    if (k >= NT && !__all_sync(0xffffffffu, mbar_wait_bounded(&freed[s], (k / NT - 1) & 1,
                                                               a.status, a.timeout_ns)))
      break;
    live &= ~(1u << s);
    unsigned long long* fb = &full[rowk::full_idx<NT, K::GROUPS>(k)];
    if (lane == 0) {
      desc[s] = d;
      mbar_arrive_tx(fb, (unsigned)K::TILE);
    }
    __syncwarp();
    const uint32_t dst = tiles + (uint32_t)(s * K::TILE);
    if (d.phase == 0 && lane < 8) {
      // half-plane: plane z = idx / 2, rows y = parity + 2 m, 16 columns per box
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const CUtensorMap* tin = PER_GRID ? tins + d.grid : tins;
      const int zb = PER_GRID ? 0 : d.grid * N;
      tma_box_hint(dst + lane * 8192, tin, 32 * lane, d.idx & 1, zb + (d.idx >> 1), fb,
                   once);
    } else if (d.phase == 1 && lane < 4) {
      // slab: rows y = k2 + 64 r, columns 32 q + 16 h, every z
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      const int r = lane >> 1, h = lane & 1, k2 = d.idx >> 2, q = d.idx & 3;
      const CUtensorMap* tout = PER_GRID ? touts + d.grid : touts;
      const int zb = PER_GRID ? 0 : d.grid * N;
      tma_box_hint(dst + (r * 2 + h) * 16384, tout, 2 * (32 * q + 16 * h), k2 + 64 * r,
                   zb, fb, once);
    }
    live |= 1u << s;
  }
  if (lane == 0)
    for (int j = 1; j <= NT; ++j) {
      const int kk = k - j;
      if (kk >= 0 && (live & (1u << (kk % NT))))
        mbar_wait_bounded(&full[rowk::full_idx<NT, Cfg<N>::GROUPS>(kk)],
                          rowk::full_par<NT, Cfg<N>::GROUPS>(kk), a.status, a.timeout_ns);
    }
}

// Signaller warp: items in order; once the compute group is done with one,
// frees its tile and, for a half-plane, publishes it to the other blocks.
template <int N>
__device__ __forceinline__ void signaller(const FusedArgs& a, unsigned long long* full,
                                          unsigned long long* empty,
                                          unsigned long long* freed, Desc* desc) {
  constexpr int NT = Cfg<N>::NTILE;
  const int lane = threadIdx.x & 31;
  for (int k = 0;; ++k) {
    const int s = k % NT;
    const unsigned par = (k / NT) & 1;
    if (!warp_wait(&full[rowk::full_idx<NT, Cfg<N>::GROUPS>(k)],
                   rowk::full_par<NT, Cfg<N>::GROUPS>(k), a))
      return;
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

template <int N, int DIR, int NM>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    splity_fft3d_kernel(const FusedArgs a, const __grid_constant__ rowk::TensorMaps<NM> m) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, H = K::H;
  constexpr long long NN = (long long)N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const uint32_t tiles = saddr(base);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(base + (size_t)NT * K::TILE);
  unsigned long long* empty = full + K::NFULL;
  unsigned long long* freed = empty + NT;
  unsigned long long* tr = freed + NT;  // per group: x done before y
  Desc* desc = reinterpret_cast<Desc*>(tr + K::GROUPS);
  unsigned short* sched = reinterpret_cast<unsigned short*>(desc + NT);
  const int w = threadIdx.x >> 5;
  if (a.nblocks <= K::SCHED)
    for (int b = threadIdx.x; b < a.nblocks; b += K::T)
      sched[b] = (unsigned short)(a.blocks[b].grid * 2 + a.blocks[b].phase);
  if (threadIdx.x == 0) {
    for (int i = 0; i < K::NFULL; ++i) mbar_init(&full[i], 1);
    for (int s = 0; s < NT; ++s) {
      mbar_init(&empty[s], K::GW);
      mbar_init(&freed[s], 1);
    }
    for (int g = 0; g < K::GROUPS; ++g) mbar_init(&tr[g], K::GW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (w < 4) {  // warpgroup 0: control
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(K::REG_CTRL));
    if (w == 0) sy::producer<N, (NM > 1)>(a, m.in, m.out, tiles, full, freed, desc, sched);
    if (w == 1) sy::signaller<N>(a, full, empty, freed, desc);
    return;
  }
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(K::REG_COMP));

  // compute group g (warpgroup g + 1), thread gt of 128
  const int g = (w - 4) / K::GW, gt = threadIdx.x - 128 - g * K::GT, lane = threadIdx.x & 31;
  unsigned halves = 0;  // half-plane items of this group (parity of its barrier)
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!warp_wait(&full[rowk::full_idx<NT, K::GROUPS>(k)], rowk::full_par<NT, K::GROUPS>(k), a))
      break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    const uint32_t t = tiles + (uint32_t)(s * K::TILE);
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2 v[H];
    // The passes of the item (half-plane: x, then y; slab: z) share one copy
    // of the 64-point DFT (the instruction cache holds one copy better than
    // three); loads and stores of each pass are chosen once per pass.
    //   x: row r = gt / 2 of the tile, this thread's points p + 2 m, then
    //      the pair radix-2 back into the tile;
    //   y: column c = gt, 64-point DFT over the rows of this parity, times
    //      W_128^(parity k2), to global memory;
    //   z: slab (k2, q): column x = 32 q + xl, output row y = k2 + 64 yr,
    //      the y radix-2 (E + O or E - O), this thread's z points p + 2 m,
    //      then the pair radix-2 to global memory.
    const int npass = d.phase == 0 ? 2 : 1;
    bool fail = false;
#pragma unroll 1
    for (int ps = 0; ps < npass; ++ps) {
      const int kind = d.phase == 0 ? ps : 2;  // 0 x, 1 y, 2 z
      if (kind == 0) {
        const int r = gt >> 1, p = gt & 1;
#pragma unroll
        for (int m = 0; m < H; ++m) v[m] = lds2(t + hoff(r, p + 2 * m));
      } else if (kind == 1) {
        const int cs = gt ^ (((gt >> 5) & 1) << 3);  // the slot of column gt
#pragma unroll
        for (int m = 0; m < H; ++m) v[m] = lds2(t + hoff(m, cs));
      } else {
        const int wl = w - 4 - g * K::GW;
        const int p = lane >> 4, xl = (wl & 1) * 16 + (lane & 15), yr = wl >> 1;
        const float sg = yr ? -1.0f : 1.0f;  // the y radix-2: E + O or E - O
#pragma unroll
        for (int m = 0; m < H; ++m) {
          const int z = p + 2 * m;
          const float2 e = lds2(t + soff(0, z, xl));
          const float2 o = lds2(t + soff(1, z, xl));
          v[m] = fma2(o, make_float2(sg, sg), e);
        }
      }
      DFT<H, DIR>::run(v);
      if (kind != 1) {
        // the pair radix-2 of x and z (one copy), in place: v[j] = X[j + 32 p],
        // v[32 + j] = X[j + 32 p + 64]
        const int p = kind == 0 ? (gt & 1) : (lane >> 4);
        pair_radix2<DIR>(v, p, kind == 0 ? 1 : 16, [&](int j, float2 a0, float2 a1, float2 b0, float2 b1) {
          v[j] = a0;
          v[j + 1] = a1;
          v[32 + j] = b0;
          v[33 + j] = b1;
        });
      }
      if (kind == 0) {
        const int r = gt >> 1, p = gt & 1;
        __syncwarp();  // both threads of the row have read it
        // write back X[c], two adjacent columns per 16-byte store, at slot
        // c ^ 8 for the odd thread's columns (bit 5 of c set), so that the
        // two threads of a row hit different banks; the y pass reads there
        const int cx = 8 * p;
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          const int c0 = j + 32 * p;
          sy::sts4(t + hoff(r, c0 ^ cx), v[j], v[j + 1]);
          sy::sts4(t + hoff(r, (c0 + 64) ^ cx), v[32 + j], v[33 + j]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&tr[g]);
        if (!warp_wait(&tr[g], halves & 1, a)) {
          fail = true;
          break;
        }
        ++halves;
      } else if (kind == 1) {
        const int par = d.idx & 1;
        if (par)  // times W_128^k2 (compile-time twiddles)
          static_for<1, H>([&](auto K) {
            constexpr int k2 = decltype(K)::value;
            v[k2] = twc<k2, 128, DIR>(v[k2]);
          });
        if (a.in == a.out && !sy::partner_loaded<N>(k, d, full, a)) {
          fail = true;
          break;
        }
        // the intermediate: kept in L2 until its slabs have read it
        const unsigned long long keep = policy_evict_last();
        float2* dst = gout + (long long)(d.idx >> 1) * NN + (long long)par * H * N + gt;
#pragma unroll
        for (int k2 = 0; k2 < H; ++k2)
          asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(dst + (long long)k2 * N),
                       "f"(v[k2].x), "f"(v[k2].y), "l"(keep)
                       : "memory");
      } else {
        const int wl = w - 4 - g * K::GW;
        const int p = lane >> 4, xl = (wl & 1) * 16 + (lane & 15), yr = wl >> 1;
        const int k2 = d.idx >> 2, q = d.idx & 3;
        float2* dst = gout + (long long)(k2 + H * yr) * N + 32 * q + xl + (long long)(32 * p) * NN;
        if (a.do_scale) {  // (uniform) the output scale only when one is asked for
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            st_stream(dst + (long long)j * NN, cscale(v[j], a.scale));
            st_stream(dst + (long long)(j + H) * NN, cscale(v[32 + j], a.scale));
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            st_stream(dst + (long long)j * NN, v[j]);
            st_stream(dst + (long long)(j + H) * NN, v[32 + j]);
          }
        }
      }
    }
    if (fail) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// Uniform batches only (packed buffers, grids in plan order).
template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off) return cudaErrorInvalidValue;
  rowk::TensorMaps<1> m;
  if (!rowk::encode_map(&m.in[0], a.in, N, a.ngrids, 2 * (N / 2), 1, 2) ||
      !rowk::encode_map(&m.out[0], a.out, N, a.ngrids, 1, N))
    return cudaErrorInvalidValue;
  splity_fft3d_kernel<N, DIR, 1><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, m);
  return cudaGetLastError();
}

// A unit of a mixed-edge plan on packed buffers: its grids at element
// offsets host_off[0 .. ngrids) of in and out (the unit's local grid l is
// the plan's grid a.grid_map[l], at a.grid_off[that]); one pair of tensor
// maps per grid, passed with the launch.
template <int N, int DIR>
cudaError_t launch_maps(const FusedArgs& a, const long long* host_off, int grid,
                        cudaStream_t stream) {
  if (a.in_ptrs || a.ngrids > kMixMaps) return cudaErrorInvalidValue;
  rowk::TensorMaps<kMixMaps> m;
  for (int l = 0; l < a.ngrids; ++l)
    if (!rowk::encode_map(&m.in[l], a.in + host_off[l], N, 1, 2 * (N / 2), 1, 2) ||
        !rowk::encode_map(&m.out[l], a.out + host_off[l], N, 1, 1, N))
      return cudaErrorInvalidValue;
  splity_fft3d_kernel<N, DIR, kMixMaps><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, m);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.launch_maps = &launch_maps<N, DIR>;
  k.func = (const void*)&splity_fft3d_kernel<N, DIR, 1>;
  k.func_maps = (const void*)&splity_fft3d_kernel<N, DIR, kMixMaps>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.twiddle_entries = N;  // (the codelets need no table; one is uploaded anyway)
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;  // the tiles and up to four tickets held ahead
  k.phase_items = Cfg<N>::ITEMS;
  return k;
}

}  // namespace sy
}  // namespace fft3d
