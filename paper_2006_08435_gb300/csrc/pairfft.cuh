// Persistent 3D FFT kernel for 32^3 .. 96^3 grids with every 1D transform
// of n points in a pair of threads: thread p of the pair holds the points
// p + 2 m (m < h = n/2), runs the h-point DFT of them in registers (E for
// p = 0, O for p = 1), and the pair finishes with one radix-2 step,
//   X[k] = E[k] + W_n^k O[k],  X[k + h] = E[k] - W_n^k O[k],
// after exchanging half of their values with warp shuffles (the thread pair
// of the split-y kernel, for h = 16, 24, 40 and 48).  A whole n-point pencil
// in one thread would need 2n registers for its points alone.
//
// Items are those of the thread-per-pencil kernels: P planes (x, then y,
// the y results straight to global memory as rows of the intermediate, kept
// in L2) or P slabs (rows y of every z: the z transforms, to the output);
// P = 4 at 32^3 (32 KB items), 2 at 48^3 (36 KB), 1 at 80^3 and 96^3 (50
// and 72 KB).  An item
// arrives as n/16 tensor boxes of 16 complex x n rows x P, 128-byte
// swizzled; tile row r is n pz + y for planes, P z + y for slabs.  Lanes:
//   x: row r = gt / 2, p = gt % 2 (adjacent lanes);
//   y and z: plane (slab) w / (n/16), column c = 16 (w mod n/16) + lane % 16
//     of warp w of the group, p = lane / 16 (lanes l and l ^ 16), so that a
//     half-warp reads or writes 16 consecutive complex (128 bytes).
// Every shared-memory access moves its bytes in the fewest wavefronts.
//
// Block: two compute groups of 2 P n threads (items k = g, g + 2, ...), a
// producer warp (tickets, slab dependencies, the item's tensor copies into
// a ring of three tiles, five at 32^3 and 48^3; full barriers per (group, tile), as
// in the split-y kernel) and a signaller warp (frees tiles, publishes
// finished planes).
// Bounded waits as in the other persistent kernels.  In place is safe by
// construction: a plane item writes only the planes it read, a slab only its
// own rows of every z.
#pragma once

#include "splity.cuh"

namespace fft3d {
namespace pf {

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
using sy::lds2;
using sy::sts4;

template <int N>
struct Cfg {
  static_assert(N == 32 || N == 48 || N == 80 || N == 96,
                "thread-pair kernel covers 32, 48, 80 and 96");
  static constexpr int H = N / 2;               // points per thread
  static constexpr int Q = H / 2;               // outputs of each half per thread
  static_assert(Q % 2 == 0, "outputs handed over two at a time");
  static constexpr int P = N == 32 ? 4 : N == 48 ? 2 : 1;  // planes (slabs) per item
  static constexpr int ROWS = P * N;            // tile rows of an item
  static constexpr int SEG = 16;                // complex per 128-byte box row
  static constexpr int NSEG = N / SEG;          // tensor boxes per item
  static constexpr int REGION = ROWS * 128;     // bytes of one box
  static constexpr int TILE = NSEG * REGION;    // bytes of one item
  static_assert(REGION % 1024 == 0, "boxes 1024-byte aligned (swizzle)");
  static constexpr int NTILE = N <= 48 ? 5 : 3;  // odd: coprime with the two groups
  static constexpr int GROUPS = 2;
  static constexpr int GT = 2 * ROWS;           // threads per compute group
  static constexpr int GW = GT / 32;
  static constexpr int NCW = GROUPS * GW;       // compute warps
  static constexpr int T = 32 * (NCW + 2);      // plus producer and signaller
  static constexpr int ITEMS = N / P;           // items per phase of a grid
  static constexpr int SCHED = 4096;            // schedule blocks kept in shared memory
  static constexpr int NFULL = NTILE * GROUPS;  // full barriers, one per (group, tile)
  // barriers: full (NFULL), empty, freed (NTILE each), tr (GROUPS)
  static constexpr size_t smem = 1024 + (size_t)NTILE * TILE +
                                 (NFULL + 2 * NTILE + GROUPS) * sizeof(unsigned long long) +
                                 NTILE * sizeof(int4) + SCHED * sizeof(unsigned short);
};

// Byte offset of complex (row r, column c) in a tile: box c / 16, row r of
// the box (128 bytes), 16-byte chunk (c mod 16) / 2 XOR r mod 8.
template <int N>
__device__ __forceinline__ uint32_t off(int r, int c) {
  return (uint32_t)((c >> 4) * Cfg<N>::REGION + r * 128 + ((((c & 15) >> 1) ^ (r & 7)) << 4) +
                    ((c & 1) << 3));
}

// The pair's radix-2 step: v holds this thread's h-point DFT (E for p = 0,
// O for p = 1) of points p + 2 m.  Thread p produces X[k] and X[k + h] for
// k = j + Q p, j < Q: it keeps its own half and receives the partner's
// values of that half (lane ^ xm), so that both threads multiply by the same
// compile-time W_n^j; the odd thread then applies W_n^Q = DIR i.  Results in
// place: v[j] = X[j + Q p], v[Q + j] = X[j + Q p + h].
template <int N, int DIR>
__device__ __forceinline__ void pair_radix2(float2* v, int p, int xm) {
  constexpr int Q = Cfg<N>::Q;
  static_for<0, Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    const float2 send = p ? v[j] : v[Q + j];
    float2 recv;
    recv.x = __shfl_xor_sync(0xffffffffu, send.x, xm);
    recv.y = __shfl_xor_sync(0xffffffffu, send.y, xm);
    const float2 mine = p ? v[Q + j] : v[j];        // this thread's k = j + Q p
    const float2 e = p ? recv : mine;
    const float2 t = twc<j, N, DIR>(p ? mine : recv);  // W_n^j O[k]
    const float2 o = p ? mul_i<DIR>(t) : t;           // times W_n^(Q p)
    v[j] = cadd(e, o);
    v[Q + j] = csub(e, o);
  });
}

// ------------------------------------------------------------- producer
// Lane 0 takes and resolves tickets (pairs, one pair ahead); lanes
// 0 .. NSEG-1 issue the tensor boxes.  Tensors are [N * batch][N][2N]
// floats (one pair of maps for a packed batch), or one pair per grid
// (PER_GRID: a unit of a mixed-edge plan; z within the grid).
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
    if (lane < K::NSEG) {
      // the tile was last read or written by the compute threads' plain
      // accesses, a slab's rows by other blocks' plain stores (seen through
      // lane 0's acquire)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (d.phase == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
      const uint32_t dst = tiles + (uint32_t)(s * K::TILE + lane * K::REGION);
      const int zb = PER_GRID ? 0 : d.grid * N;
      if (d.phase == 0)  // planes z = P idx ..: box {16 x, all y, P z}
        tma_box_hint(dst, PER_GRID ? tins + d.grid : tins, 2 * K::SEG * lane, 0,
                     zb + K::P * d.idx, fb, once);
      else  // slabs y = P idx ..: box {16 x, P y, all z}
        tma_box_hint(dst, PER_GRID ? touts + d.grid : touts, 2 * K::SEG * lane, K::P * d.idx, zb,
                     fb, once);
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

// Signaller warp: items in order; once the compute group is done with one,
// frees its tile and, for a plane, publishes it to the other blocks.
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
    pairfft_fft3d_kernel(const FusedArgs a, const __grid_constant__ rowk::TensorMaps<NM> m) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, H = K::H, Q = K::Q;
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

  if (w == K::NCW) {
    pf::producer<N, (NM > 1)>(a, m.in, m.out, tiles, full, freed, desc, sched);
    return;
  }
  if (w == K::NCW + 1) {
    pf::signaller<N>(a, full, empty, freed, desc);
    return;
  }

  // compute group g (warps g GW .. g GW + GW - 1), thread gt of 2n
  const int g = w / K::GW, wl = w - g * K::GW, gt = threadIdx.x - g * K::GT;
  const int lane = threadIdx.x & 31;
  // column passes: plane (slab) qy of the item, column cy
  const int qy = K::P == 1 ? 0 : wl / (N / 16);
  const int cy = 16 * (K::P == 1 ? wl : wl % (N / 16)) + (lane & 15), py = lane >> 4;
  unsigned planes = 0;  // plane items of this group (parity of its barrier)
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!warp_wait(&full[rowk::full_idx<NT, K::GROUPS>(k)], rowk::full_par<NT, K::GROUPS>(k),
                   a))
      break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    const uint32_t t = tiles + (uint32_t)(s * K::TILE);
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2 v[H];
    // The passes of the item (plane: x, then y; slab: z) share one copy of
    // the h-point DFT and of the pair step:
    //   x: row r = gt / 2, points p + 2 m, back into the tile;
    //   y: column cy of plane qy, rows py + 2 m, to rows of the
    //      intermediate (kept in L2 for its slabs);
    //   z: column cy of slab qy, planes py + 2 m, to the output.
    const int npass = d.phase == 0 ? 2 : 1;
    bool fail = false;
#pragma unroll 1
    for (int ps = 0; ps < npass; ++ps) {
      const int kind = d.phase == 0 ? ps : 2;  // 0 x, 1 y, 2 z
      const int p = kind == 0 ? (gt & 1) : py;
      if (kind == 0) {
        const int r = gt >> 1;
#pragma unroll
        for (int j = 0; j < H; ++j) v[j] = lds2(t + off<N>(r, p + 2 * j));
      } else if (kind == 1) {
#pragma unroll
        for (int j = 0; j < H; ++j) v[j] = lds2(t + off<N>(qy * N + py + 2 * j, cy));
      } else {
#pragma unroll
        for (int j = 0; j < H; ++j) v[j] = lds2(t + off<N>((py + 2 * j) * K::P + qy, cy));
      }
      DFT<H, DIR>::run(v);
      pf::pair_radix2<N, DIR>(v, p, kind == 0 ? 1 : 16);
      if (kind == 0) {
        // X[c] back into row r, two adjacent columns per 16-byte store
        const int r = gt >> 1;
        __syncwarp();  // both threads of the row have read it
#pragma unroll
        for (int j = 0; j < Q; j += 2) {
          const int c0 = j + Q * p;
          sts4(t + off<N>(r, c0), v[j], v[j + 1]);
          sts4(t + off<N>(r, c0 + H), v[Q + j], v[Q + j + 1]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&tr[g]);
        if (!warp_wait(&tr[g], planes & 1, a)) {
          fail = true;
          break;
        }
        ++planes;
      } else if (kind == 1) {
        // rows k = j + Q py (and + h) of plane P idx + qy of the intermediate
        const unsigned long long keep = policy_evict_last();
        float2* dst = gout + (long long)(K::P * d.idx + qy) * NN + (long long)(Q * py) * N + cy;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(dst + (long long)j * N),
                       "f"(v[j].x), "f"(v[j].y), "l"(keep)
                       : "memory");
          asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(dst + (long long)(j + H) * N),
                       "f"(v[Q + j].x), "f"(v[Q + j].y), "l"(keep)
                       : "memory");
        }
      } else {
        // planes k = j + Q py (and + h) of row y = P idx + qy, column cy
        float2* dst = gout + (long long)(K::P * d.idx + qy) * N + cy + (long long)(Q * py) * NN;
        const float sc = a.do_scale ? a.scale : 1.0f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          st_stream(dst + (long long)j * NN, cscale(v[j], sc));
          st_stream(dst + (long long)(j + H) * NN, cscale(v[Q + j], sc));
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
  if (!rowk::encode_map(&m.in[0], a.in, N, a.ngrids, N, Cfg<N>::P) ||
      !rowk::encode_map(&m.out[0], a.out, N, a.ngrids, Cfg<N>::P, N))
    return cudaErrorInvalidValue;
  pairfft_fft3d_kernel<N, DIR, 1><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, m);
  return cudaGetLastError();
}

// A unit of a mixed-edge plan on packed buffers: its grids at element
// offsets host_off[0 .. ngrids) of in and out; one pair of tensor maps per
// grid, passed with the launch.
template <int N, int DIR>
cudaError_t launch_maps(const FusedArgs& a, const long long* host_off, int grid,
                        cudaStream_t stream) {
  if (a.in_ptrs || a.ngrids > kMixMaps) return cudaErrorInvalidValue;
  rowk::TensorMaps<kMixMaps> m;
  for (int l = 0; l < a.ngrids; ++l)
    if (!rowk::encode_map(&m.in[l], a.in + host_off[l], N, 1, N, Cfg<N>::P) ||
        !rowk::encode_map(&m.out[l], a.out + host_off[l], N, 1, Cfg<N>::P, N))
      return cudaErrorInvalidValue;
  pairfft_fft3d_kernel<N, DIR, kMixMaps><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, m);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.launch_maps = &launch_maps<N, DIR>;
  k.func = (const void*)&pairfft_fft3d_kernel<N, DIR, 1>;
  k.func_maps = (const void*)&pairfft_fft3d_kernel<N, DIR, kMixMaps>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.twiddle_entries = N;  // (the codelets need no table; one is uploaded anyway)
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;  // the tiles and up to four tickets held ahead
  k.phase_items = Cfg<N>::ITEMS;
  return k;
}

}  // namespace pf
}  // namespace fft3d
