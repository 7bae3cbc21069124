// Persistent transforms of REAL n^3 grids (n = 64, 128): forward (R2C, sign -1, real
// grid -> half spectrum kx = 0 .. n/2) and inverse (C2R, sign +1), each in
// two phases of work items with the ticket schedule and L2-resident
// intermediate of the complex kernels.  Every 1D transform of n points is
// done as DFTs of h = n/2 points in one thread's registers, so a real grid
// costs about half the arithmetic and half the bytes of a complex one.
//
// Forward, real grid r -> half spectrum F (layout [kz][ky][h + 1]):
//   plane item (g, z): plane z of r (n rows of n reals) -> tile.
//     x: thread y takes row y as z[m] = r[2m] + i r[2m+1] (m < h), DFTs
//       it and splits the result into the half row X[0 .. h] of the real
//       row: E[k] = (Z[k] + conj Z[h-k]) / 2 and O[k] = (Z[k] - conj
//       Z[h-k]) / (2i) are the transforms of the even and odd samples, and
//       X[k] = E[k] + W_n^k O[k].  X[0] and X[h] are real; the row keeps
//       X[0] + i X[h] in column 0.
//     y: column c < h of the plane as two h-point DFTs (decimation in
//       frequency: half 0 transforms a[y] + a[y+h] into the outputs ky = 2k,
//       half 1 transforms (a[y] - a[y+h]) W_n^y into ky = 2k + 1).  Column 0
//       then holds C = Y0 + i Yh, the y transforms of the real columns X[0]
//       and X[h]; both are Hermitian, so Y0 = (C(ky) + conj C(-ky)) / 2 and
//       Yh = (C(ky) - conj C(-ky)) / (2i), and ky, -ky have the same parity
//       (outputs of the same thread, separated by its warp).  The plane's
//       half rows go to out[g][z][ky][0 .. h].
//   slab item (g, ky): rows (z, ky), columns 0 .. h-1 of out -> tile; z DFTs
//     as for y; results (scaled) back to those rows.
//   Nyquist item (g): column h of out.  Since F(kx, -ky, -kz) = conj F(kx,
//     ky, kz) and -h = h (mod n), only the pencils ky = 0 .. h are needed;
//     ky = 0 and ky = h are real before the z transform and share one
//     pencil (separated after it like column 0 above), the rest come from
//     conj.  The plane items leave these pencils in a workspace of n x h
//     complex per grid, [z][p] with p = ky for 0 < ky < h and p = 0 holding
//     (Yh(0), Yh(h)), so the item loads them with one copy.
// Inverse, half spectrum F -> real grid (Re of the inverse transform of F's
// Hermitian extension):
//   slab item (g, ky): rows (kz, ky) of F -> tile.  Columns 0 and h are
//     replaced by their Hermitian parts (F(k) + conj F(-k)) / 2 -- the only
//     bins where the extension is not Hermitian already -- and packed into
//     column 0 as A + i B; z DFTs of columns 0 .. h-1 into out, viewed as
//     [g][z][ky][h] complex (n^3 floats: the size of the real grid).
//   plane item (g, z): that plane -> tile; y DFTs back into the tile (column
//     0 now holds X[0] + i X[h] of every row, both real); x: thread y forms
//     Z[k] = A[k] + i B[k] with A[k] = X[k] + conj X[h-k] and B[k] = (X[k] -
//     conj X[h-k]) W_n^k, DFTs it, and z[m] = r[2m] + i r[2m+1] is the row
//     (scaled), written back with bulk copies.
//
// Every item has 128 rows: at 128^3 one plane (or one row ky of every z),
// at 64^3 two (P = 128/n), so the per-item costs (ticket, barriers,
// copies) are spread over as much data at every edge.
//
// Block: a control warpgroup (producer warp: tickets, schedule lookup,
// dependency waits, the item's copies; publisher warp: finished phase-0
// items to the other blocks, in order) and compute groups of 128 threads
// (two at 128^3, three at 64^3); a ring of three (four) tiles.  Every item
// arrives with at most five copies (the copy engine's cost is per copy,
// not per byte, at these sizes):
//   real planes: n/32 tensor boxes of 32 floats x n rows x P planes,
//     128-byte swizzled (16-byte chunk j of row r at chunk j ^ (r mod 8)),
//     so that both the thread-per-row and the thread-per-column accesses
//     are conflict-free;
//   rows (z, ky) of a half spectrum: one tensor box over a view of the half
//     spectra as ROW PAIRS (16 (h + 1) bytes, a 16-byte multiple, where a
//     single row of 8 (h + 1) bytes is not): at P = 1 pair ky/2 from float
//     0 (even ky: columns 0 .. h+1) or 2h (odd ky: column h of row ky-1,
//     then columns 0 .. h), 8 (h + 2) bytes per tile row; at P = 2 the
//     whole pair;
//   the inverse's mirror columns: two boxes of 4 floats x n per row ky, of
//     the same view;
//   contiguous planes of the intermediate or the Nyquist workspace: one
//     bulk copy (dense rows).
// A tile goes back to the producer as soon as its group has read it.
// Waits are bounded in time and report through the status word.
#pragma once

#include "rowfft.cuh"

namespace fft3d {
namespace rg {

using mb::mbar_arrive;
using mb::mbar_arrive_tx;
using mb::mbar_init;
using mb::mbar_wait_bounded;
using mb::saddr;
using mb::warp_wait;
using rowk::spin_geq;

template <int N>
struct Cfg {
  static_assert(N == 64 || N == 128, "edges 64 and 128");
  static constexpr int H = N / 2;               // points of each register DFT
  static constexpr int HC = N / 2 + 1;          // complex per half-spectrum row
  // an item is P planes (or P rows ky of every z), 128 rows in all
  static constexpr int P = 128 / N;
  static constexpr int ROWS = P * N;
  // z items: bytes per tile row, one z (one row ky from float 0 or 2h of
  // its pair, or, with P >= 2, P/2 whole pairs); 16-byte multiples
  static constexpr int PITCH = P == 1 ? (H + 2) * 8 : 8 * HC * P;
  static constexpr int XP = (H + 2) * 8;        // padded row of a plane (thread-per-row passes)
  static constexpr int MAIN = N * PITCH > ROWS * XP ? N * PITCH : ROWS * XP;
  static constexpr int MIRROR = 2 * P * N * 16; // inverse: mirror boxes of columns 0 and h
  static constexpr int TILE = MAIN + MIRROR;
  static_assert(TILE % 1024 == 0, "tiles 1024-byte aligned (swizzle)");
  // bytes of one swizzled box of the real planes (32 floats of each row)
  static constexpr int SWB = 32 * ROWS * 4;
  static constexpr int GT = ROWS;               // threads per compute group (128)
  static constexpr int GW = GT / 32;
  // compute groups: two warpgroups at 128^3 (64-point DFTs, 224 registers),
  // three at 64^3 (32-point DFTs, 152 registers)
  static constexpr int GROUPS = N == 128 ? 2 : 3;
  static constexpr int NTILE = N == 128 ? 3 : 4;  // coprime with GROUPS
  static constexpr int T = 128 + GROUPS * GT;   // control warpgroup + compute
  // registers: 65536 / T at launch (168 at 128^3, 128 at 64^3); setmaxnreg
  // moves them from the control warpgroup to the compute ones:
  // 128 * 56 + 256 * 224 = 64512 <= 384 * 168, 128 * 56 + 384 * 152 = 65536
  static constexpr int REG_CTRL = 56, REG_COMP = N == 128 ? 224 : 152;
  static constexpr int IPP = N / P;             // items per phase of a grid
  static constexpr int DQ = 16;                 // finished items queued for the publisher
  static constexpr int SCHED = 2048;            // schedule blocks kept in shared memory
  static constexpr int NFULL = NTILE * GROUPS;
  static constexpr size_t smem = 1024 + (size_t)NTILE * TILE + GROUPS * GT * sizeof(float2) +
                                 (NFULL + NTILE + GROUPS + DQ) * sizeof(unsigned long long) +
                                 NTILE * sizeof(int4) + (DQ + 1) * sizeof(int) +
                                 SCHED * sizeof(int);
};

struct Desc {
  int item, grid, phase, idx;
};

// Full barriers: one per (group, tile); item k uses tile k % NT and group
// k % G (NT, G coprime), so consecutive phases of a barrier are consecutive
// uses by the same group.
template <int NT, int G>
__device__ __forceinline__ int full_idx(int k) {
  return (k % G) * NT + k % NT;
}
template <int NT, int G>
__device__ __forceinline__ unsigned full_par(int k) {
  return (unsigned)(k / (NT * G)) & 1u;
}

// One row into the tile: a bulk copy (no tensor map) completing on `bar`.
__device__ __forceinline__ void bulk_row(uint32_t dst, const void* src, unsigned bytes,
                                         unsigned long long* bar, unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
      : "memory");
}

// Tile row (shared) -> global, tracked by this thread's bulk group.
__device__ __forceinline__ void bulk_store_row(void* dst, uint32_t src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void st_keep(float2* p, float2 v, unsigned long long policy) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
               "l"(policy)
               : "memory");
}

__device__ __forceinline__ void st_keep_f(float* p, float v, unsigned long long policy) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(policy)
               : "memory");
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Byte offset of 16-byte chunk j (floats 4j .. 4j+3) of row r of the real
// planes in their swizzled tile (boxes of 32 floats, 128-byte swizzle).
template <int N>
__device__ __forceinline__ uint32_t swz(int r, int j) {
  return (uint32_t)((j >> 3) * Cfg<N>::SWB + r * 128 + (((j & 7) ^ (r & 7)) << 4));
}

// ------------------------------------------------------------ row algebra
// Half-length DFT of a real row -> its half spectrum.  In: v = Z, the
// H-point DFT of z[m] = r[2m] + i r[2m+1].  Out: v[0] = (X[0], X[H]) (both
// real), v[k] = X[k] for 0 < k < H, X the 2H-point DFT of r with sign DIR.
template <int H, int DIR>
__device__ __forceinline__ void real_split(float2* v) {
  const float2 z0 = v[0];
  v[0] = make_float2(z0.x + z0.y, z0.x - z0.y);
  static_for<1, H / 2>([&](auto K) {
    constexpr int k = decltype(K)::value;
    const float2 A = v[k], B = v[H - k];
    const float2 e = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));  // (A + conj B) / 2
    const float2 o = make_float2(0.5f * (A.y + B.y), 0.5f * (B.x - A.x));  // (A - conj B) / 2i
    const float2 p = twc<k, 2 * H, DIR>(o);
    v[k] = make_float2(e.x + p.x, e.y + p.y);
    v[H - k] = make_float2(e.x - p.x, p.y - e.y);  // conj(e - p)
  });
  // k = H/2: E = Re Z, O = Im Z, W_2H^(H/2) = DIR i
  const float2 A = v[H / 2];
  v[H / 2] = make_float2(A.x, (float)DIR * A.y);
}

// The inverse step.  In: v[0] = (X[0], X[H]), v[k] = X[k] for 0 < k < H, the
// half spectrum of a real row (X[2H - k] = conj X[k]).  Out: v = Z with
// Z[k] = A[k] + i B[k], A[k] = X[k] + conj X[H-k], B[k] = (X[k] - conj
// X[H-k]) W_2H^k; the H-point DFT of Z (sign DIR) is z[m] = r[2m] + i
// r[2m+1], r the 2H-point DFT of X with sign DIR.
template <int H, int DIR>
__device__ __forceinline__ void real_merge(float2* v) {
  const float2 x0 = v[0];
  v[0] = make_float2(x0.x + x0.y, x0.x - x0.y);
  static_for<1, H / 2>([&](auto K) {
    constexpr int k = decltype(K)::value;
    const float2 p = v[k], q = v[H - k];
    const float2 A = make_float2(p.x + q.x, p.y - q.y);                 // p + conj q
    const float2 B = twc<k, 2 * H, DIR>(make_float2(p.x - q.x, p.y + q.y));  // (p - conj q) W^k
    v[k] = make_float2(A.x - B.y, A.y + B.x);                           // A + i B
    v[H - k] = make_float2(A.x + B.y, B.x - A.y);                       // conj A + i conj B
  });
  // k = H/2: A = 2 Re X, B = (2i Im X)(DIR i) = -2 DIR Im X
  const float2 X = v[H / 2];
  v[H / 2] = make_float2(2.0f * X.x, -2.0f * (float)DIR * X.y);
}

// ---------------------------------------------------------- column passes
// Decimation-in-frequency first step of an N-point DFT over a column whose
// point r is at at(r) (half `HALF` of the outputs): v[r] = a[r] + a[r+H]
// (HALF 0) or (a[r] - a[r+H]) W_N^r (HALF 1).  The H-point DFT of v is then
// output 2k + HALF at v[k].
template <int N, int DIR, int HALF, class At>
__device__ __forceinline__ void load_dif(At&& at, float2* v) {
  constexpr int H = N / 2;
  static_for<0, H>([&](auto R) {
    constexpr int r = decltype(R)::value;
    const float2 a = *at(r), b = *at(r + H);
    if constexpr (HALF == 0) v[r] = cadd(a, b);
    else v[r] = twc<r, N, DIR>(csub(a, b));
  });
}
// Rows P bytes apart from t, byte `col` within a row.
template <int N, int DIR, int P>
__device__ __forceinline__ void load_dif_rows(const unsigned char* t, int col, int h, float2* v) {
  auto at = [&](int r) { return reinterpret_cast<const float2*>(t + r * P + col); };
  if (h == 0) load_dif<N, DIR, 0>(at, v);
  else load_dif<N, DIR, 1>(at, v);
}

// --------------------------------------------------------------- producer
// Lane 0 takes tickets (two ahead, so the atomic's round trip overlaps the
// item before) and resolves them (schedule block by binary search over the
// block starts, kept in shared memory when they fit); phase-1 items wait
// until all N phase-0 items of their grid are published.  Lanes 0 .. 31 then
// issue the item's N row copies, four each.
template <int N, int DIR>
__device__ __forceinline__ void producer(const FusedArgs& a, const CUtensorMap* m0,
                                         const CUtensorMap* m1, uint32_t tiles,
                                         unsigned long long* full, unsigned long long* empty,
                                         unsigned long long* done, int* pubq,
                                         volatile int* pub_done, Desc* desc, const int* sched) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, DQ = K::DQ, G = K::GROUPS, H = K::H, P = K::P, IPP = K::IPP;
  const int lane = threadIdx.x & 31;
  // every schedule block has IPB tickets (forward: the plane block's last
  // ticket is empty, matching the z block's Nyquist item), so a ticket's
  // block is t / IPB; (grid, phase) of the first SCHED blocks are in shared
  // memory
  constexpr int IPB = IPP + (DIR < 0 ? 1 : 0);
  auto resolve = [&](int t, Desc& d) {
    const int b = t / IPB;
    int gp;
    if (b < K::SCHED) gp = sched[b];
    else gp = a.blocks[b].grid * 2 + a.blocks[b].phase;
    d.grid = gp >> 1;
    d.phase = gp & 1;
    d.idx = t - b * IPB;
    d.item = t;
  };
  int t1 = 0, t2 = 0;
  if (lane == 0) {
    t1 = (int)atomicAdd(a.work, 1u);
    t2 = (int)atomicAdd(a.work, 1u);
  }
  int ready_grid = -1;
  unsigned live = 0;
  const unsigned long long once = rowk::policy_evict_first();
  int k = 0;
  for (;; ++k) {
    const int s = k % NT;
    Desc d{-1, 0, 0, 0};
    int ok = 1;
    if (lane == 0) {
      int t;
      do {  // (the empty tickets are skipped)
        t = t1;
        t1 = t2;
        t2 = (int)atomicAdd(a.work, 1u);
        ok = t < a.total_items;
        if (ok) resolve(t, d);
      } while (ok && DIR < 0 && d.phase == 0 && d.idx == IPP);
      if (ok) {
        if (d.phase == 1 && d.grid != ready_grid) {
          ok = bounded_wait_geq(a.work + 1 + d.grid, (unsigned)IPP, a.status, a.timeout_ns);
          if (ok) ready_grid = d.grid;
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();  // lane 0's acquire before the copies of every lane
    if (!ok) {
      if (lane == 0) {
        // a stop for each compute group: items k .. k + G - 1, each tile once
        // its group is done with its earlier item
        for (int j = 0; j < G; ++j) {
          const int kk = k + j, sj = kk % NT;
          if (kk >= NT &&
              !mbar_wait_bounded(&empty[sj], (kk / NT - 1) & 1, a.status, a.timeout_ns))
            break;
          desc[sj] = Desc{-1, 0, 0, 0};
          mbar_arrive(&full[full_idx<NT, G>(kk)]);
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
    d.item = __shfl_sync(0xffffffffu, d.item, 0);
    d.grid = __shfl_sync(0xffffffffu, d.grid, 0);
    d.phase = __shfl_sync(0xffffffffu, d.phase, 0);
    d.idx = __shfl_sync(0xffffffffu, d.idx, 0);
    // the tile: its group is done with item k - NT; the publisher's slot of
    // item k: item k - DQ published
    int fr = 1;
    if (lane == 0) {
      if (k >= NT) fr = mbar_wait_bounded(&empty[s], (k / NT - 1) & 1, a.status, a.timeout_ns);
      if (fr) fr = spin_geq(pub_done, k - DQ + 1, a);
    }
    if (!__shfl_sync(0xffffffffu, fr, 0)) break;
    live &= ~(1u << s);
    unsigned long long* fb = &full[full_idx<NT, G>(k)];
    // the item's copies: tensor boxes or one bulk copy.  Item idx covers
    // planes (or rows ky) P idx .. P idx + P - 1.
    const int g = d.grid, i0 = P * d.idx;
    unsigned tx = 0;
    const char* bulk = nullptr;
    if (DIR < 0) {
      if (d.phase == 0) tx = P * N * N * 4;            // real planes: N/32 swizzled boxes
      else if (d.idx < IPP) tx = N * K::PITCH;         // rows (z, ky): one pair-view box
      else {                                           // Nyquist workspace
        bulk = reinterpret_cast<const char*>(a.aux) + (long long)g * N * H * 8;
        tx = N * H * 8;
      }
    } else {
      if (d.phase == 0) tx = N * K::PITCH + K::MIRROR; // rows (kz, ky) and the mirror columns
      else {                                           // planes of the intermediate
        bulk = reinterpret_cast<const char*>(a.out) + ((long long)g * N + i0) * N * H * 8;
        tx = P * N * H * 8;
      }
    }
    if (lane == 0) {
      desc[s] = d;
      pubq[k % DQ] = d.phase == 0 ? d.grid : -1;  // read by the publisher after item k
      mbar_arrive_tx(fb, tx);
    }
    __syncwarp();
    // the tile was last written by the compute threads' plain stores; the
    // intermediate by other blocks' plain stores (seen through lane 0's
    // acquire)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (d.phase == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
    const uint32_t dst = tiles + (uint32_t)(s * K::TILE);
    if (bulk) {
      if (lane == 0) bulk_row(dst, bulk, tx, fb, once);
    } else if (DIR < 0 && d.phase == 0) {
      if (lane < (N >= 32 ? N / 32 : 1))  // planes i0 ..: box {32 x, all y, P planes}
        rowk::tma_box_hint(dst + lane * K::SWB, m1, 32 * lane, 0, g * N + i0, fb, once);
    } else {
      // rows i0 .. of every z of grid g (pair i0/2; with P = 1 from float 0
      // or 2h by parity); the inverse also the mirror rows -ky: columns 0
      // and h, one box each
      if (lane == 0)
        rowk::tma_box_hint(dst, m0, (P == 1 && (i0 & 1)) ? 2 * H : 0, i0 >> 1, g * N, fb, once);
      if (DIR > 0 && lane >= 1 && lane <= 2 * P) {
        const int r = (lane - 1) >> 1, col = (lane - 1) & 1;
        const int my = (N - i0 - r) % N;
        const int x = col == 0 ? ((my & 1) ? 2 * H : 0) : ((my & 1) ? 4 * H : 2 * H);
        rowk::tma_box_hint(dst + K::MAIN + (lane - 1) * N * 16, m1, x, my >> 1, g * N, fb, once);
      }
    }
    live |= 1u << s;
  }
  // no copy may still be writing a tile when the block exits (only after a
  // failure can one be left unconsumed)
  if (lane == 0)
    for (int j = 1; j <= NT; ++j) {
      const int kk = k - j;
      if (kk >= 0 && (live & (1u << (kk % NT))))
        mbar_wait_bounded(&full[full_idx<NT, G>(kk)], full_par<NT, G>(kk), a.status,
                          a.timeout_ns);
    }
}

// Publisher warp (lane 0): finished items in order; a phase-0 item is
// published to the other blocks (per-grid counter) after a GPU-scope fence.
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

// ----------------------------------------------------------------- kernel
// Tensor maps: forward m0 = the half spectra `out` as row pairs (box n + 4
// floats x 1 x n), m1 = the real grids `in` (box 32 floats x n x 1,
// swizzled); inverse m0 = the half spectra `in` as row pairs (box n + 4 x 1
// x n), m1 = the same view with boxes of 4 floats (mirror columns).
template <int N, int DIR>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    rgrid_fft3d_kernel(const FusedArgs a, const __grid_constant__ CUtensorMap m0,
                       const __grid_constant__ CUtensorMap m1) {
  using K = Cfg<N>;
  constexpr int NT = K::NTILE, G = K::GROUPS, H = K::H, HC = K::HC, P = K::P, IPP = K::IPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // tiles 1024-byte aligned (the swizzle pattern follows address bits 7..9)
  unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const uint32_t tiles = saddr(base);
  float2* scratch = reinterpret_cast<float2*>(base + (size_t)NT * K::TILE);  // per group: GT
  unsigned long long* full = reinterpret_cast<unsigned long long*>(scratch + G * K::GT);
  unsigned long long* empty = full + K::NFULL;
  unsigned long long* tr = empty + NT;  // per group: its steps inside an item
  unsigned long long* done = tr + G;    // items finished, for the publisher
  Desc* desc = reinterpret_cast<Desc*>(done + K::DQ);
  int* pubq = reinterpret_cast<int*>(desc + NT);
  volatile int* pub_done = pubq + K::DQ;
  int* sched = pubq + K::DQ + 1;
  const int w = threadIdx.x >> 5;
  for (int b = threadIdx.x; b < a.nblocks && b < K::SCHED; b += K::T)
    sched[b] = a.blocks[b].grid * 2 + a.blocks[b].phase;
  if (threadIdx.x == 0) {
    for (int i = 0; i < K::NFULL; ++i) mbar_init(&full[i], 1);
    for (int s = 0; s < NT; ++s) mbar_init(&empty[s], K::GW);
    for (int g = 0; g < G; ++g) mbar_init(&tr[g], K::GW);
    for (int q = 0; q < K::DQ; ++q) mbar_init(&done[q], K::GW);
    *pub_done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (w < 4) {  // control warpgroup
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(K::REG_CTRL));
    if (w == 0) producer<N, DIR>(a, &m0, &m1, tiles, full, empty, done, pubq, pub_done, desc, sched);
    if (w == 1) publisher<N>(a, done, pubq, pub_done);
    return;
  }
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(K::REG_COMP));

  // compute group g (of the warpgroups 1 ..), thread gt of ROWS = P N.
  // Row passes: row gt of the item (plane gt / N).  Column passes: plane or
  // row r = gt / N of the item, column c = gt % H, output half h = (gt / H)
  // mod 2 (the same for a whole warp).
  const int g = (w - 4) / K::GW, gt = threadIdx.x - 128 - g * K::GT, lane = threadIdx.x & 31;
  const int c = gt % H, h = (gt / H) & 1, r = gt / N;
  unsigned steps = 0;  // group barriers passed (parity of tr[g])
  auto group_sync = [&]() -> bool {
    __syncwarp();
    if (lane == 0) mbar_arrive(&tr[g]);
    const bool ok = warp_wait(&tr[g], steps & 1, a);
    ++steps;
    return ok;
  };
  auto release = [&](int s) {  // this warp has read the tile
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  };
  const float sc = a.do_scale ? a.scale : 1.0f;
  for (int k = g;; k += G) {
    const int s = k % NT;
    if (!warp_wait(&full[full_idx<NT, G>(k)], full_par<NT, G>(k), a)) break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    unsigned char* t = base + (size_t)s * K::TILE;
    const long long gg = d.grid;
    const int i0 = P * d.idx;  // first plane (or row ky) of the item
    float2 v[H];
    // The item's passes share one DFT in a loop (one copy of its code for the
    // instruction cache): forward 0 plane x, 1 plane y, 2 z, 3 Nyquist;
    // inverse 0 z, 1 plane y, 2 plane x.
    int pass;
    if constexpr (DIR < 0) pass = d.phase == 0 ? 0 : (d.idx < IPP ? 2 : 3);
    else pass = d.phase;
    // z items: column 0 of row i0 + r in the tile row
    const int off = P == 1 ? 8 * (i0 & 1) : 8 * HC * r;
    // the forward Nyquist item uses the threads of row 0 only
    const bool idle = DIR < 0 && pass == 3 && r != 0;
    bool fail = false;
    if constexpr (DIR > 0) {
      if (pass == 0) {
        // rows (kz, ky = i0 + rs) of the input: columns 0 and H -> their
        // Hermitian parts, packed into column 0 (thread (rs, kz = gt % N))
        const int kz = gt % N, rs = gt / N;
        const int offs = P == 1 ? off : 8 * HC * rs;
        unsigned char* rk = t + kz * K::PITCH + offs;
        const float2 T0 = *reinterpret_cast<const float2*>(rk);
        const float2 Th = *reinterpret_cast<const float2*>(rk + 8 * H);
        // mirror row (-kz, -ky): its columns 0 and h from the mirror boxes
        const int mz = (N - kz) % N, mo = 16 * mz + 8 * (((N - i0 - rs) % N) & 1);
        const float2 M0 = *reinterpret_cast<const float2*>(t + K::MAIN + 2 * rs * N * 16 + mo);
        const float2 Mh =
            *reinterpret_cast<const float2*>(t + K::MAIN + (2 * rs + 1) * N * 16 + mo);
        const float2 A = make_float2(0.5f * (T0.x + M0.x), 0.5f * (T0.y - M0.y));
        const float2 B = make_float2(0.5f * (Th.x + Mh.x), 0.5f * (Th.y - Mh.y));
        *reinterpret_cast<float2*>(rk) = make_float2(A.x - B.y, A.y + B.x);  // A + i B
        if (!group_sync()) break;
      }
    }
#pragma unroll 1
    for (;;) {
      // ---------------------------------------------------------- in
      if constexpr (DIR < 0) {
        if (pass == 0) {
          // x: row gt, 16-byte chunks of reals = pairs of complex z[m]
#pragma unroll
          for (int j = 0; j < H / 2; ++j) {
            const float4 q = *reinterpret_cast<const float4*>(t + swz<N>(gt, j));
            v[2 * j] = make_float2(q.x, q.y);
            v[2 * j + 1] = make_float2(q.z, q.w);
          }
        } else if (pass == 1) {
          // y: column c of plane r (chunk c/2 of its rows, half c & 1)
          const unsigned char* tc = t + (c & 1) * 8;
          auto at = [&](int y) {
            return reinterpret_cast<const float2*>(tc + swz<N>(r * N + y, c >> 1));
          };
          if (h == 0) load_dif<N, DIR, 0>(at, v);
          else load_dif<N, DIR, 1>(at, v);
          release(s);
        } else if (pass == 2) {
          // z: column c of the rows (z, ky = i0 + r)
          load_dif_rows<N, DIR, K::PITCH>(t, off + 8 * c, h, v);
          release(s);
        } else {
          // Nyquist column: pencil p = c of the workspace tile (dense rows z)
          if (!idle) load_dif_rows<N, DIR, H * 8>(t, 8 * c, h, v);
          release(s);
        }
      } else {
        if (pass == 0) {
          // z: column c of the rows (kz, ky = i0 + r)
          load_dif_rows<N, DIR, K::PITCH>(t, off + 8 * c, h, v);
          release(s);
        } else if (pass == 1) {
          // y: column c of plane i0 + r (dense rows of H complex)
          load_dif_rows<N, DIR, H * 8>(t + r * N * H * 8, 8 * c, h, v);
          if (!group_sync()) {  // every column read before any row is written
            fail = true;
            break;
          }
        } else {
          // x: row gt (half spectrum, X[0] + i X[h] in column 0)
          const unsigned char* row = t + gt * K::XP;
#pragma unroll
          for (int j = 0; j < H / 2; ++j) {
            const float4 q = *reinterpret_cast<const float4*>(row + 16 * j);
            v[2 * j] = make_float2(q.x, q.y);
            v[2 * j + 1] = make_float2(q.z, q.w);
          }
          real_merge<H, DIR>(v);
        }
      }
      DFT<H, DIR>::run(v);
      // --------------------------------------------------------- out
      if constexpr (DIR < 0) {
        float2* og = const_cast<float2*>(a.out) + gg * N * N * HC;  // half spectra of grid g
        if (pass == 0) {
          real_split<H, DIR>(v);
#pragma unroll
          for (int j = 0; j < H / 2; ++j)
            *reinterpret_cast<float4*>(t + swz<N>(gt, j)) =
                make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
          if (!group_sync()) {
            fail = true;
            break;
          }
          pass = 1;
          continue;
        }
        if (pass == 1) {
          // outputs ky = 2k + h straight to out (kept in L2).  Column 0 (C =
          // Y0 + i Yh, each Hermitian) is separated in the warp that holds
          // it: ky and -ky have the same parity, so lane 0's outputs are
          // every ky of that parity; they go to the warp's scratch, and each
          // lane separates some of them: Y0 to column 0, Yh (real at ky = 0
          // and h) to the Nyquist workspace.
          const int z = i0 + r;
          float2* dst = og + (long long)z * N * HC;
          const unsigned long long keep = rowk::policy_evict_last();
#pragma unroll
          for (int kk = 0; kk < H; ++kk)
            if (c != 0) st_keep(dst + (2 * kk + h) * HC + c, v[kk], keep);
          if (c < 32) {  // the warp holding column 0 (of this plane and half)
            float2* scr = scratch + ((g * P + r) * 2 + h) * H;
            if (c == 0) {
#pragma unroll
              for (int kk = 0; kk < H; ++kk) scr[kk] = v[kk];
            }
            __syncwarp();
            float2* nq = a.aux + (gg * N + z) * H;
#pragma unroll
            for (int kk = c; kk < H; kk += 32) {
              const int ky = 2 * kk + h;
              const float2 cc = scr[kk], m = scr[h == 0 ? (H - kk) % H : H - 1 - kk];
              const float2 A = make_float2(0.5f * (cc.x + m.x), 0.5f * (cc.y - m.y));  // (C + conj M) / 2
              const float2 B = make_float2(0.5f * (cc.y + m.y), 0.5f * (m.x - cc.x));  // (C - conj M) / 2i
              st_keep(dst + ky * HC, A, keep);
              if (ky == 0) st_keep_f(&nq[0].x, B.x, keep);
              else if (ky == H) st_keep_f(&nq[0].y, B.x, keep);
              else if (ky < H) st_keep(nq + ky, B, keep);
            }
          }
        } else if (pass == 2) {
          // outputs kz = 2k + h, scaled
          float2* dst = og + (long long)(i0 + r) * HC + c;
#pragma unroll
          for (int kk = 0; kk < H; ++kk)
            st_stream(dst + (long long)(2 * kk + h) * N * HC, cscale(v[kk], sc));
        } else {
          // Nyquist pencils: ky = c and its mirror -ky (conjugate, at -kz);
          // pencil 0 packs ky = 0 and ky = h, separated like column 0 above.
          // Idle lanes (rows r > 0 of the item, whole warps) store nothing.
          if (!idle) {
#pragma unroll
            for (int kk = 0; kk < H; ++kk) {
              const int kz = 2 * kk + h, mz = (N - kz) % N;
              const float2 o = cscale(v[kk], sc);
              if (c != 0) {
                st_stream(og + ((long long)kz * N + c) * HC + H, o);
                st_stream(og + ((long long)mz * N + (N - c)) * HC + H, conjf2(o));
              }
            }
          }
          if (c < 32) {
            float2* scr = scratch + ((g * P + r) * 2 + h) * H;
            if (!idle && c == 0) {
#pragma unroll
              for (int kk = 0; kk < H; ++kk) scr[kk] = v[kk];
            }
            __syncwarp();
            if (!idle) {
              for (int kk = c; kk < H; kk += 32) {
                const int kz = 2 * kk + h;
                const float2 cc = scr[kk], m = scr[h == 0 ? (H - kk) % H : H - 1 - kk];
                const float2 A = make_float2(0.5f * (cc.x + m.x), 0.5f * (cc.y - m.y));
                const float2 B = make_float2(0.5f * (cc.y + m.y), 0.5f * (m.x - cc.x));
                st_stream(og + ((long long)kz * N) * HC + H, cscale(A, sc));
                st_stream(og + ((long long)kz * N + H) * HC + H, cscale(B, sc));
              }
            }
          }
        }
      } else {
        if (pass == 0) {
          // outputs z = 2k + h into the intermediate (kept in L2)
          float2* dst =
              const_cast<float2*>(a.out) + gg * N * N * H + (long long)(i0 + r) * H + c;
          const unsigned long long keep = rowk::policy_evict_last();
#pragma unroll
          for (int kk = 0; kk < H; ++kk)
            st_keep(dst + (long long)(2 * kk + h) * N * H, v[kk], keep);
        } else if (pass == 1) {
          // back into the tile as row y = 2k + h of plane r (padded rows)
#pragma unroll
          for (int kk = 0; kk < H; ++kk)
            *reinterpret_cast<float2*>(t + (r * N + 2 * kk + h) * K::XP + 8 * c) = v[kk];
          if (!group_sync()) {
            fail = true;
            break;
          }
          pass = 2;
          continue;
        } else {
          // n reals of row gt, scaled, back to the row and out
          unsigned char* row = t + gt * K::XP;
#pragma unroll
          for (int j = 0; j < H / 2; ++j)
            *reinterpret_cast<float4*>(row + 16 * j) = make_float4(
                sc * v[2 * j].x, sc * v[2 * j].y, sc * v[2 * j + 1].x, sc * v[2 * j + 1].y);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          float* og = reinterpret_cast<float*>(const_cast<float2*>(a.out)) + gg * N * N * N;
          bulk_store_row(og + ((long long)i0 * N + gt) * N, saddr(row), N * 4);
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          release(s);
        }
      }
      break;
    }
    if (fail) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[k % K::DQ]);  // the stores are issued, for the publisher
  }
  // every bulk store of this thread has landed before the block exits
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Tensor map of `dims` floats (innermost first) with byte strides of the
// outer dims, box `box`, no element striding.
inline bool encode(CUtensorMap* m, const void* base, const cuuint64_t dims[3],
                   const cuuint64_t strides[2], const cuuint32_t box[3], bool swizzle) {
  auto fn = rowk::encode_fn();
  if (!fn) return false;
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
            const_cast<cuuint32_t*>(box), estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Half spectra of `grids` grids as row pairs: [n * grids][n/2][2 (n/2 + 1)
// complex] floats.
inline bool encode_pairs(CUtensorMap* m, const void* base, int n, int grids, unsigned box_x,
                         unsigned box_y = 1) {
  const cuuint64_t hc = n / 2 + 1;
  const cuuint64_t dims[3] = {4 * hc, (cuuint64_t)n / 2, (cuuint64_t)n * grids};
  const cuuint64_t strides[2] = {16 * hc, (cuuint64_t)n * hc * 8};
  const cuuint32_t box[3] = {box_x, box_y, (cuuint32_t)n};
  return encode(m, base, dims, strides, box, false);
}

template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off) return cudaErrorInvalidValue;
  CUtensorMap m0, m1;
  using K = Cfg<N>;
  // z items: P = 1 one row of its pair (box PITCH/4 floats), else P/2 pairs
  const unsigned zx = K::P == 1 ? K::PITCH / 4 : 4 * K::HC, zy = K::P == 1 ? 1 : K::P / 2;
  if (DIR < 0) {
    // real planes: rows of N floats, boxes of 32 floats x N rows x P planes
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N * a.ngrids};
    const cuuint64_t strides[2] = {(cuuint64_t)N * 4, (cuuint64_t)N * N * 4};
    const cuuint32_t box[3] = {32, (cuuint32_t)N, (cuuint32_t)K::P};
    if (!encode_pairs(&m0, a.out, N, a.ngrids, zx, zy) ||
        !encode(&m1, a.in, dims, strides, box, true))
      return cudaErrorInvalidValue;
  } else {
    if (!encode_pairs(&m0, a.in, N, a.ngrids, zx, zy) || !encode_pairs(&m1, a.in, N, a.ngrids, 4))
      return cudaErrorInvalidValue;
  }
  rgrid_fft3d_kernel<N, DIR><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a, m0, m1);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = (const void*)&rgrid_fft3d_kernel<N, DIR>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.sizes[0] = N;
  k.nsizes = 1;
  // schedule lag in items per block: the tiles and the tickets held ahead;
  // twice that forward, whose plane items take longer than its z items, so
  // that the z items of a grid rarely wait for its planes (measured)
  k.items_in_flight = (Cfg<N>::NTILE + 3) * (DIR < 0 ? 2 : 1);
  // tickets per schedule block: n/P items, plus (forward) the Nyquist item
  // of a z block and an empty ticket of a plane block
  k.phase_items = Cfg<N>::IPP + (DIR < 0 ? 1 : 0);
  return k;
}

}  // namespace rg
}  // namespace fft3d
