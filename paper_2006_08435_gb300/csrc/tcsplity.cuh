// Split-precision kernel for 128^3 grids on the tcgen05 tensor cores: the
// work items, tiles, producer and signaller of the split-y kernel
// (splity.cuh), with every 64-point DFT of a thread (the x and z halves of
// the thread-pair 128-point transforms, and the 64-point y DFT of a column)
// run as the tensor-core pass of tcgen.cuh: radix-4 in registers, the
// radix-16 step as tcgen05.mma products with split half-precision operands
// in tensor memory.  The 128 threads of a compute group are the 128 rows of
// every product; the pair radix-2 steps and the W_128 twiddles stay in FP32.
#pragma once

#include "splity.cuh"
#include "tcgen.cuh"

namespace fft3d {
namespace tsy {

using mb::mbar_arrive;
using mb::mbar_init;
using mb::saddr;
using mb::warp_wait;
using rowk::Desc;
using rowk::policy_evict_last;
using sy::Cfg;
using sy::hoff;
using sy::lds2;
using sy::soff;
using sy::sts2;
using tg::group_and;
using tg::named_bar;

template <int N>
constexpr size_t kSmem = Cfg<N>::smem + 128 + tg::kBBytes + 2 * sizeof(unsigned long long) + 16;

template <int N, int DIR, int PREC>
__global__ void __launch_bounds__(Cfg<N>::T, 1)
    tcsplity_fft3d_kernel(const FusedArgs a, const __grid_constant__ CUtensorMap tin,
                          const __grid_constant__ CUtensorMap tout) {
  using K = Cfg<N>;
  static_assert(K::GT == 128, "one product row per thread of a 128-thread group");
  constexpr int NT = K::NTILE, H = K::H;
  constexpr long long NN = (long long)N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const uint32_t tiles = saddr(base);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(base + (size_t)NT * K::TILE);
  unsigned long long* empty = full + K::NFULL;
  unsigned long long* freed = empty + NT;
  unsigned long long* tr = freed + NT;
  Desc* desc = reinterpret_cast<Desc*>(tr + K::GROUPS);
  unsigned short* sched = reinterpret_cast<unsigned short*>(desc + NT);
  unsigned char* bsm_p = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(sched + K::SCHED) + 127) & ~(uintptr_t)127);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(bsm_p + tg::kBBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int w = threadIdx.x >> 5;
  if (a.nblocks <= K::SCHED)
    for (int b = threadIdx.x; b < a.nblocks; b += K::T)
      sched[b] = (unsigned short)(a.blocks[b].grid * 2 + a.blocks[b].phase);
  for (int i = threadIdx.x; i < tg::kBBytes / 16; i += K::T)
    reinterpret_cast<uint4*>(bsm_p)[i] = reinterpret_cast<const uint4*>(a.mma_frag)[i];
  if (threadIdx.x == 0) {
    for (int i = 0; i < K::NFULL; ++i) mbar_init(&full[i], 1);
    for (int s = 0; s < NT; ++s) {
      mbar_init(&empty[s], K::GW);
      mbar_init(&freed[s], 1);
    }
    for (int g = 0; g < K::GROUPS; ++g) mbar_init(&tr[g], K::GW);
    mbar_init(&mbar[0], 4);  // one commit per issuing warp of the group
    mbar_init(&mbar[1], 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 4) {  // the first compute warp owns the tensor-memory allocation
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "n"(tg::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B operands, for the tensor cores
  tg::tc_fence_before();
  __syncthreads();
  tg::tc_fence_after();

  if (w < 4) {  // warpgroup 0: control
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(K::REG_CTRL));
    if (w == 0) sy::producer<N, false>(a, &tin, &tout, tiles, full, freed, desc, sched);
    if (w == 1) sy::signaller<N>(a, full, empty, freed, desc);
    return;
  }
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(K::REG_COMP));

  // compute group g (warpgroup g + 1), thread gt of 128: product row gt
  const int g = (w - 4) / K::GW, gt = threadIdx.x - 128 - g * K::GT, lane = threadIdx.x & 31;
  tg::Pass P;
  P.bsm = saddr(bsm_p);
  P.col = *tslot + (uint32_t)(256 * g);
  P.lanes = (uint32_t)(32 * (gt >> 5)) << 16;
  P.bar = &mbar[g];
  P.g = g;
  P.gt = gt;
  unsigned phase = 0;  // completed product batches of this group
  // the 64-point DFT of v in place (natural order), on the tensor cores
  auto dft64 = [&](float2(&v)[H]) -> bool {
    return tg::pass<DIR, PREC>(v, P, phase, a, 1.0f, [&](int kp, int k2, float2 y0, float2 y1) {
      v[2 * kp + 4 * k2] = y0;
      v[2 * kp + 4 * k2 + 1] = y1;
    });
  };
  for (int k = g;; k += K::GROUPS) {
    const int s = k % NT;
    if (!group_and(1 + g, K::GT,
                   warp_wait(&full[rowk::full_idx<NT, K::GROUPS>(k)],
                             rowk::full_par<NT, K::GROUPS>(k), a)))
      break;
    const Desc d = desc[s];
    if (d.item < 0) break;
    const uint32_t t = tiles + (uint32_t)(s * K::TILE);
    const float2* gin;
    float2* gout;
    grid_ptrs(a, d.grid, N, gin, gout);
    float2 v[H];
    // The passes of the item (half-plane: x, then y; slab: z) share one copy
    // of the tensor-core pass (for the instruction cache); loads and stores
    // of each pass are chosen once per pass.
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
      if (!dft64(v)) {
        fail = true;
        break;
      }
      if (kind != 1) {
        // the pair radix-2 of x and z (one copy), in place: v[j] = X[j + 32 p],
        // v[32 + j] = X[j + 32 p + 64]
        const int p = kind == 0 ? (gt & 1) : (lane >> 4);
        sy::pair_radix2<DIR>(v, p, kind == 0 ? 1 : 16,
                             [&](int j, float2 a0, float2 a1, float2 b0, float2 b1) {
                               v[j] = a0;
                               v[j + 1] = a1;
                               v[32 + j] = b0;
                               v[33 + j] = b1;
                             });
      }
      if (kind == 0) {
        const int r = gt >> 1, p = gt & 1;
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
        named_bar(1 + g, K::GT);  // the x results are in the tile
      } else if (kind == 1) {
        const int par = d.idx & 1;
        if (par)  // times W_128^k2 (compile-time twiddles)
          static_for<1, H>([&](auto K2) {
            constexpr int k2 = decltype(K2)::value;
            v[k2] = twc<k2, 128, DIR>(v[k2]);
          });
        // in place: the partner half-plane's tile has landed (a group-wide
        // decision, so that no thread is left at a later barrier)
        if (a.in == a.out && !group_and(1 + g, K::GT, sy::partner_loaded<N>(k, d, full, a))) {
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
  // every compute warp is out of its loop: no product or tensor-memory read
  // is in flight
  tg::tc_fence_before();
  named_bar(3, 2 * K::GT);
  tg::tc_fence_after();
  if (w == 4)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot),
                 "n"(tg::kTmemCols));
}

// Uniform batches only (packed buffers, grids in plan order).
template <int N, int DIR, int PREC>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  if (a.in_ptrs || a.grid_map || a.grid_off || !a.mma_frag) return cudaErrorInvalidValue;
  CUtensorMap tin, tout;
  if (!rowk::encode_map(&tin, a.in, N, a.ngrids, 2 * (N / 2), 1, 2) ||
      !rowk::encode_map(&tout, a.out, N, a.ngrids, 1, N))
    return cudaErrorInvalidValue;
  tcsplity_fft3d_kernel<N, DIR, PREC><<<grid, Cfg<N>::T, kSmem<N>, stream>>>(a, tin, tout);
  return cudaGetLastError();
}

template <int N, int DIR, int PREC>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR, PREC>;
  k.func = (const void*)&tcsplity_fft3d_kernel<N, DIR, PREC>;
  k.threads = Cfg<N>::T;
  k.smem = kSmem<N>;
  k.twiddle_entries = N;  // (the B operands carry the 64-point twiddles; a table is uploaded anyway)
  k.tw_l1 = 8;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = Cfg<N>::NTILE + 4;
  k.phase_items = Cfg<N>::ITEMS;
  k.prec = PREC;
  k.umma_b = 1;
  return k;
}

}  // namespace tsy
}  // namespace fft3d
