// Double-buffered persistent 3D FFT kernel: the plane/slab items of the
// persistent kernel, with the next item's data copied into a second shared-
// memory tile (cp.async) while the current one is transformed, so the load
// latency of an item overlaps the arithmetic of the previous one.
//
// A block takes the ticket of its next item as soon as it starts the current
// one.  A plane item's rows are always ready; a slab item's are ready once
// every plane item of its grid has signalled.  If they are not ready yet the
// copy is issued after the current item, behind the usual bounded wait.  A
// ticket holder still waits only on smaller tickets (held by running
// blocks), so the argument against deadlock of the persistent kernel holds.
#pragma once

#include "persistent.cuh"

namespace fft3d {
namespace pref {

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// Issue the copies of item (blk, i) into `tile`: a plane with row pitch
// N + 1 (8-byte copies), or a slab as [z][x] with pitch N (16-byte copies).
template <int N, int T>
__device__ __forceinline__ void stage(const FusedArgs& a, const SchedBlock& blk, int i,
                                      float2* tile) {
  constexpr long long NN = (long long)N * N;
  constexpr int P = plane_pitch<N>();
  const float2* gin;
  float2* gout;
  grid_ptrs(a, blk.grid, N, gin, gout);
  if (blk.phase == 0) {
    const float2* src = gin + (long long)i * NN;
    for (int idx = threadIdx.x; idx < N * N; idx += T)
      cp_async8(tile + (idx / N) * P + idx % N, src + idx);
  } else {
    const float2* src = gout + (long long)i * N;
    for (int idx = threadIdx.x; idx < N * N / 2; idx += T) {
      const int z = (2 * idx) / N, x = (2 * idx) % N;
      cp_async16(tile + z * N + x, src + z * NN + x);
    }
  }
}

template <int T, int DIR, int N>
__global__ void __launch_bounds__(T) prefetch_fft3d_kernel(const FusedArgs a) {
  constexpr int TILE = tile_elems<N>();
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int s_item, s_blk, s_ready;
  float2* tw = smem;
  float2* const tile0 = smem + N;  // tile b at tile0 + b * TILE
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += T) tw[i] = a.twiddles[i];

  // thread 0: next ticket; `block` = wait for a slab's planes (bounded).
  auto take = [&](bool block) {
    int item = -1, b = -1, ready = 0;
    if (*(volatile unsigned*)a.status == kStatusOk) item = (int)atomicAdd(a.work, 1u);
    if (item >= a.total_items) item = -1;
    if (item >= 0) {
      b = find_block(a.blocks, a.nblocks, item);
      const SchedBlock blk = a.blocks[b];
      if (blk.phase == 0) {
        ready = 1;
      } else if (block) {
        ready = bounded_wait_geq(a.work + 1 + blk.grid, (unsigned)N, a.status, a.timeout_ns);
        if (!ready) item = -1;
      } else {
        ready = ld_acquire(a.work + 1 + blk.grid) >= (unsigned)N;
      }
    }
    s_item = item;
    s_blk = b;
    s_ready = ready;
  };

  if (tid == 0) take(true);
  __syncthreads();
  int cur = s_item, cb = s_blk, buf = 0;
  if (cur >= 0) {
    const SchedBlock blk = a.blocks[cb];
    stage<N, T>(a, blk, cur - blk.start, tile0);
  }
  cp_commit();
  while (cur >= 0) {
    __syncthreads();  // everyone has read s_* of the previous round
    if (tid == 0) take(false);
    __syncthreads();
    const int nxt = s_item, nb = s_blk, ready = s_ready;
    if (nxt >= 0 && ready) {
      const SchedBlock blk = a.blocks[nb];
      stage<N, T>(a, blk, nxt - blk.start, tile0 + (buf ^ 1) * TILE);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();  // the current tile is complete and visible
    const SchedBlock blk = a.blocks[cb];
    const int i = cur - blk.start;
    const float2* gin;
    float2* gout;
    grid_ptrs(a, blk.grid, N, gin, gout);
    if (blk.phase == 0) {
      const long long o = (long long)i * N * N;
      plane_item<N, T, DIR, 0, true>(nullptr, gout + o, tile0 + buf * TILE, tw, nullptr);
    } else {
      slab_item<N, T, DIR, 0, true>(nullptr, gout + (long long)i * N, tile0 + buf * TILE, tw, nullptr,
                                    a.scale, a.do_scale);
    }
    __syncthreads();  // stores issued, tile free
    if (blk.phase == 0 && tid == 0) {
      __threadfence();
      atomicAdd(a.work + 1 + blk.grid, 1u);
    }
    int next = nxt, next_b = nb;
    if (nxt >= 0 && !ready) {
      // the slab's planes were not done yet: wait for them now, then copy
      if (tid == 0) {
        const SchedBlock nblk = a.blocks[nb];
        s_ready = bounded_wait_geq(a.work + 1 + nblk.grid, (unsigned)N, a.status, a.timeout_ns);
      }
      __syncthreads();
      if (!s_ready) {
        next = -1;
      } else {
        const SchedBlock nblk = a.blocks[nb];
        stage<N, T>(a, nblk, nxt - nblk.start, tile0 + (buf ^ 1) * TILE);
      }
      cp_commit();
    }
    cur = next;
    cb = next_b;
    buf ^= 1;
  }
  cp_wait<0>();
}

template <int T, int DIR, int N>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  prefetch_fft3d_kernel<T, DIR, N>
      <<<grid, T, sizeof(float2) * (size_t)(N + 2 * tile_elems<N>()), stream>>>(a);
  return cudaGetLastError();
}

template <int T, int DIR, int N>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<T, DIR, N>;
  k.func = (const void*)&prefetch_fft3d_kernel<T, DIR, N>;
  k.threads = T;
  k.smem = sizeof(float2) * (size_t)(N + 2 * tile_elems<N>());
  k.twiddle_entries = N;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.items_in_flight = 2;
  return k;
}

}  // namespace pref
}  // namespace fft3d
