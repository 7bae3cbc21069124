// Plane-wave Hartree energy on top of the 3D FFT: the use the paper
// accelerates (the 3D FFT on the critical path of plane-wave DFT in AIMD,
// section "Introduction"; CP2K's Gaussian and plane-wave method, section
// "Results").  The paper gives no formulas for this part; these are the
// standard ones for a periodic cubic cell of side L and volume Omega = L^3
// sampled on an n^3 grid:
//
//   rho_hat(G) = F(rho)(G) / n^3          (F: forward transform of Eq. 1)
//   E_H = (Omega/2) sum_{G != 0} 4 pi |rho_hat(G)|^2 / |G|^2
//   G = (2 pi / L) m,  m_d = k_d for k_d < n/2 else k_d - n
//   dE_H / drho_j = (Omega / n^6) Re[ F^H (K F(rho)) ]_j,  K = 4 pi / |G|^2
//
// so that with s = Omega 4 pi / (n^6 (2 pi / L)^2):
//   E_H = (s/2) sum_{m != 0} |F(rho)(m)|^2 / |m|^2
//   seed(m) = dL/dE_H * s * F(rho)(m) / |m|^2,   dL/drho = Re F^H(seed).
//
// The energy is accumulated in FP64 (the only FP64 on the GPU) with a fixed
// reduction order, so repeated calls give bit-identical results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "fft3d.h"
#include "internal.h"

namespace fft3d {
namespace {

constexpr int kRedThreads = 256;

__host__ __device__ inline int energy_blocks(long long npts) {
  long long b = (npts + kRedThreads * 8 - 1) / (kRedThreads * 8);
  return (int)(b < 1 ? 1 : (b > 512 ? 512 : b));
}

__device__ __forceinline__ int signed_index(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// 1 / x by the hardware's approximate reciprocal (within 1 ulp by the PTX
// ISA's bound; the callers' x = |m|^2 is a positive integer below 2^24,
// exact in FP32).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// n / d for n < 2^32 with the multiplier and shift of make_fastdiv
// (Granlund and Montgomery, 1994).
__device__ __forceinline__ unsigned udiv(unsigned x, FastDiv d) {
  return (unsigned)(((unsigned long long)__umulhi(x, d.mul) + x) >> d.shift);
}

// One row of blocks per grid (blockIdx.y).  partials: [batch][gridDim.x];
// counters: [batch], zero on entry, left at zero by the last block, whose
// threads sum the grid's partials together (one thread reading them one
// after another took 38 us for the 512 partials of one 128^3 grid).
// The spectrum is read as a flat array, U points per thread per step at a
// grid stride (every warp load 256 consecutive bytes); a point's (kz, ky,
// kx) come from its index by multiply-shift divisions by the row length
// and by n.  (Rows of n/2 + 1 points taken one warp at a time left a
// third pass over each row with one lane of 32 busy: 0.41 of the HBM
// bandwidth at 32 grids of 128^3.)  Each term |F(m)|^2 w / |m|^2 is
// formed in FP32 (the approximate reciprocal of |m|^2: one instruction
// where the correctly rounded one takes several, and the loop is nearly
// as much instruction work as memory traffic; a term's relative error
// stays below 6 2^-24, against the FP32 rounding the spectrum already
// carries) and a thread's U terms of a step are summed in FP32, then
// accumulated in FP64: FP64 work is a few operations per hundred points,
// since FP64 runs at a small fraction of the FP32 rate on this GPU (the
// per-point FP64 form ran at 0.39 TB/s).
template <bool HALF>
__global__ void __launch_bounds__(kRedThreads) hartree_energy_kernel(
    const float2* __restrict__ f, int n, long long npts, double half_s,
    double* __restrict__ partials, unsigned* __restrict__ counters, double* __restrict__ energy,
    FastDiv div_h, FastDiv div_n) {
  const int b = blockIdx.y;
  const float2* fb = f + (long long)b * npts;
  constexpr int W = kRedThreads / 32, U = 8;  // points per thread per step
  const int h = HALF ? n / 2 + 1 : n;
  const unsigned np = (unsigned)npts, stride = gridDim.x * kRedThreads;
  double acc = 0.0;
  for (unsigned i0 = blockIdx.x * kRedThreads + threadIdx.x; i0 < np; i0 += U * stride) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned i = i0 + u * stride;
      v[u] = i < np ? __ldcs(fb + i) : make_float2(0.0f, 0.0f);
    }
    float part = 0.0f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned i = i0 + u * stride;
      const unsigned row = udiv(i, div_h), kz = udiv(row, div_n);
      const int kx = (int)(i - row * h), ky = (int)(row - kz * n);
      const int mx = signed_index(kx, n), my = signed_index(ky, n), mz = signed_index((int)kz, n);
      const int m2 = mx * mx + my * my + mz * mz;
      const float w = HALF && kx != 0 && 2 * kx != n ? 2.0f : 1.0f;
      if (i < np && m2 > 0)
        part = fmaf(fmaf(v[u].x, v[u].x, v[u].y * v[u].y), w * rcp_approx((float)m2), part);
    }
    acc += (double)part;
  }
  acc = warp_sum(acc);
  __shared__ double warp_part[W];
  __shared__ int is_last;
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += warp_part[w];
    partials[(long long)b * gridDim.x + blockIdx.x] = s;
    __threadfence();
    is_last = atomicAdd(&counters[b], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last) {  // (block-uniform) the grid's partials, summed by the whole block
    __threadfence();
    double s = 0.0;
    const volatile double* p = partials + (long long)b * gridDim.x;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) s += p[j];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = s;  // (read above before the barrier)
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < W; ++w) t += warp_part[w];
      energy[b] = half_s * t;
      counters[b] = 0u;
    }
  }
}

// The seed: the spectrum as a flat array, U points per thread per step at a
// grid stride (coalesced loads and stores), indices and reciprocal as in
// the energy kernel.
template <bool HALF>
__global__ void __launch_bounds__(kRedThreads) hartree_seed_kernel(
    const float2* __restrict__ f, int n, long long npts, double s,
    const double* __restrict__ grad_e, float2* __restrict__ seed, FastDiv div_h, FastDiv div_n) {
  const int b = blockIdx.y;
  const float scale = (float)(s * grad_e[b]);
  const float2* fb = f + (long long)b * npts;
  float2* sb = seed + (long long)b * npts;
  constexpr int U = 4;  // points per thread per step
  const int h = HALF ? n / 2 + 1 : n;
  const unsigned np = (unsigned)npts, stride = gridDim.x * kRedThreads;
  for (unsigned i0 = blockIdx.x * kRedThreads + threadIdx.x; i0 < np; i0 += U * stride) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned i = i0 + u * stride;
      v[u] = i < np ? __ldcs(fb + i) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned i = i0 + u * stride;
      if (i >= np) continue;
      const unsigned row = udiv(i, div_h), kz = udiv(row, div_n);
      const int kx = (int)(i - row * h), ky = (int)(row - kz * n);
      const int mx = signed_index(kx, n), my = signed_index(ky, n), mz = signed_index((int)kz, n);
      const int m2 = mx * mx + my * my + mz * mz;
      float2 o = make_float2(0.0f, 0.0f);
      if (m2 != 0) {
        const float w = scale * rcp_approx((float)m2);
        o = make_float2(v[u].x * w, v[u].y * w);
      }
      __stcs(sb + i, o);
    }
  }
}

// Blocks of the energy (SEED false) or seed kernel the device holds at
// once (one wave), found once per process; 2048 if the runtime cannot say.
template <bool HALF, bool SEED>
int resident_blocks() {
  static const int r = [] {
    const void* fn = SEED ? reinterpret_cast<const void*>(hartree_seed_kernel<HALF>)
                          : reinterpret_cast<const void*>(hartree_energy_kernel<HALF>);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRedThreads, 0) != cudaSuccess ||
        sms < 1 || per_sm < 1) {
      cudaGetLastError();
      return 2048;
    }
    return sms * per_sm;
  }();
  return r;
}

__global__ void real_to_complex_kernel(const float* __restrict__ re, float2* __restrict__ out,
                                       long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2(re[i], 0.0f);
}

__global__ void complex_to_real_kernel(const float2* __restrict__ in, float* __restrict__ re,
                                       long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    re[i] = in[i].x;
}

int grid_for(long long count, int threads) {
  long long b = (count + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

bool valid_grid(int n, int batch, double L) {
  return n >= 2 && n <= 1024 && batch >= 1 && batch <= 65535 && L > 0.0 && std::isfinite(L);
}

// s = Omega 4 pi / (n^6 (2 pi / L)^2)
double hartree_s(int n, double L) {
  const double n3 = (double)n * n * n, g = 2.0 * 3.14159265358979323846 / L;
  return L * L * L * 4.0 * 3.14159265358979323846 / (n3 * n3 * g * g);
}

}  // namespace
}  // namespace fft3d

using namespace fft3d;

extern "C" {

size_t fft3d_hartree_workspace_bytes(int n, int batch) {
  if (n < 2 || batch < 1) return 0;
  const long long npts = (long long)n * n * n;
  const size_t partials = sizeof(double) * (size_t)batch * (size_t)energy_blocks(npts);
  return ((partials + 255) & ~size_t(255)) + sizeof(unsigned) * (size_t)batch;
}

}  // extern "C"

namespace {

template <bool HALF>
int energy_impl(const void* rhohat, int n, int batch, double L, double* energy, void* workspace,
                size_t workspace_bytes, void* stream) {
  if (!rhohat || !energy || !workspace) return FFT3D_ERR_NULL_PTR;
  if (!valid_grid(n, batch, L) || (HALF && (n & 1))) return FFT3D_ERR_INVALID_ARG;
  if (workspace_bytes < fft3d_hartree_workspace_bytes(n, batch)) return FFT3D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(rhohat) & 7u || reinterpret_cast<uintptr_t>(workspace) & 7u)
    return FFT3D_ERR_MISALIGNED;
  const long long npts = (long long)n * n * (HALF ? n / 2 + 1 : n);
  // one wave of resident blocks in all (each ends with a fenced counter
  // update, so many short blocks cost more than the points they read; 2048
  // blocks, 2.7 waves at 128^3 x 32, left the last wave a third empty), at
  // most the workspace's energy_blocks per grid
  const int blocks =
      std::max(1, std::min(energy_blocks(npts), resident_blocks<HALF, false>() / batch));
  const size_t partial_bytes = sizeof(double) * (size_t)batch * (size_t)energy_blocks(npts);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  unsigned* counters = reinterpret_cast<unsigned*>(ws + ((partial_bytes + 255) & ~size_t(255)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(counters, 0, sizeof(unsigned) * (size_t)batch, s) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  hartree_energy_kernel<HALF><<<dim3(blocks, batch), kRedThreads, 0, s>>>(
      static_cast<const float2*>(rhohat), n, npts, 0.5 * hartree_s(n, L),
      reinterpret_cast<double*>(ws), counters, energy,
      make_fastdiv((unsigned)(HALF ? n / 2 + 1 : n)), make_fastdiv((unsigned)n));
  if (cudaGetLastError() != cudaSuccess) return FFT3D_ERR_CUDA;
  return FFT3D_SUCCESS;
}

template <bool HALF>
int seed_impl(const void* rhohat, int n, int batch, double L, const double* grad_energy,
              void* seed, void* stream) {
  if (!rhohat || !grad_energy || !seed) return FFT3D_ERR_NULL_PTR;
  if (!valid_grid(n, batch, L) || (HALF && (n & 1))) return FFT3D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(rhohat) & 7u || reinterpret_cast<uintptr_t>(seed) & 7u)
    return FFT3D_ERR_MISALIGNED;
  const long long npts = (long long)n * n * (HALF ? n / 2 + 1 : n);
  // one wave of resident blocks in all, no more than one step of U = 4
  // points per thread covers
  const long long per_block = (long long)kRedThreads * 4;
  const int bx = (int)std::max(1LL, std::min((long long)resident_blocks<HALF, true>() / batch,
                                            (npts + per_block - 1) / per_block));
  hartree_seed_kernel<HALF><<<dim3(bx, batch), kRedThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float2*>(rhohat), n, npts, hartree_s(n, L), grad_energy,
      static_cast<float2*>(seed), make_fastdiv((unsigned)(HALF ? n / 2 + 1 : n)),
      make_fastdiv((unsigned)n));
  if (cudaGetLastError() != cudaSuccess) return FFT3D_ERR_CUDA;
  return FFT3D_SUCCESS;
}

}  // namespace

extern "C" {

int fft3d_hartree_energy(const void* rhohat, int n, int batch, double L, double* energy,
                         void* workspace, size_t workspace_bytes, void* stream) {
  return energy_impl<false>(rhohat, n, batch, L, energy, workspace, workspace_bytes, stream);
}

int fft3d_hartree_energy_half(const void* rhohat_half, int n, int batch, double L, double* energy,
                              void* workspace, size_t workspace_bytes, void* stream) {
  return energy_impl<true>(rhohat_half, n, batch, L, energy, workspace, workspace_bytes, stream);
}

int fft3d_hartree_seed(const void* rhohat, int n, int batch, double L, const double* grad_energy,
                       void* seed, void* stream) {
  return seed_impl<false>(rhohat, n, batch, L, grad_energy, seed, stream);
}

int fft3d_hartree_seed_half(const void* rhohat_half, int n, int batch, double L,
                            const double* grad_energy, void* seed_half, void* stream) {
  return seed_impl<true>(rhohat_half, n, batch, L, grad_energy, seed_half, stream);
}

int fft3d_real_to_complex(const float* re, void* out, int64_t count, void* stream) {
  if (!re || !out) return FFT3D_ERR_NULL_PTR;
  if (count < 0) return FFT3D_ERR_INVALID_ARG;
  if (count == 0) return FFT3D_SUCCESS;
  real_to_complex_kernel<<<grid_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      re, static_cast<float2*>(out), count);
  return cudaGetLastError() == cudaSuccess ? FFT3D_SUCCESS : FFT3D_ERR_CUDA;
}

int fft3d_complex_to_real(const void* in, float* re, int64_t count, void* stream) {
  if (!in || !re) return FFT3D_ERR_NULL_PTR;
  if (count < 0) return FFT3D_ERR_INVALID_ARG;
  if (count == 0) return FFT3D_SUCCESS;
  complex_to_real_kernel<<<grid_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float2*>(in), re, count);
  return cudaGetLastError() == cudaSuccess ? FFT3D_SUCCESS : FFT3D_ERR_CUDA;
}

}  // extern "C"
