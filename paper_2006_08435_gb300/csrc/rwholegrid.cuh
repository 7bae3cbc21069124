// Whole-grid real transforms for 16^3 and 32^3 grids: one block holds a
// grid in shared memory and runs the three passes of the paper's
// decomposition, one thread per row or pencil; blocks loop over the grids of
// the batch.  No block waits for another, so there are no work counters, no
// schedule and no memset before a launch.
//
// Forward (real grid -> half spectrum, kx = 0 .. h, h = n/2):
//   x: a thread takes row n z + y as h complex points
//      w[m] = r[2m] + i r[2m+1], whose h-point DFT W gives the half spectrum
//      of the row (E, O the transforms of the even and odd samples,
//      E[k] = (W[k] + conj W[h-k]) / 2, O[k] = (W[k] - conj W[h-k]) / 2i):
//        X[k] = E[k] + W_n^k O[k],  k = 0 .. h  (indices of W mod h);
//   y, z: n-point DFTs of the n (h + 1) columns (z, kx) and pencils
//      (ky, kx), the z results straight to global memory.
// Inverse (half spectrum -> real grid): Re of the inverse transform of the
// Hermitian extension.  That extension's real part is the inverse transform
// of its Hermitian part, which differs from the input only in the planes
// kx = 0 and h: there the z pass first takes (X(k) + conj X(-k)) / 2.
// Inverse n-point DFTs along z and y; then per row, from X[0 .. h] (with
// X[k + h] = conj X[h - k]),
//   V[k] = (X[k] + conj X[h-k]) + i W_n^-k (X[k] - conj X[h-k]),  k < h,
// is 2 E[k] + 2 i O[k], and its inverse h-point DFT is
// n (r[2m] + i r[2m+1]): the unnormalised inverse of the row.
//
// Shared memory: the spectrum at S[z * SZ + y * (h + 1) + kx] with
// SZ = n (h + 1) + 1 (a plane and one spare, SZ = 1 mod 16, so that every
// pass is free of bank conflicts: half-warps take 16 rows y of one z, 16
// planes z of one kx, or 16 consecutive pencils).  The forward transform
// reads its rows straight from global memory and the inverse its pencils;
// the inverse's real rows go out through shared memory at a pitch of n + 4
// floats (eight lanes' 16-byte row chunks fall on distinct banks), over the
// same bytes as the spectrum, with a block barrier between their uses, so
// that the stores are coalesced.
//
// 16^3: 256 threads (one per row), 20.5 KB, four or five blocks per
// multiprocessor.  32^3: 544 threads (one per y column and z pencil, two
// rows each for x), 144 KB, one block per multiprocessor; its first thread
// asks L2 for the block's next grid (bulk prefetch) as it starts a grid, so
// that the next grid's reads meet L2 rather than HBM.
#pragma once

#include "persistent.cuh"

namespace fft3d {
namespace rwg {

template <int N>
struct Cfg {
  static_assert(N == 16 || N == 32, "the whole-grid real kernels cover 16^3 and 32^3");
  static constexpr int H = N / 2, HC = H + 1;   // complex per row, bins per row
  static constexpr int COLS = N * HC;           // pencils along y and z (144, 544)
  static constexpr int T = N == 16 ? N * N : COLS;  // threads (256, 544)
  static constexpr int ROWS = N * N;
  static constexpr int RPT = (ROWS + T - 1) / T;    // rows per thread in the x pass (1, 2)
  static constexpr int SY = HC, SZ = N * HC + 1;
  static constexpr int RP = N + 4;              // real row pitch (floats)
  static constexpr int MINB_F = N == 16 ? 5 : 1;  // blocks per multiprocessor
  static constexpr int MINB_I = N == 16 ? 4 : 1;
  static constexpr bool PREFETCH = N >= 32;     // one block per SM: prefetch the next grid
  static constexpr size_t spec_bytes = sizeof(float2) * (size_t)N * SZ;
  static constexpr size_t real_bytes = sizeof(float) * (size_t)ROWS * RP;
  static constexpr size_t smem = spec_bytes > real_bytes ? spec_bytes : real_bytes;
  // the inverse's first x phase writes real rows ROWS - T .. ROWS - 1 while
  // spectrum rows 0 .. ROWS - T - 1 are still to be read: disjoint bytes
  static_assert(RPT <= 2, "at most two x phases");
  static_assert(RPT == 1 || (size_t)(ROWS - T) * RP * 4 >=
                                sizeof(float2) * ((size_t)((ROWS - T - 1) / N) * SZ +
                                                  (size_t)((ROWS - T - 1) % N) * SY + HC),
                "first-phase real rows clear of the unread spectrum rows");
};

// L2 prefetch of `bytes` (a multiple of 16) from 16-byte aligned `p`, in
// pieces of at most 32 KB.
__device__ __forceinline__ void prefetch_l2(const void* p, int bytes) {
  const char* c = static_cast<const char*>(p);
  for (int o = 0; o < bytes; o += 32768) {
    const int n = bytes - o < 32768 ? bytes - o : 32768;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + o), "r"(n) : "memory");
  }
}

// Forward kernel: a.in holds real grids of N^3 floats, a.out half spectra of
// N * N * (N/2 + 1) complex points.
template <int N>
__global__ void __launch_bounds__(Cfg<N>::T, Cfg<N>::MINB_F) rwholegrid_fwd_kernel(const FusedArgs a) {
  using K = Cfg<N>;
  constexpr int H = K::H, HC = K::HC;
  extern __shared__ __align__(16) float2 S[];
  const int t = threadIdx.x;
  const float sc = a.do_scale ? a.scale : 1.0f;
  for (int grid = blockIdx.x; grid < a.ngrids; grid += gridDim.x) {
    const float4* gin =
        reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.in) + (long long)grid * N * N * N);
    float2* gout = a.out + (long long)grid * N * N * HC;
    if (K::PREFETCH && t == 0 && grid + (int)gridDim.x < a.ngrids)
      prefetch_l2(reinterpret_cast<const float*>(a.in) + (long long)(grid + gridDim.x) * N * N * N,
                  4 * N * N * N);
    // x: rows t, t + T, ... straight from global memory, 16-byte loads (a
    // warp's rows are consecutive bytes; the second load of each 32-byte
    // sector finds it in L1)
#pragma unroll
    for (int i = 0; i < K::RPT; ++i) {
      const int r = t + K::T * i;
      if (K::RPT == 1 || r < K::ROWS) {
        float2 w[H];
#pragma unroll
        for (int j = 0; j < N / 4; ++j) {
          const float4 q = __ldg(gin + r * (N / 4) + j);
          w[2 * j] = make_float2(q.x, q.y);
          w[2 * j + 1] = make_float2(q.z, q.w);
        }
        DFT<H, -1>::run(w);
        float2 X[HC];
        X[0] = make_float2(w[0].x + w[0].y, 0.0f);
        X[H] = make_float2(w[0].x - w[0].y, 0.0f);
        static_for<1, H>([&](auto KK) {
          constexpr int k = decltype(KK)::value;
          const float2 p = w[k], q = make_float2(w[H - k].x, -w[H - k].y);  // W[k], conj W[h-k]
          const float2 e = make_float2(0.5f * (p.x + q.x), 0.5f * (p.y + q.y));
          const float2 o = make_float2(0.5f * (p.y - q.y), -0.5f * (p.x - q.x));  // (p - q) / 2i
          X[k] = cadd(e, twc<k, N, -1>(o));
        });
        float2* row = S + (r / N) * K::SZ + (r % N) * K::SY;
#pragma unroll
        for (int k = 0; k < HC; ++k) row[k] = X[k];
      }
    }
    __syncthreads();
    float2 v[N];
    // y: column (z, kx), z = t % n, kx = t / n
    if (t < K::COLS) {
      float2* col = S + (t % N) * K::SZ + t / N;
#pragma unroll
      for (int y = 0; y < N; ++y) v[y] = col[y * K::SY];
      DFT<N, -1>::run(v);
#pragma unroll
      for (int y = 0; y < N; ++y) col[y * K::SY] = v[y];
    }
    __syncthreads();
    // z: pencil p = (h + 1) ky + kx, to global memory (consecutive threads,
    // consecutive points)
    if (t < K::COLS) {
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = S[z * K::SZ + t];
      DFT<N, -1>::run(v);
#pragma unroll
      for (int z = 0; z < N; ++z) st_stream(gout + z * K::COLS + t, cscale(v[z], sc));
    }
    __syncthreads();  // the shared copy is rewritten by the next grid
  }
}

// Inverse kernel: a.in holds half spectra, a.out real grids.
template <int N>
__global__ void __launch_bounds__(Cfg<N>::T, Cfg<N>::MINB_I) rwholegrid_inv_kernel(const FusedArgs a) {
  using K = Cfg<N>;
  constexpr int H = K::H, HC = K::HC;
  extern __shared__ __align__(16) float2 S[];
  float* R = reinterpret_cast<float*>(S);
  const int t = threadIdx.x;
  const float sc = a.do_scale ? a.scale : 1.0f;
  for (int grid = blockIdx.x; grid < a.ngrids; grid += gridDim.x) {
    const float2* gin = a.in + (long long)grid * N * N * HC;
    float4* gout =
        reinterpret_cast<float4*>(reinterpret_cast<float*>(a.out) + (long long)grid * N * N * N);
    if (K::PREFETCH && t == 0 && grid + (int)gridDim.x < a.ngrids)
      prefetch_l2(a.in + (long long)(grid + gridDim.x) * N * N * HC, 8 * N * N * HC);
    float2 v[N];
    // z: pencil p = (h + 1) ky + kx straight from global memory (consecutive
    // threads, consecutive points); in the planes kx = 0 and h its Hermitian
    // part (X(kz, ky) + conj X(-kz, -ky)) / 2, the mirror pencil read again
    // (from L1 or L2)
    if (t < K::COLS) {
      const int ky = t / HC, kx = t % HC;
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = __ldg(gin + z * K::COLS + t);
      if (kx == 0 || kx == H) {
        const float2* mir = gin + ((N - ky) % N) * HC + kx;
#pragma unroll
        for (int z = 0; z < N; ++z) {
          const float2 c = __ldg(mir + ((N - z) % N) * K::COLS);
          v[z] = make_float2(0.5f * (v[z].x + c.x), 0.5f * (v[z].y - c.y));
        }
      }
      DFT<N, 1>::run(v);
#pragma unroll
      for (int z = 0; z < N; ++z) S[z * K::SZ + t] = v[z];
    }
    __syncthreads();
    // y: column (z, kx), z = t % n, kx = t / n
    if (t < K::COLS) {
      float2* col = S + (t % N) * K::SZ + t / N;
#pragma unroll
      for (int y = 0; y < N; ++y) v[y] = col[y * K::SY];
      DFT<N, 1>::run(v);
#pragma unroll
      for (int y = 0; y < N; ++y) col[y * K::SY] = v[y];
    }
    __syncthreads();
    // x: row n z + y of the spectrum -> n reals, in two phases when a thread
    // has two rows: first rows ROWS - T .. ROWS - 1 (one per thread), whose
    // real rows lie above every spectrum row still unread, then rows
    // 0 .. ROWS - T - 1; each phase reads its rows before a barrier and
    // writes them after it
#pragma unroll
    for (int ph = 0; ph < K::RPT; ++ph) {
      const int r = ph == 0 ? K::ROWS - K::T + t : t;
      const bool on = ph == 0 || r < K::ROWS - K::T;
      float2 w[H];
      if (on) {
        const float2* row = S + (r / N) * K::SZ + (r % N) * K::SY;
        float2 X[HC];
#pragma unroll
        for (int k = 0; k < HC; ++k) X[k] = row[k];
        // X[0] and X[h] are real for the Hermitian part: their real parts
        w[0] = make_float2(X[0].x + X[H].x, X[0].x - X[H].x);
        static_for<1, H>([&](auto KK) {
          constexpr int k = decltype(KK)::value;
          const float2 p = X[k], q = make_float2(X[H - k].x, -X[H - k].y);  // X[k], conj X[h-k]
          const float2 d = twc<k, N, 1>(csub(p, q));                        // W_n^-k (p - q)
          w[k] = cadd(cadd(p, q), mul_i<1>(d));
        });
        DFT<H, 1>::run(w);
      }
      __syncthreads();  // the rows this phase overwrites are read
      if (on) {
#pragma unroll
        for (int j = 0; j < N / 4; ++j)
          *reinterpret_cast<float4*>(R + r * K::RP + 4 * j) = make_float4(
              sc * w[2 * j].x, sc * w[2 * j].y, sc * w[2 * j + 1].x, sc * w[2 * j + 1].y);
      }
    }
    __syncthreads();
    // the reals out, coalesced: float4 e is row e / (n/4), quarter e % (n/4)
#pragma unroll 4
    for (int e = t; e < N * N * N / 4; e += K::T)
      __stcs(gout + e,
             *reinterpret_cast<const float4*>(R + (e / (N / 4)) * K::RP + 4 * (e % (N / 4))));
    __syncthreads();  // the shared copy is rewritten by the next grid
  }
}

template <int N, int DIR>
cudaError_t launch(const FusedArgs& a, int grid, cudaStream_t stream) {
  grid = grid < a.ngrids ? grid : a.ngrids;  // one block per grid at most
  if (DIR < 0)
    rwholegrid_fwd_kernel<N><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a);
  else
    rwholegrid_inv_kernel<N><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR>
KernelInfo info() {
  KernelInfo k;
  k.launch = &launch<N, DIR>;
  k.func = DIR < 0 ? (const void*)&rwholegrid_fwd_kernel<N> : (const void*)&rwholegrid_inv_kernel<N>;
  k.threads = Cfg<N>::T;
  k.smem = Cfg<N>::smem;
  k.sizes[0] = N;
  k.nsizes = 1;
  k.uses_work = 0;  // no tickets: no schedule, no counters to clear before a launch
  return k;
}

}  // namespace rwg
}  // namespace fft3d
