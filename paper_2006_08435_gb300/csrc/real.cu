// Transforms of REAL grids (a real density, the setting of the paper's
// plane-wave DFT application, section "Introduction") on top of the complex
// transform of Eq. 1.
//
// Forward (R2C): for a real grid r, F(-k) = conj(F(k)), so only the half
// spectrum kx = 0 .. n/2 is returned.  Two real grids a, b of the batch are
// transformed by ONE complex transform of c = a + i b: with C = F(c),
//   F(a)(k) = (C(k) + conj(C(-k))) / 2,   F(b)(k) = (C(k) - conj(C(-k))) / (2i),
// -k taken modulo n on every axis.  So a batch of B real grids costs
// ceil(B/2) complex transforms plus a packing pass before and a separating
// pass after.
// Inverse (C2R): the grid is the real part of the inverse transform of the
// Hermitian extension E(X) of the half spectrum X (E(X)(k) = X(k) for
// kx <= n/2, conj(X(-k)) above).  That real part is the inverse transform of
// the Hermitian part H(X)(k) = (E(X)(k) + conj(E(X)(-k))) / 2, which differs
// from E(X) only in the self-mirrored columns kx = 0 and n/2.  Two half
// spectra A, B are rebuilt as one full spectrum H(A) + i H(B), transformed
// once, and the real and imaginary parts of the result are the two grids.
//
// At 16^3 .. 128^3 in FP32 the transforms run instead as dedicated kernels
// with half-length row transforms: at 16^3 and 32^3 a whole grid per block
// (rwholegrid.cuh), at 64^3 and 128^3 two phases (rgrid.cuh: one pass over
// the real grid and one over the half spectrum, a workspace of n^2/2
// complex per grid for the Nyquist column of the forward transform); everywhere else the
// pair scheme above, whose kernels here move data only (pack, separate,
// rebuild, split) and whose transforms are the library's complex plans.
// Packing two grids into one makes each grid's rounding error relative to
// the larger of the pair.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fft3d.h"
#include "internal.h"
#include "schedule.h"

struct fft3d_real_plan_s {
  int n = 0, batch = 0, pairs = 0, direction = FFT3D_FORWARD;
  // pair scheme
  fft3d_plan inner = nullptr;  // complex plan of `pairs` n^3 grids
  float2* d_work = nullptr;    // pairs * n^3 complex points
  // dedicated kernels (rgrid.cuh)
  bool fused = false;
  fft3d::KernelInfo kern;
  fft3d::SchedBlock* d_blocks = nullptr;
  unsigned* d_count = nullptr;   // [0] ticket, [1 + g] phase-0 items of grid g done
  unsigned* d_status = nullptr;
  float2* d_aux = nullptr;       // forward: n * n/2 complex per grid (Nyquist pencils)
  int nblocks = 0, total_items = 0, grid = 0;
  float scale = 1.0f;
  int do_scale = 0;
};

namespace fft3d {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 8;

// Launch shape: the points of a pair along x, at most two pairs along y at a
// time (a block row loops over the pairs), about kMaxBlocks blocks in all.
// The separating and rebuilding kernels read every row of a pair twice,
// directly and as a mirror about half a pair later; with two pairs in flight
// (34 MB at 128^3) the second read still finds the row in L2.
dim3 grid_for(long long per_pair, int pairs) {
  const int by = pairs < 2 ? pairs : 2;
  long long bx = (per_pair + kThreads - 1) / kThreads;
  const long long cap = kMaxBlocks / by > 0 ? kMaxBlocks / by : 1;
  if (bx > cap) bx = cap;
  return dim3((unsigned)(bx < 1 ? 1 : bx), (unsigned)by);
}

// c_j = r_{2j} + i r_{2j+1} (0 for a missing partner), 4 points per
// thread: q = n^3 / 4 float4 per real grid, 2 q per complex grid.  Reads
// r[2j q + e] (2j <= batch - 1) and, when 2j + 1 < batch, r[(2j + 1) q + e];
// writes c[2 (j q + e)] and the next float4 (< 2 pairs q).
__global__ void pack_pairs_kernel(const float4* __restrict__ r, float4* __restrict__ c, int q,
                                  int batch, int pairs) {
  for (int j = blockIdx.y; j < pairs; j += gridDim.y) {
    const float4* ra = r + 2LL * j * q;
    const bool has_b = 2 * j + 1 < batch;
    float4* cj = c + 2LL * j * q;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < q; e += gridDim.x * blockDim.x) {
      const float4 a = __ldcs(ra + e);
      float4 b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (has_b) b = __ldcs(ra + q + e);
      cj[2 * e] = make_float4(a.x, b.x, a.y, b.y);
      cj[2 * e + 1] = make_float4(a.z, b.z, a.w, b.w);
    }
  }
}

// The inverse of the packing: r_{2j} = Re c_j, r_{2j+1} = Im c_j.
__global__ void split_pairs_kernel(const float4* __restrict__ c, float4* __restrict__ r, int q,
                                   int batch, int pairs) {
  for (int j = blockIdx.y; j < pairs; j += gridDim.y) {
    const float4* cj = c + 2LL * j * q;
    float4* ra = r + 2LL * j * q;
    const bool has_b = 2 * j + 1 < batch;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < q; e += gridDim.x * blockDim.x) {
      const float4 u = __ldcs(cj + 2 * e), v = __ldcs(cj + 2 * e + 1);
      __stcs(ra + e, make_float4(u.x, u.z, v.x, v.z));
      if (has_b) __stcs(ra + q + e, make_float4(u.y, u.w, v.y, v.w));
    }
  }
}

// Half spectra of grids 2j and 2j + 1 from C_j: point i = (kz n + ky) h + kx
// of the half layout (h = n/2 + 1; contiguous writes), read from C_j at
// (kz, ky, kx) and at -k = ((n - kz) mod n, (n - ky) mod n, (n - kx) mod n).
// A pair's C_j (n^3 points, 16.8 MB at 128^3) is read through L2: every row
// is read once directly and once as a mirror while the pair is in flight.
__global__ void separate_pairs_kernel(const float2* __restrict__ c, float2* __restrict__ out,
                                      int n, int batch, int pairs) {
  const int h = n / 2 + 1, m = n * n * h;
  for (int j = blockIdx.y; j < pairs; j += gridDim.y) {
    const float2* cj = c + (long long)j * n * n * n;
    float2* oa = out + 2LL * j * m;
    const bool has_b = 2 * j + 1 < batch;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
      const int row = i / h, kx = i - row * h;
      const int kz = row / n, ky = row - kz * n;
      const int mz = kz ? n - kz : 0, my = ky ? n - ky : 0;
      const float2 C = __ldg(cj + row * n + kx);
      const float2 M = __ldg(cj + (mz * n + my) * n + (kx ? n - kx : 0));  // C(-k)
      oa[i] = make_float2(0.5f * (C.x + M.x), 0.5f * (C.y - M.y));
      if (has_b) oa[m + i] = make_float2(0.5f * (C.y + M.y), 0.5f * (M.x - C.x));
    }
  }
}

// Full spectrum H(A) + i H(B) of pair j, A = X_{2j}, B = X_{2j+1} (0 when
// missing), point i = (kz n + ky) n + kx.  Columns kx < n/2 but 0 come
// straight from the half rows, kx > n/2 from conj of the mirrored row at
// column n - kx (in 1 .. n/2 - 1), and the self-mirrored columns 0 and n/2
// are the mean of the bin and the conjugate of its mirror.
__global__ void rebuild_pairs_kernel(const float2* __restrict__ x, float2* __restrict__ c,
                                     int n, int batch, int pairs) {
  const int h = n / 2 + 1, half = n / 2, m = n * n * h, nf = n * n * n;
  for (int j = blockIdx.y; j < pairs; j += gridDim.y) {
    const float2* xa = x + 2LL * j * m;
    const bool has_b = 2 * j + 1 < batch;
    float2* cj = c + (long long)j * nf;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
      const int row = i / n, kx = i - row * n;
      const int kz = row / n, ky = row - kz * n;
      const int mz = kz ? n - kz : 0, my = ky ? n - ky : 0;
      const float2* ar = xa + row * h;
      const float2* am = xa + (mz * n + my) * h;
      float2 A, B = make_float2(0.0f, 0.0f);
      if (kx == 0 || kx == half) {
        const float2 p = __ldg(ar + kx), q = __ldg(am + kx);
        A = make_float2(0.5f * (p.x + q.x), 0.5f * (p.y - q.y));
        if (has_b) {
          const float2 s = __ldg(ar + m + kx), t = __ldg(am + m + kx);
          B = make_float2(0.5f * (s.x + t.x), 0.5f * (s.y - t.y));
        }
      } else if (kx < half) {
        A = __ldg(ar + kx);
        if (has_b) B = __ldg(ar + m + kx);
      } else {
        const float2 p = __ldg(am + (n - kx));
        A = make_float2(p.x, -p.y);
        if (has_b) {
          const float2 s = __ldg(am + m + (n - kx));
          B = make_float2(s.x, -s.y);
        }
      }
      cj[i] = make_float2(A.x - B.y, A.y + B.x);  // A + i B
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

void set_real_norm(fft3d_real_plan p, int norm, int n) {
  const double n3 = (double)n * n * n;
  if (norm == FFT3D_NORM_BY_N) {
    p->scale = (float)(1.0 / n3);
    p->do_scale = 1;
  } else if (norm == FFT3D_NORM_ORTHO) {
    p->scale = (float)(1.0 / std::sqrt(n3));
    p->do_scale = 1;
  }
}

void free_fused(fft3d_real_plan p) {
  cudaFree(p->d_aux);
  cudaFree(p->d_blocks);
  cudaFree(p->d_count);
  cudaFree(p->d_status);
}

}  // namespace

// Plan of the dedicated kernels: per grid, phase 0 has n/P items (forward:
// P planes each; inverse: P rows ky of every z), phase 1 n/P items (forward:
// rows, plus the Nyquist column; inverse: planes); forward blocks have one
// ticket more.  (P = 128/n: every item has 128 rows.)  The schedule's L2 budget counts 8 n^3
// bytes of intermediate per grid (a complex grid); a real grid's is about
// half of that, so the budget passed is scaled by the ratio.  The forward
// transform keeps more grids in flight (60% of L2 against 40%): its input
// is read once and its longer lag between planes and z items pays
// (measured); the inverse re-reads the mirror columns of its input and is
// faster with the smaller share.
int create_fused_real(int n, int batch, int direction, int norm, const KernelInfo& k,
                      fft3d_real_plan* out_plan) {
  int dev = -1, sms = 0, l2 = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_NO_DEVICE;
  }
  if (major != 10 || minor != 3) return FFT3D_ERR_NO_DEVICE;
  if (cudaFuncSetAttribute(k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.func, k.threads, k.smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  const int resident = per_sm * sms;
  const int forward = direction == FFT3D_FORWARD;
  if (!k.uses_work) {
    // a kernel without tickets (whole grids per block): no schedule, no
    // counters, no workspace; a block per grid, up to the resident blocks
    auto* p = new (std::nothrow) fft3d_real_plan_s();
    if (!p) return FFT3D_ERR_ALLOC;
    p->n = n;
    p->batch = batch;
    p->direction = direction;
    p->fused = true;
    p->kern = k;
    p->grid = batch < resident ? batch : resident;
    set_real_norm(p, norm, n);
    if (cudaMalloc(&p->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      free_fused(p);
      delete p;
      return FFT3D_ERR_ALLOC;
    }
    *out_plan = p;
    return FFT3D_SUCCESS;
  }
  const double n3 = (double)n * n * n;
  const double inter = forward ? (double)n * n * (n / 2 + 1) * 8.0 : 4.0 * n3;
  std::vector<int> dims(batch, n), order(batch), plane_end(batch);
  for (int g = 0; g < batch; ++g) order[g] = g;
  std::vector<SchedBlock> blocks(2 * (size_t)batch);
  int total = 0;
  // the kernel's tickets per block (forward: the z block's last is the
  // Nyquist item, the plane block's last is empty)
  const int nb = schedule_blocks(batch, dims.data(), order.data(), resident * k.items_in_flight,
                                 (forward ? 0.6 : 0.4) * (double)l2 * (8.0 * n3 / inter),
                                 k.phase_items, plane_end.data(), blocks.data(), &total);
  auto* p = new (std::nothrow) fft3d_real_plan_s();
  if (!p) return FFT3D_ERR_ALLOC;
  p->n = n;
  p->batch = batch;
  p->direction = direction;
  p->fused = true;
  p->kern = k;
  p->nblocks = nb;
  p->total_items = total;
  p->grid = total < resident ? total : resident;
  set_real_norm(p, norm, n);
  if (cudaMalloc(&p->d_blocks, sizeof(SchedBlock) * (size_t)nb) != cudaSuccess ||
      cudaMalloc(&p->d_count, sizeof(unsigned) * (size_t)(batch + 1)) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMemcpy(p->d_blocks, blocks.data(), sizeof(SchedBlock) * (size_t)nb,
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
      (forward && cudaMalloc(&p->d_aux, sizeof(float2) * (size_t)batch * n * (n / 2)) !=
                      cudaSuccess)) {
    cudaGetLastError();
    free_fused(p);
    delete p;
    return FFT3D_ERR_ALLOC;
  }
  *out_plan = p;
  return FFT3D_SUCCESS;
}

int execute_fused_real(fft3d_real_plan p, const void* in, void* out, cudaStream_t s) {
  if (p->kern.uses_work &&
      cudaMemsetAsync(p->d_count, 0, sizeof(unsigned) * (size_t)(p->batch + 1), s) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  FusedArgs a{};
  a.in = static_cast<const float2*>(in);
  a.out = static_cast<float2*>(out);
  a.blocks = p->d_blocks;
  a.nblocks = p->nblocks;
  a.total_items = p->total_items;
  a.work = p->d_count;
  a.status = p->d_status;
  a.scale = p->scale;
  a.do_scale = p->do_scale;
  a.timeout_ns = kDefaultWaitNs;
  a.ngrids = p->batch;
  a.aux = p->d_aux;
  if (p->kern.launch(a, p->grid, s) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  return FFT3D_SUCCESS;
}

}  // namespace fft3d

extern "C" {

int fft3d_real_plan_create(int n, int batch, int precision, int direction, int norm,
                           fft3d_real_plan* out_plan) {
  if (!out_plan) return FFT3D_ERR_NULL_PTR;
  *out_plan = nullptr;
  if (batch < 1 || batch > (1 << 24)) return FFT3D_ERR_INVALID_ARG;
  if (n < 2 || (n & 1) || !fft3d_size_supported(n)) return FFT3D_ERR_UNSUPPORTED_SIZE;
  if (direction != FFT3D_FORWARD && direction != FFT3D_INVERSE) return FFT3D_ERR_INVALID_ARG;
  if (norm < FFT3D_NORM_NONE || norm > FFT3D_NORM_ORTHO) return FFT3D_ERR_INVALID_ARG;
  const char* path = std::getenv("FFT3D_REAL_PATH");  // "pairs": the pair scheme everywhere
  const bool pairs_only = path && std::strcmp(path, "pairs") == 0;
  if (precision == FFT3D_FP32 && !pairs_only) {
    const fft3d::KernelInfo k = fft3d::real_kernel_info(n, direction == FFT3D_FORWARD ? -1 : 1);
    if (k.launch) return fft3d::create_fused_real(n, batch, direction, norm, k, out_plan);
  }
  const int pairs = (batch + 1) / 2;
  fft3d_plan inner = nullptr;
  int rc = fft3d_plan_create(n, n, n, pairs, precision, direction, norm, &inner);
  if (rc) return rc;
  auto* p = new (std::nothrow) fft3d_real_plan_s();
  if (!p) {
    fft3d_plan_destroy(inner);
    return FFT3D_ERR_ALLOC;
  }
  p->n = n;
  p->batch = batch;
  p->pairs = pairs;
  p->direction = direction;
  p->inner = inner;
  const size_t bytes = (size_t)pairs * n * n * n * sizeof(float2);
  if (cudaMalloc(&p->d_work, bytes) != cudaSuccess) {
    cudaGetLastError();
    fft3d_plan_destroy(inner);
    delete p;
    return FFT3D_ERR_ALLOC;
  }
  *out_plan = p;
  return FFT3D_SUCCESS;
}

int fft3d_real_execute(fft3d_real_plan plan, const void* in, void* out, void* stream) {
  using namespace fft3d;
  if (!plan || !in || !out) return FFT3D_ERR_NULL_PTR;
  if (!aligned16(in) || !aligned16(out)) return FFT3D_ERR_MISALIGNED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (plan->fused) return execute_fused_real(plan, in, out, s);
  const int n = plan->n, batch = plan->batch, pairs = plan->pairs;
  const int q = n * n * n / 4, h = n / 2 + 1;
  if (plan->direction == FFT3D_FORWARD) {
    pack_pairs_kernel<<<grid_for(q, pairs), kThreads, 0, s>>>(
        static_cast<const float4*>(in), reinterpret_cast<float4*>(plan->d_work), q, batch, pairs);
    if (cudaGetLastError() != cudaSuccess) return FFT3D_ERR_CUDA;
    const int rc = fft3d_execute(plan->inner, plan->d_work, plan->d_work, stream);
    if (rc) return rc;
    separate_pairs_kernel<<<grid_for((long long)n * n * h, pairs), kThreads, 0, s>>>(
        plan->d_work, static_cast<float2*>(out), n, batch, pairs);
  } else {
    rebuild_pairs_kernel<<<grid_for((long long)n * n * n, pairs), kThreads, 0, s>>>(
        static_cast<const float2*>(in), plan->d_work, n, batch, pairs);
    if (cudaGetLastError() != cudaSuccess) return FFT3D_ERR_CUDA;
    const int rc = fft3d_execute(plan->inner, plan->d_work, plan->d_work, stream);
    if (rc) return rc;
    split_pairs_kernel<<<grid_for(q, pairs), kThreads, 0, s>>>(
        reinterpret_cast<const float4*>(plan->d_work), static_cast<float4*>(out), q, batch,
        pairs);
  }
  return cudaGetLastError() == cudaSuccess ? FFT3D_SUCCESS : FFT3D_ERR_CUDA;
}

int fft3d_real_get_device_status(fft3d_real_plan plan, void* stream) {
  if (!plan) return FFT3D_ERR_NULL_PTR;
  if (!plan->fused) return fft3d_get_device_status(plan->inner, stream);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  unsigned st = 0;
  if (cudaMemcpy(&st, plan->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(plan->d_status, 0, sizeof(unsigned)) != cudaSuccess)
    return FFT3D_ERR_CUDA;
  return st == fft3d::kStatusOk ? FFT3D_SUCCESS : FFT3D_ERR_DEVICE_TIMEOUT;
}

int fft3d_real_plan_destroy(fft3d_real_plan plan) {
  if (!plan) return FFT3D_SUCCESS;
  if (plan->fused) {
    fft3d::free_fused(plan);
    delete plan;
    return FFT3D_SUCCESS;
  }
  cudaFree(plan->d_work);
  const int rc = fft3d_plan_destroy(plan->inner);
  delete plan;
  return rc;
}

}  // extern "C"
