// Host side of the C ABI: argument validation, planning (size split,
// FP64 twiddle tables rounded to FP32, work schedule), device buffers and
// launches.  See include/fft3d.h for the contract of each entry point.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fft3d.h"
#include "internal.h"
#include "schedule.h"
#include "sizes.h"
#include "tc_stage.cuh"

namespace fft3d {

KernelInfo fused_kernel_info_n16(int dir, int variant);
KernelInfo fused_kernel_info_n32(int dir, int variant);
KernelInfo fused_kernel_info_n48(int dir, int variant);
KernelInfo fused_kernel_info_n64(int dir, int variant);
KernelInfo fused_kernel_info_n80(int dir, int variant);
KernelInfo fused_kernel_info_n96(int dir, int variant);
KernelInfo fused_kernel_info_n128(int dir, int variant);
KernelInfo tc_kernel_info_n64(int dir, int prec, int variant);
KernelInfo tc_kernel_info_n128(int dir, int prec, int variant);

KernelInfo tc_kernel_info(int n, int dir, int prec, int variant) {
  switch (n) {
    case 64: return tc_kernel_info_n64(dir, prec, variant);
    case 128: return tc_kernel_info_n128(dir, prec, variant);
    default: return KernelInfo{};
  }
}
static bool tc_size(int n) { return n == 64 || n == 128; }

KernelInfo fused_kernel_info(int n, int dir, int variant) {
  switch (n) {
    case 16: return fused_kernel_info_n16(dir, variant);
    case 32: return fused_kernel_info_n32(dir, variant);
    case 48: return fused_kernel_info_n48(dir, variant);
    case 64: return fused_kernel_info_n64(dir, variant);
    case 80: return fused_kernel_info_n80(dir, variant);
    case 96: return fused_kernel_info_n96(dir, variant);
    case 128: return fused_kernel_info_n128(dir, variant);
    default: return KernelInfo{};
  }
}

// W_n^m = exp(-2 pi i m / n) for the table entry (n1, k2) of edge n split
// as n = l1 * l2: tw[k2 * l1 + n1] = W_n^((n1 * k2) mod n), evaluated in FP64
// by the host math library on the reduced exponent and rounded to nearest
// FP32.
static void twiddle_table(int n, int l1, float* out /* 2 * n floats */) {
  const int l2 = n / l1;
  for (int k2 = 0; k2 < l2; ++k2)
    for (int n1 = 0; n1 < l1; ++n1) {
      const int m = (n1 * k2) % n;
      const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)n;
      out[2 * (k2 * l1 + n1)] = (float)std::cos(a);
      out[2 * (k2 * l1 + n1) + 1] = (float)(-std::sin(a));
    }
}

// B fragments of the tensor-core radix-16 stage (layout in tc_stage.cuh):
// the 32 x 32 real form of the forward DFT_16 matrix, B[2j+c][2k+d] from
// W_16^(jk) = wr + i wi: (c,d) = (0,0) wr, (1,0) -wi, (0,1) wi, (1,1) wr,
// evaluated in FP64, split as hi = rn(b), lo = rn(b - hi) in FP16 (prec 1,
// 3) or BF16 (prec 2).
static void mma_fragments(int prec, uint32_t* out /* tc::kFragWords */) {
  auto entry = [](int kr, int nr) {
    const int j = kr / 2, c = kr % 2, k = nr / 2, d = nr % 2;
    const double a = -2.0 * 3.14159265358979323846 * (double)((j * k) % 16) / 16.0;
    const double wr = std::cos(a), wi = std::sin(a);
    return c == 0 ? (d == 0 ? wr : wi) : (d == 0 ? -wi : wr);
  };
  auto split = [prec](double v, unsigned short& hi, unsigned short& lo) {
    if (prec == 2) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
      const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
      hi = __bfloat16_as_ushort(h);
      lo = __bfloat16_as_ushort(l);
    } else {
      const __half h = __float2half_rn((float)v);
      const __half l = __float2half_rn((float)(v - (double)__half2float(h)));
      hi = __half_as_ushort(h);
      lo = __half_as_ushort(l);
    }
  };
  for (int term = 0; term < 2; ++term)
    for (int s = 0; s < 2; ++s)
      for (int u = 0; u < 4; ++u)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane >> 2, t = lane & 3, col = 8 * u + g;
          for (int reg = 0; reg < 2; ++reg) {
            const int r0 = 16 * s + 2 * t + 8 * reg;
            unsigned short h0, l0, h1, l1;
            split(entry(r0, col), h0, l0);
            split(entry(r0 + 1, col), h1, l1);
            const unsigned short a0 = term ? l0 : h0, a1 = term ? l1 : h1;
            out[(((term * 2 + s) * 4 + u) * 32 + lane) * 2 + reg] =
                (uint32_t)a0 | ((uint32_t)a1 << 16);
          }
        }
}

// B operands of the tcgen05 64^3 kernel (tcgen.cuh): for k1 = 0..3 the
// 32 x 32 real form of M_k1[n2][k2] = W_64^(n2 (k1 + 4 k2)) (forward root;
// the radix-16 DFT with the twiddles of the radix-4 x 16 split folded in),
// rows and columns interleaved re/im as for mma_fragments, stored K-major
// (row = output column 2 k2 + d, 32 input entries 2 n2 + c per row) in
// 8 x 16-byte core matrices: byte ((row / 8) * 4 + kk / 8) * 128 +
// (row % 8) * 16 + (kk % 8) * 2 of block (term * 4 + k1) * 2048, term 0 the
// hi halves, 1 the lo halves (FP16, or BF16 for prec 2): hi = rn(b),
// lo = rn(b - hi), each rounded once from the FP64 value.
static void umma_b_table(int prec, uint16_t* out /* 8192 */) {
  if (prec == FFT3D_SPLIT_FP8 || prec == FFT3D_FP8) {
    // E4M3 entries of 16 b: hi = rn(16 b), lo = rn(16 b - hi) (round to
    // nearest even, saturating), byte ((row / 8) * 2 + kk / 16) * 128 +
    // (row % 8) * 16 + kk % 16 of block (term * 4 + k1) * 1024
    unsigned char* bytes = reinterpret_cast<unsigned char*>(out);
    std::memset(bytes, 0, 16384);
    for (int k1 = 0; k1 < 4; ++k1)
      for (int row = 0; row < 32; ++row)
        for (int kk = 0; kk < 32; ++kk) {
          const int k2 = row / 2, d = row % 2, n2 = kk / 2, c = kk % 2;
          const int m = (n2 * (k1 + 4 * k2)) % 64;
          const double a = -2.0 * 3.14159265358979323846 * (double)m / 64.0;
          const double wr = std::cos(a), wi = std::sin(a);
          const double v = 16.0 * (c == 0 ? (d == 0 ? wr : wi) : (d == 0 ? -wi : wr));
          const __nv_fp8_storage_t hi = __nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
          const __half_raw hr = __nv_cvt_fp8_to_halfraw(hi, __NV_E4M3);
          const double hv = (double)__half2float(__half(hr));
          const __nv_fp8_storage_t lo = __nv_cvt_double_to_fp8(v - hv, __NV_SATFINITE, __NV_E4M3);
          const int byte = ((row / 8) * 2 + kk / 16) * 128 + (row % 8) * 16 + kk % 16;
          bytes[(0 * 4 + k1) * 1024 + byte] = hi;
          bytes[(1 * 4 + k1) * 1024 + byte] = lo;
        }
    return;
  }
  for (int k1 = 0; k1 < 4; ++k1)
    for (int row = 0; row < 32; ++row)
      for (int kk = 0; kk < 32; ++kk) {
        const int k2 = row / 2, d = row % 2, n2 = kk / 2, c = kk % 2;
        const int m = (n2 * (k1 + 4 * k2)) % 64;
        const double a = -2.0 * 3.14159265358979323846 * (double)m / 64.0;
        const double wr = std::cos(a), wi = std::sin(a);
        const double v = c == 0 ? (d == 0 ? wr : wi) : (d == 0 ? -wi : wr);
        uint16_t hi, lo;
        if (prec == 2) {
          const __nv_bfloat16 h = __double2bfloat16(v);
          const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
          hi = __bfloat16_as_ushort(h);
          lo = __bfloat16_as_ushort(l);
        } else {
          const __half h = __double2half(v);
          const __half l = __double2half(v - (double)__half2float(h));
          hi = __half_as_ushort(h);
          lo = __half_as_ushort(l);
        }
        const int byte = ((row / 8) * 4 + kk / 8) * 128 + (row % 8) * 16 + (kk % 8) * 2;
        out[(0 * 4 + k1) * 1024 + byte / 2] = hi;
        out[(1 * 4 + k1) * 1024 + byte / 2] = lo;
      }
}

static bool fused_size(int n) { return fused_slot(n) >= 0; }

// Kernel variants of a single-size FP32 plan (each the fastest for some
// edge and batch on the GB300): 0 plain persistent kernel, 1 the same with
// twice the threads (16^3 to 96^3), 3 the cluster-fused single-pass kernel
// (16^3, 32^3), 12 a whole 16^3 grid per block, 4 the double-buffered persistent kernel (32^3, 48^3, 80^3,
// 96^3), 5 the warp-owned two-phase kernel (64^3, 128^3), 6 to 8 the
// tensor-TMA thread-per-pencil kernels (128^3 split-y; 64^3 one-plane and
// two-plane items).  Tensor-core precisions: 0 the plain persistent kernel,
// 9 the tensor-TMA items with tcgen05 products (64^3 two-plane, 128^3
// split-y).
// Variant 10 (kGeneralVariant): the general path, one pencil pass per axis
// (axis.cu), the only one for non-cubic grids and edges without a fused
// kernel, selectable for the others.  Mixed plans: 0 one
// launch of the mixed-edge kernel, 1 one launch per distinct edge with that
// edge's default kernel, 2 the launches of 1 as concurrent branches.
std::vector<int> variant_candidates(bool mixed, int n, int precision) {
  if (mixed) return {0, 1, 2};
  // the block-floating-point and FP8 kinds exist on the tcgen05 kernels only
  if (precision >= FFT3D_BFP16) return {9};
  if (precision != FFT3D_FP32) return {0, 9};
  if (!fused_size(n)) return {kGeneralVariant};
  switch (n) {
    case 16: return {0, 1, 3, kGeneralVariant, 12};
    case 32: return {0, 1, 3, 4, kGeneralVariant, 13};
    case 64: return {0, 1, 5, 7, 8, kGeneralVariant};
    case 128: return {0, 5, 6, kGeneralVariant};
    default: return {0, 1, 4, kGeneralVariant, 13};  // 48, 80, 96
  }
}

// The fastest variant measured on the GB300 for each edge and batch
// (back-to-back executes; one grid also with L2 flushed):
//   16^3: cluster-fused below 128 grids, whole grid per block from 128;
//   32^3: cluster-fused below 128 grids, thread pairs from 128;
//   48^3: plain persistent below 32 grids, thread pairs from 32;  80^3:
//     plain persistent for one grid, the
//     double-buffered persistent kernel from 4, the thread-pair kernel from
//     8;  96^3: plain persistent below 4 grids, the thread-pair kernel from 4;
//   64^3: warp-owned for one grid, the persistent kernel with twice the
//     threads below 16, thread-per-pencil below 64, two-plane from 64;
//   128^3: warp-owned for one grid, split-y from 2;
//   tensor-core precisions: the plain persistent kernel (mma.sync) for few
//     grids, the tcgen05 kernels from 16 (64^3) and 2 (128^3) grids.
int builtin_default_variant(bool mixed, int n, int batch, int precision) {
  // mixed edges: one launch per distinct edge, as concurrent branches (the
  // mixed workload of 64 grids, forward + inverse in one graph: 0.65 ms
  // against 0.70 ms with the launches in sequence, which in turn beat one
  // mixed-edge launch per direction)
  if (mixed) return 2;
  if (precision >= FFT3D_BFP16) return 9;
  if (precision != FFT3D_FP32) return (n == 64 && batch >= 16) || (n == 128 && batch >= 2) ? 9 : 0;
  switch (n) {
    // 16^3: the cluster-fused kernel (8 blocks per grid) below 128 grids (one
    // grid, L2 flushed: 8.9 us against 11.9 for the persistent kernel;
    // 2-64 grids: 8.3-9.9 us against 9.6-11.7 for the whole-grid kernel),
    // the whole-grid kernel from 128 (x 256: 0.29 against 0.15; x 4096:
    // 0.53 against 0.17)
    case 16: return batch >= 128 ? 12 : 3;
    // 32^3: the cluster-fused kernel (16 blocks per grid) below 128 grids
    // (one grid, L2 flushed: 10.9 us against 11.9; 2-64 grids: 11.6-23.2 us
    // against 13.0-26.6 for the persistent kernel), the thread-pair kernel
    // (four-plane items of 32 KB) from 128 (x 256: 0.46; x 1024: 0.51)
    case 32: return batch >= 128 ? 13 : 3;
    case 64: return batch == 1 ? 5 : batch < 16 ? 1 : batch < 64 ? 7 : 8;
    // 80^3, 96^3: the thread-pair kernel from 8 (80) and 4 (96) grids (x 256:
    // 0.57 / 0.62 of the roofline against 0.30 / 0.25; x 12-14: 0.41-0.43
    // against 0.25-0.27); below, the double-buffered kernel (80) or the
    // plain persistent one
    case 80: return batch >= 8 ? 13 : batch >= 4 ? 4 : 0;
    case 96: return batch >= 4 ? 13 : 0;
    // 48^3: the thread-pair kernel (two-plane items of 36 KB) from 32 grids
    // (x 64: 0.39 against 0.28; x 256: 0.52 against 0.30), the plain kernel
    // below
    case 48: return batch >= 32 ? 13 : 0;
    case 128: return batch == 1 ? 5 : 6;
    default: return 0;
  }
}

}  // namespace fft3d

using namespace fft3d;

// One persistent launch: a kernel and the grids it transforms.  Local grid l
// of the unit is grid grids[l] of the plan (device map d_map, or identity).
struct Unit {
  KernelInfo kernel;
  std::vector<int> grids;
  int grid = 0;          // persistent blocks launched
  int total_items = 0;
  int nblocks = 0;
  float2* d_tw = nullptr;
  uint32_t* d_frag = nullptr;
  SchedBlock* d_blocks = nullptr;
  unsigned* d_work = nullptr;
  size_t work_bytes = 0;
  int* d_map = nullptr;
  // mixed-edge plans on packed buffers: the kernel's per-grid tensor maps
  // (KernelInfo::launch_maps) over these element offsets of the unit's grids
  bool use_maps = false;
  std::vector<long long> host_off;
};

struct HostIO;

struct fft3d_plan_s {
  HostIO* hio = nullptr;             // host-buffer pipeline (fft3d_plan_host_io)
  int device = -1;
  int nx = 0, ny = 0, nz = 0, batch = 0;
  int precision = 0, direction = -1, norm = 0;
  bool mixed = false;
  int variant = 0;
  std::vector<int> dims;             // per-grid edge
  std::vector<long long> offsets;    // per-grid element offset in packed buffers
  long long total_points = 0;
  float scale = 1.0f;
  int do_scale = 0;
  long long timeout_ns = kDefaultWaitNs;
  std::vector<Unit> units;
  // mixed-edge plans whose units use per-grid tensor maps on packed buffers:
  // the units for calls with pointer arrays (the same edges, kernels that
  // address grids through pointers)
  std::vector<Unit> units_ptr;
  // mixed variant 2: the units as concurrent branches, one side stream and
  // one join event per unit, forked from the caller's stream (owned)
  bool branches = false;
  cudaEvent_t fork = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  // device buffers shared by the units (owned)
  long long* d_off = nullptr;
  unsigned* d_status = nullptr;
  // general path (variant kGeneralVariant): one pass per axis over chunks of
  // `chunk` grids (the last chunk `tail` grids); pass[axis][0] for a full
  // chunk, pass[axis][1] for the tail
  bool general = false;
  std::vector<AxisTable> tables;
  AxisLaunch pass[3][2];
  bool xy_fused = false;  // x and y in one plane pass (the plane fits shared memory)
  PlaneLaunch plane[2];
  int chunk = 0, nchunks = 0, tail = 0;
};

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

void free_plan_buffers(fft3d_plan p) {
  if (!p) return;
  for (std::vector<Unit>* list : {&p->units, &p->units_ptr})
  for (Unit& u : *list) {
    cudaFree(u.d_tw);
    cudaFree(u.d_frag);
    cudaFree(u.d_blocks);
    cudaFree(u.d_work);
    cudaFree(u.d_map);
    u.d_tw = nullptr;
    u.d_frag = nullptr;
    u.d_blocks = nullptr;
    u.d_work = nullptr;
    u.d_map = nullptr;
  }
  cudaFree(p->d_off);
  cudaFree(p->d_status);
  p->d_off = nullptr;
  p->d_status = nullptr;
  for (cudaStream_t s : p->side)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : p->join)
    if (e) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  p->side.clear();
  p->join.clear();
  p->fork = nullptr;
  for (AxisTable& t : p->tables) {
    cudaFree(t.d_tw);
    cudaFree(t.d_pos);
    t.d_tw = nullptr;
    t.d_pos = nullptr;
  }
}

int check_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_NO_DEVICE;
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_NO_DEVICE;
  }
  if (major != 10 || minor != 3) return FFT3D_ERR_NO_DEVICE;
  return FFT3D_SUCCESS;
}

// Ticket order (schedule_blocks, schedule.h) into a vector.
std::vector<SchedBlock> build_schedule(const std::vector<int>& dims, const std::vector<int>& order,
                                       int concurrency, double l2_budget, int phase_items,
                                       int* total_items) {
  std::vector<SchedBlock> blocks(2 * dims.size());
  std::vector<int> plane_end(dims.size());
  const int nb = schedule_blocks((int)dims.size(), dims.data(), order.data(), concurrency,
                                 l2_budget, phase_items, plane_end.data(), blocks.data(),
                                 total_items);
  blocks.resize(nb);
  return blocks;
}

// The order in which a unit's grids are scheduled: largest edge first,
// ties in grid order.
std::vector<int> schedule_order(const std::vector<int>& dims) {
  std::vector<int> order(dims.size());
  for (size_t l = 0; l < dims.size(); ++l) order[l] = (int)l;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dims[a] > dims[b]; });
  return order;
}

template <class T>
int upload(T** dst, const T* src, size_t count) {
  if (cudaMalloc(dst, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_ALLOC;
  }
  if (cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  return FFT3D_SUCCESS;
}

// Device buffers and launch geometry of one unit; `identity` units address
// grids by their own index (no map).  Local grids are scheduled largest
// edge first.
int finish_unit(fft3d_plan p, Unit& u, bool identity) {
  cudaError_t e = cudaFuncSetAttribute(u.kernel.func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)u.kernel.smem);
  if (e == cudaSuccess && u.use_maps)
    e = cudaFuncSetAttribute(u.kernel.func_maps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)u.kernel.smem);
  if (e != cudaSuccess) return FFT3D_ERR_CUDA;
  int per_sm = 0, sms = 0, l2_bytes = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, u.kernel.func, u.kernel.threads,
                                                    u.kernel.smem);
  if (e != cudaSuccess || per_sm < 1) return FFT3D_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, p->device) != cudaSuccess)
    return FFT3D_ERR_CUDA;
  const int m = (int)u.grids.size();
  int cluster_blocks = 0;  // > 0: launch this many blocks (whole clusters)
  if (u.kernel.cluster > 0) {
    if (u.kernel.cluster > 8 &&
        cudaFuncSetAttribute(u.kernel.func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return FFT3D_ERR_UNSUPPORTED_SIZE;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = u.kernel.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(u.kernel.cluster * sms, 1, 1);
    cfg.blockDim = dim3(u.kernel.threads, 1, 1);
    cfg.dynamicSmemBytes = u.kernel.smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, u.kernel.func, &cfg) != cudaSuccess ||
        clusters < 1) {
      cudaGetLastError();
      return FFT3D_ERR_UNSUPPORTED_SIZE;
    }
    cluster_blocks = std::min(clusters, m) * u.kernel.cluster;
  }
  std::vector<int> ldims(m);
  for (int l = 0; l < m; ++l) ldims[l] = p->dims[u.grids[l]];
  const std::vector<int> order = schedule_order(ldims);
  const int resident = per_sm * sms;
  int total_items = 0;
  const std::vector<SchedBlock> blocks = build_schedule(
      ldims, order, resident * u.kernel.items_in_flight, 0.4 * (double)l2_bytes,
      u.kernel.phase_items, &total_items);
  u.total_items = total_items;
  u.nblocks = (int)blocks.size();
  u.grid = cluster_blocks > 0 ? cluster_blocks : std::max(1, std::min(total_items, resident));

  // twiddles for every edge the kernel handles, concatenated in its order
  std::vector<float> tw(2 * (size_t)u.kernel.twiddle_entries);
  size_t off = 0;
  for (int i = 0; i < u.kernel.nsizes; ++i) {
    const int n = u.kernel.sizes[i];
    twiddle_table(n, u.kernel.tw_l1 ? u.kernel.tw_l1 : item_l1(n, u.kernel.prec), tw.data() + 2 * off);
    off += n;
  }
  int rc;
  if ((rc = upload(&u.d_tw, reinterpret_cast<const float2*>(tw.data()), tw.size() / 2))) return rc;
  if (u.kernel.prec && u.kernel.umma_b) {
    std::vector<uint16_t> b(8192);
    umma_b_table(u.kernel.prec, b.data());
    std::vector<uint32_t> words(4096);
    std::memcpy(words.data(), b.data(), sizeof(uint16_t) * b.size());
    if ((rc = upload(&u.d_frag, words.data(), words.size()))) return rc;
  } else if (u.kernel.prec) {
    std::vector<uint32_t> frag(tc::kFragWords);
    mma_fragments(u.kernel.prec, frag.data());
    if ((rc = upload(&u.d_frag, frag.data(), frag.size()))) return rc;
  }
  if ((rc = upload(&u.d_blocks, blocks.data(), blocks.size()))) return rc;
  if (!identity && (rc = upload(&u.d_map, u.grids.data(), u.grids.size()))) return rc;
  u.work_bytes = sizeof(unsigned) * (size_t)(1 + m);
  if (cudaMalloc(&u.d_work, u.work_bytes) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_ALLOC;
  }
  if (cudaMemset(u.d_work, 0, u.work_bytes) != cudaSuccess) return FFT3D_ERR_CUDA;
  return FFT3D_SUCCESS;
}

int finish_plan(fft3d_plan p) {
  int rc;
  if (cudaMalloc(&p->d_status, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_ALLOC;
  }
  if (cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess) return FFT3D_ERR_CUDA;
  if (p->mixed && (rc = upload(&p->d_off, p->offsets.data(), p->offsets.size()))) return rc;
  const bool identity = p->units.size() == 1;
  for (Unit& u : p->units)
    if ((rc = finish_unit(p, u, identity))) return rc;
  for (Unit& u : p->units_ptr)
    if ((rc = finish_unit(p, u, identity))) return rc;
  return FFT3D_SUCCESS;
}

void set_scale(fft3d_plan p, double points) {
  if (p->norm == FFT3D_NORM_BY_N) {
    p->scale = (float)(1.0 / points);
    p->do_scale = 1;
  } else if (p->norm == FFT3D_NORM_ORTHO) {
    p->scale = (float)(1.0 / std::sqrt(points));
    p->do_scale = 1;
  }
}

int validate_common(int precision, int direction, int norm, fft3d_plan* out_plan) {
  if (!out_plan) return FFT3D_ERR_NULL_PTR;
  *out_plan = nullptr;
  if (precision < FFT3D_FP32 || precision > FFT3D_FP8) return FFT3D_ERR_INVALID_ARG;
  if (direction != FFT3D_FORWARD && direction != FFT3D_INVERSE) return FFT3D_ERR_INVALID_ARG;
  if (norm < FFT3D_NORM_NONE || norm > FFT3D_NORM_ORTHO) return FFT3D_ERR_INVALID_ARG;
  return FFT3D_SUCCESS;
}

// General path: per chunk of grids, the x pass (in -> out), then y and z in
// place on out; a chunk's intermediate (at most 40% of L2 when the grids
// allow) stays in L2 between its passes.
int launch_general(fft3d_plan p, const float2* in, float2* out, cudaStream_t stream) {
  const long long grid_pts = (long long)p->nx * p->ny * p->nz;
  for (int c = 0; c < p->nchunks; ++c) {
    const int w = (c == p->nchunks - 1 && p->tail != p->chunk) ? 1 : 0;
    const long long off = (long long)c * p->chunk * grid_pts;
    const bool xy_ok =
        p->xy_fused
            ? launch_plane_pass(p->plane[w], in + off, out + off, stream) == cudaSuccess
            : launch_axis_pass(p->pass[0][w], in + off, out + off, stream) == cudaSuccess &&
                  launch_axis_pass(p->pass[1][w], out + off, out + off, stream) == cudaSuccess;
    if (!xy_ok || launch_axis_pass(p->pass[2][w], out + off, out + off, stream) != cudaSuccess) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
  }
  return FFT3D_SUCCESS;
}

int launch_unit(fft3d_plan p, const Unit& u, const float2* in, float2* out,
                const float2* const* in_ptrs, float2* const* out_ptrs, cudaStream_t stream) {
  {
    // ticket kernels start from zeroed counters; cluster and whole-grid
    // kernels use none
    if (u.kernel.cluster == 0 && u.kernel.uses_work &&
        cudaMemsetAsync(u.d_work, 0, u.work_bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
    FusedArgs a{};
    a.in = in;
    a.out = out;
    a.in_ptrs = in_ptrs;
    a.out_ptrs = out_ptrs;
    a.grid_off = p->d_off;
    a.grid_map = u.d_map;
    a.blocks = u.d_blocks;
    a.nblocks = u.nblocks;
    a.total_items = u.total_items;
    a.twiddles = u.d_tw;
    a.work = u.d_work;
    a.status = p->d_status;
    a.scale = p->scale;
    a.do_scale = p->do_scale;
    a.timeout_ns = p->timeout_ns;
    a.mma_frag = u.d_frag;
    a.ngrids = (int)u.grids.size();
    const cudaError_t e = u.use_maps && !in_ptrs
                              ? u.kernel.launch_maps(a, u.host_off.data(), u.grid, stream)
                              : u.kernel.launch(a, u.grid, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
  }
  return FFT3D_SUCCESS;
}

int launch(fft3d_plan p, const float2* in, float2* out, const float2* const* in_ptrs,
           float2* const* out_ptrs, cudaStream_t stream) {
  if (p->general) return launch_general(p, in, out, stream);
  const std::vector<Unit>& units = in_ptrs && !p->units_ptr.empty() ? p->units_ptr : p->units;
  if (!p->branches) {
    for (const Unit& u : units) {
      const int rc = launch_unit(p, u, in, out, in_ptrs, out_ptrs, stream);
      if (rc) return rc;
    }
    return FFT3D_SUCCESS;
  }
  // concurrent branches: every side stream waits for the caller's stream,
  // takes one unit (the smallest first, so that short launches find free
  // multiprocessors before the persistent ones take them all), and the
  // caller's stream waits for every branch; a captured graph records the
  // fork and joins as edges
  if (cudaEventRecord(p->fork, stream) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  int rc = FFT3D_SUCCESS;
  for (size_t i = units.size(); i-- > 0;) {
    if (cudaStreamWaitEvent(p->side[i], p->fork, 0) != cudaSuccess) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
    rc = launch_unit(p, units[i], in, out, in_ptrs, out_ptrs, p->side[i]);
    // a forked branch is joined even when its launch failed: the caller's
    // stream then still waits for every branch already launched, and a
    // capture does not end with an unjoined stream
    if (cudaEventRecord(p->join[i], p->side[i]) != cudaSuccess ||
        cudaStreamWaitEvent(stream, p->join[i], 0) != cudaSuccess) {
      cudaGetLastError();
      if (!rc) rc = FFT3D_ERR_CUDA;
    }
    if (rc) return rc;
  }
  return FFT3D_SUCCESS;
}

// W_L^m = exp(-2 pi i m / L), m < L, evaluated in FP64 by the host math
// library and rounded to nearest FP32: the twiddle table of the general
// path's passes.
void root_table(int L, float* out /* 2 * L */) {
  for (int m = 0; m < L; ++m) {
    const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)L;
    out[2 * m] = (float)std::cos(a);
    out[2 * m + 1] = (float)(-std::sin(a));
  }
}

// Plan of the general path: tables for each distinct edge, chunking by the
// L2 budget, the three passes prepared for a full chunk and for the tail.
int create_general(fft3d_plan p) {
  int rc;
  const int lens[3] = {p->nx, p->ny, p->nz};
  int tab_of[3];
  for (int a = 0; a < 3; ++a) {
    tab_of[a] = -1;
    for (size_t t = 0; t < p->tables.size(); ++t)
      if (p->tables[t].L == lens[a]) tab_of[a] = (int)t;
    if (tab_of[a] >= 0) continue;
    AxisTable t;
    t.L = lens[a];
    t.nst = axis_stages(t.L, t.radix);
    if (!t.nst) return FFT3D_ERR_UNSUPPORTED_SIZE;
    std::vector<float> tw(2 * (size_t)t.L);
    root_table(t.L, tw.data());
    std::vector<int> pos(t.L);
    axis_positions(t.L, t.nst, t.radix, pos.data());
    std::vector<unsigned short> pos16(pos.begin(), pos.end());
    p->tables.push_back(t);
    AxisTable& tt = p->tables.back();
    if ((rc = upload(&tt.d_tw, reinterpret_cast<const float2*>(tw.data()), (size_t)t.L))) return rc;
    if ((rc = upload(&tt.d_pos, pos16.data(), pos16.size()))) return rc;
    tab_of[a] = (int)p->tables.size() - 1;
  }
  int sms = 0, l2_bytes = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, p->device) != cudaSuccess)
    return FFT3D_ERR_CUDA;
  const long long nx = p->nx, ny = p->ny, nz = p->nz;
  const double grid_bytes = 8.0 * (double)(nx * ny * nz);
  long long chunk = (long long)(0.4 * (double)l2_bytes / grid_bytes);
  // a pass's tile count stays below 2^31 (every pass has fewer tiles than
  // pencils, at most max(ny nz, nz nx, ny nx) per grid)
  const long long cap = std::max(1LL, (1LL << 30) / std::max({ny * nz, nz * nx, ny * nx}));
  chunk = std::max(1LL, std::min({chunk, (long long)p->batch, cap}));
  p->chunk = (int)chunk;
  p->nchunks = (int)((p->batch + chunk - 1) / chunk);
  // x and y in one pass where a plane fits shared memory and holds enough
  // points for a block's iteration (measured: 64^3 x 256 0.20 -> 0.24,
  // 96 x 128 x 64 0.19 -> 0.24 of the roofline; 16^3 planes of 256 points
  // 0.22 -> 0.09, so small planes keep the separate passes' larger tiles)
  p->xy_fused = (long long)p->nx * p->ny >= 4096 && plane_pass_smem(p->nx, p->ny) != 0;
  p->tail = p->batch - (p->nchunks - 1) * p->chunk;
  for (int w = 0; w < 2; ++w) {
    const long long c = w == 0 ? p->chunk : p->tail;
    AxisGeom gx, gy, gz;
    gx.contiguous = 1;
    gx.rows = c * ny * nz;
    gy.outer = c * nz;  // (grid, z) slices: base = outer * ny * nx
    gy.nx = (int)nx;
    gy.d1 = 1;
    gy.s1 = ny * nx;
    gy.pi = nx;
    gz.outer = c * ny;  // (grid, y) slices: base = grid * nz ny nx + y nx
    gz.nx = (int)nx;
    gz.d1 = (int)ny;
    gz.s1 = nz * ny * nx;
    gz.s0 = nx;
    gz.pi = nx * ny;
    gz.scale = p->scale;
    gz.do_scale = p->do_scale;
    const AxisGeom* gs[3] = {&gx, &gy, &gz};
    for (int a = p->xy_fused ? 2 : 0; a < 3; ++a)
      if ((rc = prepare_axis_pass(p->tables[tab_of[a]], p->direction, *gs[a], sms, &p->pass[a][w])))
        return rc;
    if (p->xy_fused &&
        (rc = prepare_plane_pass(p->tables[tab_of[0]], p->tables[tab_of[1]], p->direction, c * nz,
                                 sms, &p->plane[w])))
      return rc;
  }
  return FFT3D_SUCCESS;
}

// Validated arguments -> plan (variant < 0: environment override, tuning
// cache, or the built-in default).
int create_uniform(int nx, int ny, int nz, int batch, int precision, int direction, int norm,
                   int variant, fft3d_plan* out_plan) {
  int rc;
  if ((rc = check_device())) return rc;
  const bool fused = nx == ny && ny == nz && fused_size(nx);
  if (!fused) {
    // the general path is the only one for these edges
    if (precision != FFT3D_FP32) return FFT3D_ERR_UNSUPPORTED_PRECISION;
    if (variant < 0) variant = kGeneralVariant;
    if (variant != kGeneralVariant) return FFT3D_ERR_INVALID_ARG;
  } else {
    if (variant < 0) variant = pick_variant(false, nx, batch, precision, direction, nullptr, 0);
    const std::vector<int> cand = variant_candidates(false, nx, precision);
    if (std::find(cand.begin(), cand.end(), variant) == cand.end()) return FFT3D_ERR_INVALID_ARG;
  }
  fft3d_plan p = new (std::nothrow) fft3d_plan_s();
  if (!p) return FFT3D_ERR_ALLOC;
  cudaGetDevice(&p->device);
  p->nx = nx; p->ny = ny; p->nz = nz; p->batch = batch;
  p->precision = precision; p->direction = direction; p->norm = norm;
  p->variant = variant;
  const long long pts = (long long)nx * ny * nz;
  p->dims.assign(batch, nx);
  p->offsets.resize(batch);
  for (int g = 0; g < batch; ++g) p->offsets[g] = (long long)g * pts;
  p->total_points = pts * batch;
  set_scale(p, (double)pts);
  if (variant == kGeneralVariant) {
    p->general = true;
    if (cudaMalloc(&p->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess)
      rc = FFT3D_ERR_ALLOC;
    else
      rc = create_general(p);
    if (rc) {
      cudaGetLastError();
      free_plan_buffers(p);
      delete p;
      return rc;
    }
    *out_plan = p;
    return FFT3D_SUCCESS;
  }
  Unit u;
  u.kernel = precision == FFT3D_FP32 ? fused_kernel_info(nx, direction, variant)
                                     : tc_kernel_info(nx, direction, precision, variant);
  u.grids.resize(batch);
  for (int g = 0; g < batch; ++g) u.grids[g] = g;
  p->units.push_back(u);
  rc = finish_plan(p);
  if (rc) {
    free_plan_buffers(p);
    delete p;
    return rc;
  }
  *out_plan = p;
  return FFT3D_SUCCESS;
}

int create_mixed(int count, const int* dims, int direction, int norm, int variant,
                 fft3d_plan* out_plan) {
  int rc;
  if ((rc = check_device())) return rc;
  if (variant < 0) variant = pick_variant(true, 0, count, FFT3D_FP32, direction, dims, count);
  if (variant < 0 || variant > 2) return FFT3D_ERR_INVALID_ARG;
  fft3d_plan p = new (std::nothrow) fft3d_plan_s();
  if (!p) return FFT3D_ERR_ALLOC;
  cudaGetDevice(&p->device);
  p->mixed = true;
  p->variant = variant;
  p->batch = count;
  p->precision = FFT3D_FP32; p->direction = direction; p->norm = norm;
  p->dims.assign(dims, dims + count);
  p->offsets.resize(count);
  long long off = 0;
  for (int g = 0; g < count; ++g) {
    p->offsets[g] = off;
    off += (long long)dims[g] * dims[g] * dims[g];
  }
  p->total_points = off;
  if (norm != FFT3D_NORM_NONE) {
    // one scale per plan: every grid must have the same edge
    const bool same =
        std::all_of(p->dims.begin(), p->dims.end(), [&](int d) { return d == p->dims[0]; });
    if (!same) {
      delete p;
      return FFT3D_ERR_INVALID_ARG;
    }
    set_scale(p, (double)p->dims[0] * p->dims[0] * p->dims[0]);
  }
  if (variant == 0) {
    Unit u;
    u.kernel = mixed_kernel_info(direction);
    u.grids.resize(count);
    for (int g = 0; g < count; ++g) u.grids[g] = g;
    p->units.push_back(u);
  } else {
    // one unit per distinct edge, largest edges first (variants 1 and 2)
    bool any_maps = false;
    std::vector<Unit> ptr_units;
    std::vector<int> edges(p->dims);
    std::sort(edges.begin(), edges.end(), std::greater<int>());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    for (int n : edges) {
      Unit u;
      for (int g = 0; g < count; ++g)
        if (p->dims[g] == n) u.grids.push_back(g);
      // the edge's default kernel.  The tensor-map kernels read a packed
      // batch: at 128^3 the split-y kernel (6) takes one pair of tensor maps
      // per grid with the launch (up to kMixMaps grids) on packed buffers,
      // and calls with pointer arrays use the warp-owned kernel (5) in a
      // unit of their own; at 64^3 (7, 8) the plain persistent kernel (0),
      // as fast at the grid counts of a mixed batch
      const int ng = (int)u.grids.size();
      int v = builtin_default_variant(false, n, ng, FFT3D_FP32);
      // the tensor-map kernels with per-grid maps: split-y (128^3) and the
      // thread-pair kernel (80^3, 96^3); for pointer arrays a kernel that
      // addresses grids through the plan's map
      const bool maps = (v == 6 || v == 13) && ng <= kMixMaps;
      const int v_ptr = n == 128 ? 5 : (n == 80 && ng >= 4) ? 4 : n == 32 ? 3 : 0;
      if ((n == 64 && (v == 7 || v == 8)) || ((v == 6 || v == 13) && !maps)) v = n == 64 ? 0 : v_ptr;
      u.kernel = fused_kernel_info(n, direction, v);
      Unit w = u;
      if (maps) {
        u.use_maps = true;
        for (int g : u.grids) u.host_off.push_back(p->offsets[g]);
        w.kernel = fused_kernel_info(n, direction, v_ptr);
        any_maps = true;
      }
      p->units.push_back(u);
      ptr_units.push_back(w);
    }
    if (any_maps) p->units_ptr = ptr_units;
  }
  if (variant == 2 && p->units.size() > 1) {
    p->branches = true;
    p->side.resize(p->units.size(), nullptr);
    p->join.resize(p->units.size(), nullptr);
    bool ok = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess;
    for (size_t i = 0; ok && i < p->units.size(); ++i)
      ok = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_plan_buffers(p);
      delete p;
      return FFT3D_ERR_CUDA;
    }
  }
  rc = finish_plan(p);
  if (rc) {
    free_plan_buffers(p);
    delete p;
    return rc;
  }
  *out_plan = p;
  return FFT3D_SUCCESS;
}

bool general_size(int n) {
  int r[kAxisMaxStages];
  return axis_stages(n, r) > 0;
}

int validate_uniform(int nx, int ny, int nz, int batch, int precision) {
  if (nx < 1 || ny < 1 || nz < 1 || batch < 1) return FFT3D_ERR_INVALID_ARG;
  if (batch > (1 << 24)) return FFT3D_ERR_INVALID_ARG;
  if (!(nx == ny && ny == nz && fused_size(nx))) {
    // general path: every edge 2..512 with prime factors 2, 3, 5; FP32
    if (!general_size(nx) || !general_size(ny) || !general_size(nz))
      return FFT3D_ERR_UNSUPPORTED_SIZE;
    if (precision != FFT3D_FP32) return FFT3D_ERR_UNSUPPORTED_PRECISION;
    if ((long long)nx * ny * nz * batch >= (1LL << 40)) return FFT3D_ERR_INVALID_ARG;
    return FFT3D_SUCCESS;
  }
  if (precision != FFT3D_FP32 && !tc_size(nx)) return FFT3D_ERR_UNSUPPORTED_PRECISION;
  // ticket counters are 32-bit: 2 * n items per grid
  if ((long long)batch * 2 * nx >= (1LL << 31)) return FFT3D_ERR_INVALID_ARG;
  return FFT3D_SUCCESS;
}

int validate_mixed(int count, const int* dims, int precision) {
  if (!dims) return FFT3D_ERR_NULL_PTR;
  if (count < 1 || count > FFT3D_MAX_MIXED_GRIDS) return FFT3D_ERR_INVALID_ARG;
  long long items = 0;
  for (int g = 0; g < count; ++g) {
    if (dims[g] < 1) return FFT3D_ERR_INVALID_ARG;
    if (!fused_size(dims[g])) return FFT3D_ERR_UNSUPPORTED_SIZE;
    items += 2LL * dims[g];
  }
  if (items >= (1LL << 31)) return FFT3D_ERR_INVALID_ARG;
  if (precision != FFT3D_FP32) return FFT3D_ERR_UNSUPPORTED_PRECISION;
  return FFT3D_SUCCESS;
}

}  // namespace

// Plan creation for the autotuner (tune.cu): a plan with a forced variant.
int fft3d_internal_create_variant(bool mixed, int nx, int batch, int precision, int direction,
                                  const int* dims, int count, int variant, fft3d_plan* out) {
  *out = nullptr;
  if (mixed) return create_mixed(count, dims, direction, FFT3D_NORM_NONE, variant, out);
  return create_uniform(nx, nx, nx, batch, precision, direction, FFT3D_NORM_NONE, variant, out);
}

// Host-buffer pipeline: chunks of `grids` grids go host -> device on one
// stream, through the chunk plan on a second, device -> host on a third, with
// two device buffers of each kind so that copies in both directions overlap
// the transforms of neighbouring chunks.
struct HostIO {
  fft3d_plan chunk = nullptr;  // plan for `grids` grids
  fft3d_plan tail = nullptr;   // plan for the last, shorter chunk (if any)
  int grids = 0;
  size_t grid_bytes = 0;
  void* in_buf[2] = {nullptr, nullptr};
  void* out_buf[2] = {nullptr, nullptr};
  cudaStream_t s_h2d = nullptr, s_cmp = nullptr, s_d2h = nullptr;
  cudaEvent_t in_ready[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
  cudaEvent_t start = nullptr, done = nullptr;
};

static void free_host_io(HostIO* h) {
  if (!h) return;
  fft3d_plan_destroy(h->chunk);
  fft3d_plan_destroy(h->tail);
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->in_buf[b]);
    cudaFree(h->out_buf[b]);
    if (h->in_ready[b]) cudaEventDestroy(h->in_ready[b]);
    if (h->in_free[b]) cudaEventDestroy(h->in_free[b]);
    if (h->out_ready[b]) cudaEventDestroy(h->out_ready[b]);
    if (h->out_free[b]) cudaEventDestroy(h->out_free[b]);
  }
  if (h->start) cudaEventDestroy(h->start);
  if (h->done) cudaEventDestroy(h->done);
  if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
  if (h->s_cmp) cudaStreamDestroy(h->s_cmp);
  if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
  delete h;
}

extern "C" {

int fft3d_plan_host_io(fft3d_plan plan, int chunk_grids) {
  if (!plan) return FFT3D_ERR_NULL_PTR;
  if (plan->mixed || chunk_grids < 1 || chunk_grids > plan->batch) return FFT3D_ERR_INVALID_ARG;
  if (plan->hio) {
    free_host_io(plan->hio);
    plan->hio = nullptr;
  }
  HostIO* h = new (std::nothrow) HostIO();
  if (!h) return FFT3D_ERR_ALLOC;
  const int nx = plan->nx, ny = plan->ny, nz = plan->nz;
  h->grids = chunk_grids;
  h->grid_bytes = sizeof(float2) * (size_t)nx * ny * nz;
  int rc = create_uniform(nx, ny, nz, chunk_grids, plan->precision, plan->direction, plan->norm,
                          plan->variant, &h->chunk);
  const int rem = plan->batch % chunk_grids;
  if (!rc && rem)
    rc = create_uniform(nx, ny, nz, rem, plan->precision, plan->direction, plan->norm,
                        plan->variant, &h->tail);
  const size_t bytes = h->grid_bytes * (size_t)chunk_grids;
  for (int b = 0; b < 2 && !rc; ++b)
    if (cudaMalloc(&h->in_buf[b], bytes) != cudaSuccess ||
        cudaMalloc(&h->out_buf[b], bytes) != cudaSuccess)
      rc = FFT3D_ERR_ALLOC;
  if (!rc &&
      (cudaStreamCreateWithFlags(&h->s_h2d, cudaStreamNonBlocking) != cudaSuccess ||
       cudaStreamCreateWithFlags(&h->s_cmp, cudaStreamNonBlocking) != cudaSuccess ||
       cudaStreamCreateWithFlags(&h->s_d2h, cudaStreamNonBlocking) != cudaSuccess))
    rc = FFT3D_ERR_CUDA;
  for (int b = 0; b < 2 && !rc; ++b)
    if (cudaEventCreateWithFlags(&h->in_ready[b], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->in_free[b], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->out_ready[b], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->out_free[b], cudaEventDisableTiming) != cudaSuccess)
      rc = FFT3D_ERR_CUDA;
  if (!rc && (cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess))
    rc = FFT3D_ERR_CUDA;
  if (rc) {
    cudaGetLastError();
    free_host_io(h);
    return rc;
  }
  plan->hio = h;
  return FFT3D_SUCCESS;
}

int fft3d_execute_host(fft3d_plan plan, const void* host_in, void* host_out, void* stream) {
  if (!plan || !host_in || !host_out) return FFT3D_ERR_NULL_PTR;
  HostIO* h = plan->hio;
  if (!h) return FFT3D_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const char* hin = static_cast<const char*>(host_in);
  char* hout = static_cast<char*>(host_out);
  bool ok = cudaEventRecord(h->start, s) == cudaSuccess &&
            cudaStreamWaitEvent(h->s_h2d, h->start, 0) == cudaSuccess &&
            cudaStreamWaitEvent(h->s_cmp, h->start, 0) == cudaSuccess &&
            cudaStreamWaitEvent(h->s_d2h, h->start, 0) == cudaSuccess;
  const int nchunks = (plan->batch + h->grids - 1) / h->grids;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int b = c & 1, g0 = c * h->grids, m = std::min(h->grids, plan->batch - g0);
    const size_t off = h->grid_bytes * (size_t)g0, bytes = h->grid_bytes * (size_t)m;
    fft3d_plan cp = m == h->grids ? h->chunk : h->tail;
    ok = (c < 2 || cudaStreamWaitEvent(h->s_h2d, h->in_free[b], 0) == cudaSuccess) &&
         cudaMemcpyAsync(h->in_buf[b], hin + off, bytes, cudaMemcpyHostToDevice, h->s_h2d) ==
             cudaSuccess &&
         cudaEventRecord(h->in_ready[b], h->s_h2d) == cudaSuccess &&
         cudaStreamWaitEvent(h->s_cmp, h->in_ready[b], 0) == cudaSuccess &&
         (c < 2 || cudaStreamWaitEvent(h->s_cmp, h->out_free[b], 0) == cudaSuccess) &&
         fft3d_execute(cp, h->in_buf[b], h->out_buf[b], h->s_cmp) == FFT3D_SUCCESS &&
         cudaEventRecord(h->in_free[b], h->s_cmp) == cudaSuccess &&
         cudaEventRecord(h->out_ready[b], h->s_cmp) == cudaSuccess &&
         cudaStreamWaitEvent(h->s_d2h, h->out_ready[b], 0) == cudaSuccess &&
         cudaMemcpyAsync(hout + off, h->out_buf[b], bytes, cudaMemcpyDeviceToHost, h->s_d2h) ==
             cudaSuccess &&
         cudaEventRecord(h->out_free[b], h->s_d2h) == cudaSuccess;
  }
  // the caller's stream continues after the last copy back (and after the
  // last transform, which every copy back follows)
  ok = ok && cudaEventRecord(h->done, h->s_d2h) == cudaSuccess &&
       cudaStreamWaitEvent(s, h->done, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  return FFT3D_SUCCESS;
}

}  // extern "C"

extern "C" {

int fft3d_size_supported(int n) { return fused_size(n) || general_size(n) ? 1 : 0; }

int fft3d_tc_operand_table(int precision, uint16_t* out) {
  if (!out) return FFT3D_ERR_NULL_PTR;
  if (precision < FFT3D_SPLIT_FP16 || precision > FFT3D_FP8) return FFT3D_ERR_INVALID_ARG;
  umma_b_table(precision, out);
  return FFT3D_SUCCESS;
}

int fft3d_twiddle_table(int n, float* out, int* l1, int* l2) {
  if (!out || !l1 || !l2) return FFT3D_ERR_NULL_PTR;
  if (!fused_size(n)) return FFT3D_ERR_UNSUPPORTED_SIZE;
  twiddle_table(n, split_l1(n), out);
  *l1 = split_l1(n);
  *l2 = split_l2(n);
  return FFT3D_SUCCESS;
}

int fft3d_schedule_preview(int count, const int* dims, int concurrency, double l2_budget_bytes,
                           int phase_items, int max_blocks, int* grid, int* phase, int* start,
                           int* nblocks, int* total_items) {
  if (!dims || !grid || !phase || !start || !nblocks || !total_items) return FFT3D_ERR_NULL_PTR;
  if (count < 1 || count > FFT3D_MAX_MIXED_GRIDS || concurrency < 0 || phase_items < 0 ||
      !(l2_budget_bytes >= 0.0) || max_blocks < 2 * count)
    return FFT3D_ERR_INVALID_ARG;
  std::vector<int> d(dims, dims + count);
  for (int e : d)
    if (e < 1 || e > 1024) return FFT3D_ERR_INVALID_ARG;
  int total = 0;
  const std::vector<SchedBlock> blocks =
      build_schedule(d, schedule_order(d), concurrency, l2_budget_bytes, phase_items, &total);
  for (size_t i = 0; i < blocks.size(); ++i) {
    grid[i] = blocks[i].grid;
    phase[i] = blocks[i].phase;
    start[i] = blocks[i].start;
  }
  *nblocks = (int)blocks.size();
  *total_items = total;
  return FFT3D_SUCCESS;
}

int fft3d_plan_create(int nx, int ny, int nz, int batch, int precision, int direction, int norm,
                      fft3d_plan* out_plan) {
  int rc = validate_common(precision, direction, norm, out_plan);
  if (rc) return rc;
  if ((rc = validate_uniform(nx, ny, nz, batch, precision))) return rc;
  return create_uniform(nx, ny, nz, batch, precision, direction, norm, -1, out_plan);
}

int fft3d_plan_create_mixed(int count, const int* dims, int precision, int direction, int norm,
                            fft3d_plan* out_plan) {
  int rc = validate_common(precision, direction, norm, out_plan);
  if (rc) return rc;
  if ((rc = validate_mixed(count, dims, precision))) return rc;
  return create_mixed(count, dims, direction, norm, -1, out_plan);
}

int fft3d_plan_variant(fft3d_plan plan, int* variant) {
  if (!plan || !variant) return FFT3D_ERR_NULL_PTR;
  *variant = plan->variant;
  return FFT3D_SUCCESS;
}

int fft3d_plan_grid_offset(fft3d_plan plan, int g, int64_t* offset) {
  if (!plan || !offset) return FFT3D_ERR_NULL_PTR;
  const int count = (int)plan->dims.size();
  if (g < 0 || g > count) return FFT3D_ERR_INVALID_ARG;
  *offset = g == count ? plan->total_points : plan->offsets[g];
  return FFT3D_SUCCESS;
}

int fft3d_execute(fft3d_plan plan, const void* in, void* out, void* stream) {
  if (!plan || !in || !out) return FFT3D_ERR_NULL_PTR;
  if (!aligned16(in) || !aligned16(out)) return FFT3D_ERR_MISALIGNED;
  return launch(plan, static_cast<const float2*>(in), static_cast<float2*>(out), nullptr, nullptr,
                static_cast<cudaStream_t>(stream));
}

int fft3d_execute_mixed(fft3d_plan plan, const void* const* in_ptrs, void* const* out_ptrs,
                        void* stream) {
  if (!plan || !in_ptrs || !out_ptrs) return FFT3D_ERR_NULL_PTR;
  if (!plan->mixed) return FFT3D_ERR_INVALID_ARG;
  return launch(plan, nullptr, nullptr, reinterpret_cast<const float2* const*>(in_ptrs),
                reinterpret_cast<float2* const*>(out_ptrs), static_cast<cudaStream_t>(stream));
}

int fft3d_get_device_status(fft3d_plan plan, void* stream) {
  if (!plan) return FFT3D_ERR_NULL_PTR;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  unsigned s = 0;
  if (cudaMemcpy(&s, plan->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(plan->d_status, 0, sizeof(unsigned)) != cudaSuccess)
    return FFT3D_ERR_CUDA;
  if (plan->hio) {  // the chunk plans of the host-buffer pipeline
    for (fft3d_plan cp : {plan->hio->chunk, plan->hio->tail})
      if (cp) {
        const int rc = fft3d_get_device_status(cp, plan->hio->s_cmp);
        if (rc == FFT3D_ERR_DEVICE_TIMEOUT) s = kStatusTimeout;
        else if (rc != FFT3D_SUCCESS) return rc;
      }
  }
  return s == kStatusOk ? FFT3D_SUCCESS : FFT3D_ERR_DEVICE_TIMEOUT;
}

int fft3d_plan_destroy(fft3d_plan plan) {
  if (!plan) return FFT3D_SUCCESS;
  free_host_io(plan->hio);
  plan->hio = nullptr;
  free_plan_buffers(plan);
  delete plan;
  return FFT3D_SUCCESS;
}

const char* fft3d_error_string(int code) {
  switch (code) {
    case FFT3D_SUCCESS: return "success";
    case FFT3D_ERR_INVALID_ARG: return "invalid argument";
    case FFT3D_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case FFT3D_ERR_NULL_PTR: return "null pointer";
    case FFT3D_ERR_MISALIGNED: return "data pointer not 16-byte aligned";
    case FFT3D_ERR_CUDA: return "CUDA runtime error";
    case FFT3D_ERR_DEVICE_TIMEOUT: return "bounded device-side wait timed out";
    case FFT3D_ERR_ALLOC: return "allocation failed";
    case FFT3D_ERR_NO_DEVICE: return "no compute capability 10.3 device";
    case FFT3D_ERR_UNSUPPORTED_PRECISION: return "precision unsupported for this plan";
    case FFT3D_ERR_EXCEEDS_STATIC_SCRATCH: return "batch exceeds the static scratch of fft3d_execute_noalloc";
    default: return "unknown error code";
  }
}

int fft3d_selftest_wait_timeout(int64_t timeout_ns) {
  if (timeout_ns <= 0 || timeout_ns > 10000000000LL) return FFT3D_ERR_INVALID_ARG;
  int rc = check_device();
  if (rc) return rc;
  unsigned* buf = nullptr;
  if (cudaMalloc(&buf, 2 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_ALLOC;
  }
  unsigned host[2] = {0u, 0u};
  rc = FFT3D_ERR_CUDA;
  if (cudaMemset(buf, 0, 2 * sizeof(unsigned)) == cudaSuccess &&
      launch_wait_selftest(buf, buf + 1, (long long)timeout_ns, nullptr) == cudaSuccess &&
      cudaDeviceSynchronize() == cudaSuccess &&
      cudaMemcpy(host, buf, sizeof(host), cudaMemcpyDeviceToHost) == cudaSuccess)
    rc = host[1] == kStatusTimeout ? FFT3D_ERR_DEVICE_TIMEOUT : FFT3D_SUCCESS;
  cudaGetLastError();
  cudaFree(buf);
  return rc;
}

}  // extern "C"
