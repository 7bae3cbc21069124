// fft3d_execute_noalloc: the batched cubic transform without a plan and
// without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// transform: a solver loop whose host framework hands out all device memory
// up front and forbids cudaMalloc afterwards (cudaMalloc can synchronise the
// device and can fail under memory pressure), or code running where no
// allocation call is permitted.  For them this entry point keeps everything
// the persistent kernel needs besides the caller's input and output -- the
// work counters, the ticket schedule, the twiddle table and the status word
// -- in one file-scope device array of fixed size, which every GPU that
// loads this library holds until the process exits.
//
// The kernels are the same ones the planned path launches; only where their
// scratch lives differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "fft3d.h"
#include "internal.h"
#include "sizes.h"

namespace fft3d {
namespace {

constexpr size_t kNoallocScratchBytes = 160 * 1024;
constexpr int kMaxDevices = 64;

// Layout inside the array (byte offsets, 256-aligned regions):
//   [0, 256)                status word
//   [256, 256 + 4*(1+B))    ticket counter and per-grid plane counters
//   then 2*B schedule blocks, then the twiddle table (n complex)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch
  int sms = 0;
  size_t l2 = 0;
  int per_sm[2][kNumFusedSizes] = {};  // occupancy per (direction, size), 0 = not queried
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// Host staging for the schedule and the twiddles; copied to the device array
// with cudaMemcpyAsync from pageable memory, which returns once the bytes
// are staged, so the buffers can be reused by the next call.
SchedBlock g_host_blocks[2 * FFT3D_NOALLOC_MAX_BATCH];
int g_plane_end[FFT3D_NOALLOC_MAX_BATCH];
float g_host_tw[2 * 128];

// The planner's ticket order for `batch` grids of edge n, written without
// heap storage: plane blocks grid after grid; grid g's slab block once
// `concurrency` more tickets have been handed out after its last plane
// ticket, or earlier when the grids still waiting for their slabs would
// exceed `l2_budget` bytes.  Grids leave that waiting set in FIFO order, so
// it is the index range [head, next).  Returns the number of blocks.
int uniform_schedule(int n, int batch, int concurrency, double l2_budget, SchedBlock* out,
                     int* total_items) {
  const double bytes = 8.0 * n * n * n;
  int start = 0, nb = 0, head = 0;
  double pending = 0.0;
  auto emit = [&](int g, int phase) {
    out[nb++] = SchedBlock{g, phase, start, n};
    start += n;
  };
  auto flush = [&](int next, bool force_one) {
    while (head < next) {
      if (start - g_plane_end[head] < concurrency && !force_one) break;
      force_one = false;
      pending -= bytes;
      emit(head++, 1);
    }
  };
  for (int g = 0; g < batch; ++g) {
    while (head < g && pending + bytes > l2_budget) flush(g, true);
    emit(g, 0);
    g_plane_end[g] = start;
    pending += bytes;
    flush(g + 1, false);
  }
  while (head < batch) flush(batch, true);
  *total_items = start;
  return nb;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t scratch_need(int n, int batch, size_t* off_work, size_t* off_blocks, size_t* off_tw) {
  *off_work = 256;
  *off_blocks = align256(*off_work + sizeof(unsigned) * (size_t)(1 + batch));
  *off_tw = align256(*off_blocks + sizeof(SchedBlock) * (size_t)(2 * batch));
  return *off_tw + sizeof(float2) * (size_t)n;
}

}  // namespace
}  // namespace fft3d

using namespace fft3d;

extern "C" int fft3d_execute_noalloc(int n, int batch, int direction, int norm, const void* in,
                                     void* out, void* stream) {
  if (!in || !out) return FFT3D_ERR_NULL_PTR;
  if ((reinterpret_cast<uintptr_t>(in) & 15u) || (reinterpret_cast<uintptr_t>(out) & 15u))
    return FFT3D_ERR_MISALIGNED;
  if (direction != FFT3D_FORWARD && direction != FFT3D_INVERSE) return FFT3D_ERR_INVALID_ARG;
  if (norm < FFT3D_NORM_NONE || norm > FFT3D_NORM_ORTHO) return FFT3D_ERR_INVALID_ARG;
  if (fused_slot(n) < 0) return FFT3D_ERR_UNSUPPORTED_SIZE;
  if (batch < 1) return FFT3D_ERR_INVALID_ARG;
  size_t off_work, off_blocks, off_tw;
  if (batch > FFT3D_NOALLOC_MAX_BATCH ||
      scratch_need(n, batch, &off_work, &off_blocks, &off_tw) > kNoallocScratchBytes)
    return FFT3D_ERR_EXCEEDS_STATIC_SCRATCH;

  int dev = -1, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_NO_DEVICE;
  }
  if (major != 10 || minor != 3) return FFT3D_ERR_NO_DEVICE;

  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& st = g_dev[dev];
  // One-time set-up on this device, with it current: the device address of
  // the array (its host-side name is only a stand-in) and the SM count.
  if (!st.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
    int sms = 0, l2 = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
    st.base = static_cast<unsigned char*>(p);
    st.sms = sms;
    st.l2 = (size_t)l2;
    st.ready = true;
  }

  const KernelInfo k = fused_kernel_info(n, direction, n == 128 ? 2 : 0);
  const int di = direction < 0 ? 0 : 1, si = fused_slot(n);
  if (st.per_sm[di][si] == 0) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.func, k.threads, k.smem) !=
            cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      return FFT3D_ERR_CUDA;
    }
    st.per_sm[di][si] = per_sm;
  }
  const int resident = st.per_sm[di][si] * st.sms;

  // schedule and twiddles (FP64 host values rounded to FP32), as a plan does
  int total_items = 0;
  const int nblocks = uniform_schedule(n, batch, resident * k.items_in_flight, 0.4 * (double)st.l2,
                                       g_host_blocks, &total_items);
  int l1 = 0, l2 = 0;
  if (fft3d_twiddle_table(n, g_host_tw, &l1, &l2) != FFT3D_SUCCESS) return FFT3D_ERR_CUDA;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = st.base;
  // the counters and the status word must start at zero on every call
  if (cudaMemsetAsync(base, 0, off_blocks, s) != cudaSuccess ||
      cudaMemcpyAsync(base + off_blocks, g_host_blocks, sizeof(SchedBlock) * (size_t)nblocks,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + off_tw, g_host_tw, sizeof(float2) * (size_t)n,
                      cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }

  FusedArgs a{};
  a.in = static_cast<const float2*>(in);
  a.out = static_cast<float2*>(out);
  a.blocks = reinterpret_cast<const SchedBlock*>(base + off_blocks);
  a.nblocks = nblocks;
  a.total_items = total_items;
  a.twiddles = reinterpret_cast<const float2*>(base + off_tw);
  a.work = reinterpret_cast<unsigned*>(base + off_work);
  a.status = reinterpret_cast<unsigned*>(base);
  const double pts = (double)n * n * n;
  if (norm == FFT3D_NORM_BY_N) {
    a.scale = (float)(1.0 / pts);
    a.do_scale = 1;
  } else if (norm == FFT3D_NORM_ORTHO) {
    a.scale = (float)(1.0 / std::sqrt(pts));
    a.do_scale = 1;
  } else {
    a.scale = 1.0f;
  }
  a.timeout_ns = kDefaultWaitNs;
  a.ngrids = batch;
  const int grid = std::max(1, std::min(total_items, resident));
  if (k.launch(a, grid, s) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  return FFT3D_SUCCESS;
}
