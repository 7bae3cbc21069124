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
// scratch lives differs.  A call enqueues two kernels and nothing else: a
// set-up kernel that clears the counters and the status word and writes the
// schedule and the twiddle table into the array (both computed on the host
// and handed over as kernel parameters), then the transform.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "fft3d.h"
#include "internal.h"
#include "schedule.h"
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

// Host storage of the schedule builder (shared with the planner), reused by
// every call under g_mu.
SchedBlock g_host_blocks[2 * FFT3D_NOALLOC_MAX_BATCH];
int g_dims[FFT3D_NOALLOC_MAX_BATCH];
int g_order[FFT3D_NOALLOC_MAX_BATCH];
int g_plane_end[FFT3D_NOALLOC_MAX_BATCH];

// What the set-up kernel writes.  A uniform batch's schedule is fixed by
// the phase of each block: plane blocks come in grid order, slab blocks in
// grid order too (a grid's slabs follow its planes, first in, first out),
// and every block is n tickets.  So block i is grid "number of blocks of
// its phase before i" and starts at ticket i * n; bit i of `phase` holds
// its phase.
constexpr int kPhaseWords = 2 * FFT3D_NOALLOC_MAX_BATCH / 32;
struct SetupArgs {
  unsigned phase[kPhaseWords];
  float2 tw[128];
  int n, batch, nblocks;
  unsigned work_words;  // ticket counter and per-grid plane counters
  size_t off_work, off_blocks, off_tw;
};

// One block of kPhaseWords threads: thread t expands the 32 blocks of word
// t (an exclusive prefix count of slab bits over the words gives the grid
// numbers), copies twiddles, and clears the counters and the status word.
__global__ void __launch_bounds__(kPhaseWords) noalloc_setup_kernel(const SetupArgs s) {
  __shared__ int before[kPhaseWords];
  const int t = threadIdx.x;
  const unsigned w = s.phase[t];
  before[t] = __popc(w);
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int i = 0; i < kPhaseWords; ++i) {
      const int c = before[i];
      before[i] = acc;
      acc += c;
    }
  }
  __syncthreads();
  SchedBlock* blocks = reinterpret_cast<SchedBlock*>(g_noalloc_scratch + s.off_blocks);
  for (int j = 0; j < 32; ++j) {
    const int i = 32 * t + j;
    if (i >= s.nblocks) break;
    const int slabs_before = before[t] + __popc(w & ((1u << j) - 1u));
    const int phase = (w >> j) & 1u;
    blocks[i] = SchedBlock{phase ? slabs_before : i - slabs_before, phase, i * s.n, s.n};
  }
  float2* tw = reinterpret_cast<float2*>(g_noalloc_scratch + s.off_tw);
  for (int i = t; i < s.n; i += blockDim.x) tw[i] = s.tw[i];
  unsigned* work = reinterpret_cast<unsigned*>(g_noalloc_scratch + s.off_work);
  for (unsigned i = t; i < s.work_words; i += blockDim.x) work[i] = 0u;
  if (t == 0) *reinterpret_cast<unsigned*>(g_noalloc_scratch) = kStatusOk;
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

  const KernelInfo k = fused_kernel_info(n, direction, 0);
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

  // schedule (the planner's builder) and twiddles (FP64 host values rounded
  // to FP32), as a plan computes them, handed to the set-up kernel by value
  static SetupArgs su;  // under g_mu; copied into the launch
  for (int g = 0; g < batch; ++g) {
    g_dims[g] = n;
    g_order[g] = g;  // equal edges: the planner's largest-first order is the grid order
  }
  int total_items = 0;
  const int nblocks = schedule_blocks(batch, g_dims, g_order, resident * k.items_in_flight,
                                      0.4 * (double)st.l2, 0, g_plane_end, g_host_blocks,
                                      &total_items);
  std::memset(su.phase, 0, sizeof(su.phase));
  for (int i = 0; i < nblocks; ++i)
    if (g_host_blocks[i].phase) su.phase[i >> 5] |= 1u << (i & 31);
  int l1 = 0, l2 = 0;
  if (fft3d_twiddle_table(n, reinterpret_cast<float*>(su.tw), &l1, &l2) != FFT3D_SUCCESS)
    return FFT3D_ERR_CUDA;
  su.n = n;
  su.batch = batch;
  su.nblocks = nblocks;
  su.work_words = (unsigned)(1 + batch);
  su.off_work = off_work;
  su.off_blocks = off_blocks;
  su.off_tw = off_tw;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = st.base;
  noalloc_setup_kernel<<<1, kPhaseWords, 0, s>>>(su);
  if (cudaGetLastError() != cudaSuccess) return FFT3D_ERR_CUDA;

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

extern "C" int fft3d_noalloc_get_device_status(void* stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return FFT3D_ERR_NO_DEVICE;
  }
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  const DeviceState& st = g_dev[dev];
  if (!st.ready) return FFT3D_SUCCESS;  // no call on this device yet
  unsigned w = 0;
  if (cudaMemcpy(&w, st.base, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(st.base, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return FFT3D_ERR_CUDA;
  }
  return w == kStatusOk ? FFT3D_SUCCESS : FFT3D_ERR_DEVICE_TIMEOUT;
}
