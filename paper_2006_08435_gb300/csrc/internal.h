// Host/device structures shared by the planner (plan.cu) and the kernel
// translation units.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fft3d.h"

namespace fft3d {

// Device status word values (sticky until read by fft3d_get_device_status).
constexpr unsigned kStatusOk = 0u;
constexpr unsigned kStatusTimeout = 1u;

// Default limit of one inter-block wait (nanoseconds of %globaltimer).
constexpr long long kDefaultWaitNs = 2000000000LL;

// One run of consecutive work items: all plane items (phase 0: x then y
// transform of plane z = i) or all slab items (phase 1: z transform of the
// slab y = i) of one grid.  Items [start, start + n) of the global ticket
// sequence, i = ticket - start.
struct SchedBlock {
  int grid;
  int phase;
  int start;
  int n;  // edge of that grid (cubic), also the number of items
};

struct FusedArgs {
  const float2* in;             // packed input base (unused when in_ptrs)
  float2* out;                  // packed output base (unused when out_ptrs)
  const float2* const* in_ptrs; // device array of per-grid inputs, or null
  float2* const* out_ptrs;      // device array of per-grid outputs, or null
  const long long* grid_off;    // per-grid element offsets, or null (g * n^3)
  const int* grid_map;          // local grid -> plan grid index, or null (identity)
  const SchedBlock* blocks;
  int nblocks;
  int total_items;
  const float2* twiddles;       // concatenated tables in kernel size order
  unsigned* work;               // [0] ticket, [1 + g] plane items done for grid g
  unsigned* status;             // sticky status word
  float scale;                  // output scale of the last pass
  int do_scale;
  long long timeout_ns;
  const uint32_t* mma_frag;     // tensor-core B fragments (split precisions), or null
  int ngrids;                   // grids of the launch unit
  float2* aux;                  // a kernel's own workspace (real grids: Nyquist columns), or null
};

using LaunchFn = cudaError_t (*)(const FusedArgs&, int grid, cudaStream_t);
// Launch of a unit of a mixed-edge plan on packed buffers with per-grid
// tensor maps (at most kMixMaps grids, passed with the launch): host_off[l]
// = element offset of the unit's grid l.
constexpr int kMixMaps = 32;
using LaunchMapsFn = cudaError_t (*)(const FusedArgs&, const long long* host_off, int grid,
                                     cudaStream_t);

struct KernelInfo {
  LaunchFn launch = nullptr;
  const void* func = nullptr;   // for occupancy / attributes
  int threads = 0;
  size_t smem = 0;              // dynamic shared memory bytes
  int twiddle_entries = 0;      // complex entries in the concatenated table
  int sizes[8] = {0};           // edges handled, in table order
  int nsizes = 0;
  int items_in_flight = 1;      // work items a block holds at once (schedule lag)
  int prec = 0;                 // 0 FP32, else fft3d_precision of the tensor-core kinds
  int cluster = 0;              // > 0: cluster kernel of this many blocks per cluster
  int tw_l1 = 0;                // twiddle table split n = l1 * (n / l1); 0: item_l1(n, prec)
  int phase_items = 0;          // work items per phase of a grid; 0: the grid's edge
  int umma_b = 0;               // mma_frag holds the tcgen05 B table (tcgen.cuh), not mma.sync fragments
  int uses_work = 1;            // 0: no ticket counters (nothing to clear before a launch)
  LaunchMapsFn launch_maps = nullptr;  // mixed-edge units on packed buffers (tensor-map kernels)
  const void* func_maps = nullptr;     // its kernel
};

// ---------------------------------------------------------------- general path
// Pencil passes for any edge 2..kAxisMaxLen with prime factors 2, 3, 5, one
// axis at a time (axis.cu).
constexpr int kAxisMaxLen = 512;
constexpr int kGeneralVariant = 10;  // plan variant of the general path
constexpr int kAxisMaxStages = 12;

// n / d = (hi32(n * mul) + n) >> shift for every n < 2^32 (make_fastdiv).
struct FastDiv {
  unsigned mul;
  int shift;
};
FastDiv make_fastdiv(unsigned d);

// One pencil length, planned on the host: the radices of its
// decimation-in-frequency stages and the device tables (W_L^m, m < L, FP64
// rounded to FP32; the position each output K holds after the stages).
struct AxisTable {
  int L = 0, nst = 0;
  int radix[kAxisMaxStages] = {};
  float2* d_tw = nullptr;
  unsigned short* d_pos = nullptr;
};
int axis_stages(int L, int* radix);                              // 0: not plannable
void axis_positions(int L, int nst, const int* radix, int* pos);  // pos[K], K < L

// Which pencils a pass transforms.  contiguous: `rows` rows of L points
// packed back to back (the x pass).  Strided: for each of `outer` slices,
// the nx pencils at base + x (x < nx), element i at + i * pi, with
// base = (outer / d1) * s1 + (outer % d1) * s0.
struct AxisGeom {
  int contiguous = 0;
  long long rows = 0;
  long long outer = 0;
  int nx = 0, d1 = 1;
  long long s1 = 0, s0 = 0, pi = 0;
  float scale = 1.0f;
  int do_scale = 0;
};

// Kernel arguments of one pass (axis.cu).
struct AxisArgs {
  const float2* in;  // may equal out (a tile is read before it is written)
  float2* out;
  const float2* tw;
  const unsigned short* pos;
  int L, nst, W, lw;  // W = 2^lw pencils per tile
  int radix[kAxisMaxStages], span[kAxisMaxStages], sub[kAxisMaxStages], twst[kAxisMaxStages];
  FastDiv divsub[kAxisMaxStages];  // division by sub[t], the span M of a stage's sub-blocks
  FastDiv divL;
  int swsh, swmask;  // tile slot of (i, c): i * (W + 1) + (c ^ ((i >> swsh) & swmask))
  int contiguous;
  unsigned ntiles;
  long long rows;
  long long outer;     // strided: slices in all
  int nx, xtiles, d1;  // strided: tile -> (slice group, x0 = 16 * (tile % xtiles))
  FastDiv divx, divd1;
  long long s1, s0, pi;
  float scale;
  int do_scale;
};
// The x and y passes fused for planes that fit shared memory (axis.cu):
// one nx x ny plane per block at a time, x stages over its rows, y stages
// over its columns, one read and one write of the plane.
struct AxisStages {
  int L, nst;
  int radix[kAxisMaxStages], span[kAxisMaxStages], sub[kAxisMaxStages], twst[kAxisMaxStages];
  FastDiv divsub[kAxisMaxStages];
};
struct PlaneArgs {
  const float2* in;
  float2* out;
  const float2 *twx, *twy;
  const unsigned short *posx, *posy;
  AxisStages sx, sy;
  int nx, ny, px;      // row pitch px: odd, >= nx
  int rsh, rmask;      // element x of a row sits at x ^ ((x >> rsh) & rmask)
  FastDiv divnx, divny;
  unsigned nplanes;
};
struct PlaneLaunch {
  PlaneArgs args{};
  int dir = -1;
  int grid = 0, threads = 0;
  size_t smem = 0;
};
// Shared memory a plane pass of an nx x ny plane needs (0 if it does not fit).
size_t plane_pass_smem(int nx, int ny);
int prepare_plane_pass(const AxisTable& tx, const AxisTable& ty, int dir, long long planes, int sms,
                       PlaneLaunch* out);
cudaError_t launch_plane_pass(const PlaneLaunch& l, const float2* in, float2* out,
                              cudaStream_t stream);

struct AxisLaunch {
  AxisArgs args{};
  int dir = -1;
  int nbuf = 1;  // tile buffers per block
  int grid = 0;
  size_t smem = 0;
};
int prepare_axis_pass(const AxisTable& tab, int dir, const AxisGeom& g, int sms, AxisLaunch* out);
cudaError_t launch_axis_pass(const AxisLaunch& l, const float2* in, float2* out, cudaStream_t stream);

// Defined in the inst_*.cu translation units.
KernelInfo fused_kernel_info(int n, int dir, int variant);   // single-size kernel
KernelInfo mixed_kernel_info(int dir);          // all fused sizes
KernelInfo tc_kernel_info(int n, int dir, int prec, int variant);  // tensor-core kinds
KernelInfo real_kernel_info(int n, int dir);    // real grids (rgrid.cuh); launch null: none
cudaError_t launch_wait_selftest(unsigned* flag, unsigned* status, long long timeout_ns,
                                 cudaStream_t stream);

// Variant choice at plan creation (tune.cu): FFT3D_VARIANT / FFT3D_MIXED_VARIANT
// override; else the FFT3D_TUNE_CACHE entry for this device and problem;
// else, with FFT3D_TUNE=1, tune now (and record); else the built-in default.
int pick_variant(bool mixed, int n, int batch, int precision, int direction, const int* dims,
                 int count);
std::vector<int> variant_candidates(bool mixed, int n, int precision);
int builtin_default_variant(bool mixed, int n, int batch, int precision);

}  // namespace fft3d

// A plan with a forced variant (plan.cu), for the autotuner.
int fft3d_internal_create_variant(bool mixed, int nx, int batch, int precision, int direction,
                                  const int* dims, int count, int variant, fft3d_plan* out);
