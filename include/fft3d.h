/*
 * fft3d.h -- C ABI of the GB300 (sm_103a) 3D complex-to-complex FFT library.
 *
 * The operation (the paper, section "Approach", Eq. 1):
 *
 *   F(kx,ky,kz) = sum_{z<nz} sum_{y<ny} sum_{x<nx}
 *                   f(x,y,z) * W_nx^(x*kx) * W_ny^(y*ky) * W_nz^(z*kz),
 *   W_n = exp(s * 2*pi*i / n),  s = -1 (FFT3D_FORWARD) or +1 (FFT3D_INVERSE),
 *
 * computed, as the same section decomposes it, as 1D FFTs along x, then y,
 * then z.  Eq. 1 prints per-axis roots W_x, W_y, W_z; each axis uses the root
 * of its own length.
 *
 * Data layout (every entry point): interleaved single-precision complex
 * (re, im float pairs, 8 bytes per point), index ((b*nz + z)*ny + y)*nx + x,
 * x fastest, grids of one batch packed back to back.  Natural order on input
 * and output (the paper's FPGA pipeline streams bit-reversed data
 * internally; that ordering never reaches this interface).
 *
 * Pointers: `in`/`out` are DEVICE pointers owned by the caller, 16-byte
 * aligned, valid for the whole grid set.  `in == out` (in place) is allowed;
 * other overlaps are not.  (Kernels whose work items cover part of a plane,
 * such as the 128^3 half-plane items, order an item's stores after the
 * loads of the items that read the same rows.)  A plan owns the device memory it allocates at
 * create (twiddle tables, schedule, work counters, status word) and frees it
 * at destroy.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).
 *
 * Errors: every function returns 0 on success or one of the negative
 * FFT3D_ERR_* codes below; no C++ exception crosses this boundary.  Execute
 * calls are asynchronous: a device-side failure (a bounded wait that ran
 * out) is recorded in the plan's status word and reported by
 * fft3d_get_device_status.
 *
 * Threads: a plan may be executed from one stream at a time; executes that
 * overlap on the device on different streams share the plan's work counters
 * and race.  Different plans are independent.
 */
#ifndef FFT3D_H
#define FFT3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft3d_plan_s* fft3d_plan;

/* Arithmetic of the butterflies.  Input/output stay complex64 in all. */
typedef enum {
  FFT3D_FP32 = 0,        /* plain single precision (the paper's FP64->FP32 step, Abstract/Results) */
  FFT3D_SPLIT_FP16 = 1,  /* radix-16 stages on tensor cores, hi+lo FP16 operands, FP32 accumulate */
  FFT3D_SPLIT_BF16 = 2,  /* same with BF16 hi+lo operands */
  FFT3D_FP16 = 3,        /* radix-16 stages on tensor cores, FP16 hi only (reported, not gated) */
  /* Custom precisions (the paper's closing paragraph names custom-precision
   * floating-point units as future work): operand formats of the tcgen05
   * kernels only (64^3 and 128^3, variant 9), each with one power-of-two
   * exponent per 64-point pencil; reported, not gated. */
  FFT3D_BFP16 = 4,       /* block floating point: 11-bit fixed-point mantissas in FP16, B = hi + lo */
  FFT3D_SPLIT_FP8 = 5,   /* E4M3 hi + lo operands, three products (kind::f8f6f4) */
  FFT3D_FP8 = 6          /* E4M3 operands, one product */
} fft3d_precision;

/* Sign of the exponent of W (Eq. 1 uses -1). */
typedef enum { FFT3D_FORWARD = -1, FFT3D_INVERSE = 1 } fft3d_direction;

/* Output scaling: none, 1/(nx*ny*nz), or 1/sqrt(nx*ny*nz). */
typedef enum { FFT3D_NORM_NONE = 0, FFT3D_NORM_BY_N = 1, FFT3D_NORM_ORTHO = 2 } fft3d_norm;

enum {
  FFT3D_SUCCESS = 0,
  FFT3D_ERR_INVALID_ARG = -1,      /* a count, enum or plan handle is out of range */
  FFT3D_ERR_UNSUPPORTED_SIZE = -2, /* an edge the library does not plan (see fft3d_size_supported) */
  FFT3D_ERR_NULL_PTR = -3,         /* a required pointer is NULL */
  FFT3D_ERR_MISALIGNED = -4,       /* a data pointer is not 16-byte aligned */
  FFT3D_ERR_CUDA = -5,             /* a CUDA runtime call or kernel launch failed */
  FFT3D_ERR_DEVICE_TIMEOUT = -6,   /* a bounded device-side wait ran out (status word) */
  FFT3D_ERR_ALLOC = -7,            /* device or host allocation failed at plan create */
  FFT3D_ERR_NO_DEVICE = -8,        /* no CUDA device, or not compute capability 10.3 */
  FFT3D_ERR_UNSUPPORTED_PRECISION = -9, /* precision not available for this plan's sizes */
  FFT3D_ERR_EXCEEDS_STATIC_SCRATCH = -10 /* fft3d_execute_noalloc: batch above FFT3D_NOALLOC_MAX_BATCH */
};

/* Largest number of grids in one mixed plan. */
#define FFT3D_MAX_MIXED_GRIDS 4096

/*
 * 1 if an edge length n can be planned on every axis, else 0.  Host only,
 * needs no GPU.  Supported: 2 <= n <= 512 with prime factors 2, 3 and 5.
 * Cubic grids of edge 16, 32, 48, 64, 80, 96 or 128 have fused single-launch
 * kernels (and the tensor-core precisions at 64 and 128); every other grid,
 * cubic or not (nx, ny, nz each supported), runs on the general path: one
 * pencil pass per axis (FP32).
 */
int fft3d_size_supported(int n);

/*
 * Host-only view of the general path's 1D plan for edge n (needs no GPU):
 * the radices R_0 .. R_(s-1) (product n) of its decimation-in-frequency
 * stages, *nstages = s <= 12, and the digit-reversal map: after the stages
 * output K = k_0 + R_0 (k_1 + R_1 (k_2 + ...)), k_t < R_t, sits at position
 * pos[K] = sum_t k_t * n / (R_0 ... R_t) of the pencil.  radix holds 12
 * ints, pos n ints.  Errors: FFT3D_ERR_NULL_PTR, FFT3D_ERR_UNSUPPORTED_SIZE
 * (n outside 2..512 or with a prime factor above 5).
 */
int fft3d_axis_digit_map(int n, int* nstages, int* radix, int* pos);

/*
 * Host-only view of the planner's split and twiddle table for edge n (needs
 * no GPU).  *l1, *l2 receive the split n = L1*L2 of the four-step 1D
 * transform; out[2*(k2*L1 + n1)] and out[2*(k2*L1 + n1) + 1] receive re and
 * im of W_n^(n1*k2) = exp(-2 pi i ((n1*k2) mod n) / n), evaluated in FP64 by
 * the host math library and rounded to nearest FP32 (the table the kernels
 * use).  `out` holds 2*n floats.  Returns FFT3D_ERR_UNSUPPORTED_SIZE for an
 * edge without a fused kernel.
 */
int fft3d_twiddle_table(int n, float* out, int* l1, int* l2);

/*
 * Host-only view of the planner's ticket schedule (needs no GPU): the order
 * in which the persistent kernels hand out work items.  Each grid g of
 * edge dims[g] has a plane phase (x and y; planes or half-planes) and a slab
 * phase (z); each phase is one block of `phase_items` consecutive tickets
 * (dims[g] tickets when phase_items is 0).  Grids are taken largest edge
 * first; a grid's slab block follows its plane block once `concurrency`
 * more tickets have been emitted (the items resident at once), or earlier
 * when the intermediates of the grids whose planes are done but whose slabs
 * are not yet scheduled would exceed `l2_budget_bytes` (8 n^3 bytes each).
 * A slab item waits only on plane items of its own grid, which hold smaller
 * tickets, so the schedule cannot deadlock.  Plans call this with
 * concurrency = resident blocks x items in flight per block and 40% of L2.
 *   count      : 1 .. FFT3D_MAX_MIXED_GRIDS grids; dims: HOST array, 1..1024.
 *   max_blocks : capacity of grid/phase/start (>= 2 * count).
 *   grid, phase, start : HOST arrays receiving block i's grid, phase (0
 *                plane, 1 slab) and first ticket; *nblocks = 2 * count;
 *                *total_items = tickets in all.
 * Errors: FFT3D_ERR_NULL_PTR, FFT3D_ERR_INVALID_ARG.
 */
int fft3d_schedule_preview(int count, const int* dims, int concurrency, double l2_budget_bytes,
                           int phase_items, int max_blocks, int* grid, int* phase, int* start,
                           int* nblocks, int* total_items);

/*
 * Host-only view of the B operands of the tcgen05 tensor-core kernels
 * (variant 9; needs no GPU).  For k1 = 0..3, the 32 x 32 real form of the
 * complex 16 x 16 matrix M_k1[n2][k2] = W_64^(n2 (k1 + 4 k2)) (forward root,
 * the radix-16 stage of a 64-point DFT split n = 16 n1 + n2, k = k1 + 4 k2,
 * with the split's twiddles folded in): entry (kk = 2 n2 + c, nn = 2 k2 + d)
 * is Re w for (c, d) = (0, 0) and (1, 1), Im w for (0, 1), -Im w for (1, 0),
 * w = M_k1[n2][k2].  Halfword ((term * 4 + k1) * 2048 + ((nn / 8) * 4 +
 * kk / 8) * 128 + (nn % 8) * 16 + (kk % 8) * 2) / 2 of `out` holds term 0
 * hi = rn(b) and term 1 lo = rn(b - hi) of entry b, each rounded once from
 * its FP64 value to FP16 (precision FFT3D_SPLIT_FP16 or FFT3D_FP16) or BF16
 * (FFT3D_SPLIT_BF16).  `out` holds 8192 halfwords.  FFT3D_BFP16 uses the
 * FP16 table.  FFT3D_SPLIT_FP8 / FFT3D_FP8: byte (term * 4 + k1) * 1024 +
 * ((nn / 8) * 2 + kk / 16) * 128 + (nn % 8) * 16 + kk % 16 of `out` (the
 * first 8 KB; the rest is zero) holds the E4M3 code of hi = rn(16 b)
 * (term 0) and lo = rn(16 b - hi) (term 1), rounded to nearest even with
 * saturation.  Errors: FFT3D_ERR_NULL_PTR, FFT3D_ERR_INVALID_ARG (precision
 * FFT3D_FP32 or out of range).
 */
int fft3d_tc_operand_table(int precision, uint16_t* out);

/*
 * Plan `batch` grids of nx*ny*nz points (Eq. 1 per grid).
 *   nx, ny, nz : edge lengths, each fft3d_size_supported (non-cubic grids
 *                and edges without a fused kernel take the general path).
 *   batch      : number of grids, >= 1, packed back to back.
 *   precision  : fft3d_precision; the tensor-core kinds (SPLIT_FP16,
 *                SPLIT_BF16, FP16, BFP16, SPLIT_FP8, FP8) are planned for
 *                cubic n = 64 and 128 (FFT3D_ERR_UNSUPPORTED_PRECISION
 *                otherwise).
 *   direction  : FFT3D_FORWARD or FFT3D_INVERSE.
 *   norm       : fft3d_norm.
 *   out_plan   : receives the handle (set to NULL on failure).
 * Validates every argument BEFORE touching the GPU, so argument errors are
 * reported on machines without one.  Allocates the plan's device buffers on
 * the current device; the plan must be executed on that device.
 */
int fft3d_plan_create(int nx, int ny, int nz, int batch, int precision,
                      int direction, int norm, fft3d_plan* out_plan);

/*
 * Plan `count` cubic grids of different edges dims[g] (g < count) that are
 * transformed together in one persistent launch (mixed radix 2/3/5).
 *   count : 1..FFT3D_MAX_MIXED_GRIDS.
 *   dims  : HOST array of `count` edge lengths.
 * Grid g's points live at element offset fft3d_plan_grid_offset(plan, g)
 * of the packed buffers given to fft3d_execute, or at the pointers given to
 * fft3d_execute_mixed.  precision must be FFT3D_FP32.
 */
int fft3d_plan_create_mixed(int count, const int* dims, int precision,
                            int direction, int norm, fft3d_plan* out_plan);

/* Element offset (in complex points) of grid g inside the packed buffers,
 * written to *offset.  Total packed size for g == count. */
int fft3d_plan_grid_offset(fft3d_plan plan, int g, int64_t* offset);

/*
 * Transform all grids of the plan: out = F(in) (scaled per norm).
 *   in, out : device pointers to the packed grids (see layout above).
 *   stream  : cudaStream_t or NULL.
 * Asynchronous, allocates nothing, never synchronises, and is capturable in
 * a CUDA graph (per launch unit a memset node for its work counters, when
 * its kernel uses them, and a kernel node; mixed variant 2 puts the units
 * on the plan's side streams between event fork and join nodes).
 */
int fft3d_execute(fft3d_plan plan, const void* in, void* out, void* stream);

/*
 * Mixed plans only: like fft3d_execute, but grid g is read from in_ptrs[g]
 * and written to out_ptrs[g].  `in_ptrs` and `out_ptrs` are DEVICE arrays of
 * `count` device pointers that must stay valid until the launch completes.
 */
int fft3d_execute_mixed(fft3d_plan plan, const void* const* in_ptrs,
                        void* const* out_ptrs, void* stream);

/*
 * Prepare a single-edge plan for fft3d_execute_host: a chunk plan of
 * `chunk_grids` grids (and one for the shorter last chunk), two device input
 * and two device output buffers of chunk_grids grids each, three internal
 * streams and their events.  All allocated here, freed by
 * fft3d_plan_destroy; calling it again replaces them.  The paper measures
 * the host <-> accelerator transfer next to the transform (Table 1); this
 * overlaps the two.
 */
int fft3d_plan_host_io(fft3d_plan plan, int chunk_grids);

/*
 * Transform `batch` grids that live in HOST memory: host_in and host_out are
 * host pointers to the packed grids (page-locked memory for asynchronous
 * copies; pageable memory works but the copies then serialise with the
 * host).  Chunks are copied in, transformed and copied out on the plan's
 * internal streams so that both copy directions and the transforms overlap.
 * Ordered after prior work on `stream`; `stream` waits for the last copy
 * back, so synchronising `stream` means host_out is complete.  Requires
 * fft3d_plan_host_io; allocates nothing.
 */
int fft3d_execute_host(fft3d_plan plan, const void* host_in, void* host_out, void* stream);

/*
 * Synchronise `stream`, then read and clear the plan's device status word.
 * Returns FFT3D_SUCCESS, FFT3D_ERR_DEVICE_TIMEOUT (a bounded inter-block
 * wait ran out; the affected outputs are undefined) or FFT3D_ERR_CUDA.
 */
int fft3d_get_device_status(fft3d_plan plan, void* stream);

/* Release the plan's device memory.  NULL is accepted. */
int fft3d_plan_destroy(fft3d_plan plan);

/* Static English description of an error code. */
const char* fft3d_error_string(int code);

/*
 * Launch one block that waits on a flag nobody sets, with the same bounded
 * wait the persistent kernel uses between its passes, and return what that
 * wait reports: FFT3D_ERR_DEVICE_TIMEOUT when the wait gave up after
 * `timeout_ns` (the expected result), FFT3D_SUCCESS if the flag was seen.
 * Synchronises the device.  Exists so the timeout path can be tested without
 * hanging or faulting the GPU.
 */
int fft3d_selftest_wait_timeout(int64_t timeout_ns);

/*
 * The kernel variant a plan uses (written to *variant).  Single-edge FP32
 * plans (each variant the fastest for some edge and batch on the GB300):
 * 0 plain persistent kernel, 1 the same with twice the threads per block
 * (16^3 .. 96^3), 3 the cluster-fused single-pass kernel (16^3, 32^3), 12
 * a whole 16^3 grid per block (three passes of thread-per-pencil 16-point
 * DFTs in shared memory, no work counters), 4
 * the double-buffered persistent kernel (32^3, 48^3, 80^3, 96^3), 5 the
 * warp-owned two-phase kernel (64^3, 128^3), 7 the thread-per-pencil
 * kernel (each 1D FFT in one thread's registers, items loaded by swizzled
 * tensor TMA; 64^3), 8 the same with two-plane items and a register split
 * (64^3); for 128^3, 6 is the split-y kernel (64 KB items: half-planes and
 * quarter-slabs, 128-point FFTs by thread pairs); 13 the thread-pair plane
 * kernel (32^3 .. 96^3: whole planes and slabs by tensor TMA, every
 * n-point pencil in a pair of threads).  The tensor-TMA variants (64^3: 7,
 * 8; 128^3: 6; 32^3, 48^3, 80^3, 96^3: 13) need packed, 16-byte aligned buffers of one
 * batch (they encode tensor maps of `in` and `out` at each execute).
 * Tensor-core precision plans (64^3, 128^3): 0 the plain persistent kernel
 * (mma.sync radix-16 stage), 9 the tensor-TMA items with tcgen05 products,
 * operands and accumulators in tensor memory (64^3 two-plane, 128^3
 * split-y; all of a multiprocessor's tensor memory, one block per
 * multiprocessor), with the buffer requirements of the tensor-TMA FP32
 * variants; the block-floating-point and FP8 kinds exist on 9 only.  10:
 * the general path (every plan that is not cubic with a fused edge;
 * selectable for those too): per chunk of grids that fits 40% of L2, the x
 * pass (in -> out) and the y and z passes in place on out, each a batched
 * 1D transform of the pencils of one axis in shared-memory tiles (mixed
 * radices 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16; fft3d_axis_digit_map);
 * where a plane of at least 4096 points fits shared memory, x and y run as
 * one plane pass (two launches per chunk instead of three).  Mixed plans:
 * 0 one launch of the mixed-edge kernel, 1 one launch per distinct edge (the
 * tensor-TMA kernels of 128^3 and 32^3 .. 96^3 take one pair of
 * tensor maps per grid, up to 32 grids of an edge; an edge whose default is
 * a tensor-TMA kernel otherwise takes variant 0 at 32^3 .. 96^3
 * (4 at 80^3 from 4 grids) and 5 at 128^3, as do calls with pointer
 * arrays), 2 the
 * launches of 1 as concurrent branches: the plan's own side streams, one
 * per edge, wait on the caller's stream and the caller's stream waits on
 * each of them (in a captured graph, parallel branches between a fork and
 * a join).
 * At create the variant comes from FFT3D_VARIANT / FFT3D_MIXED_VARIANT if
 * set, else from the tuning cache named by FFT3D_TUNE_CACHE (tuned on the
 * spot when FFT3D_TUNE=1 and the entry is missing), else a built-in default.
 */
int fft3d_plan_variant(fft3d_plan plan, int* variant);

/* Milliseconds per execute of `variant`, or a negative value if it failed. */
typedef double (*fft3d_tune_timer)(int variant, void* ctx);

/*
 * Autotuner core, usable without a GPU: if the JSON file `cache_path` (may
 * be NULL) maps `key` to one of `candidates`, return it (*from_cache = 1,
 * timer not called).  Otherwise time every candidate with `timer`, pick the
 * fastest (ties: first), skip failed ones (FFT3D_ERR_CUDA if all failed) and
 * record the choice in the file (atomic rewrite; unreadable entries are
 * dropped).  from_cache may be NULL.
 */
int fft3d_tune_select(const char* key, int ncand, const int* candidates,
                      fft3d_tune_timer timer, void* ctx, const char* cache_path,
                      int* best_variant, int* from_cache);

/*
 * Time the variants of a (n^3 x batch, precision, direction) plan on the
 * current device with CUDA events (allocates two temporary buffers of the
 * problem's size), record the fastest under a key of device name, SM count
 * and problem in `cache_path` (may be NULL), and return it.
 */
int fft3d_autotune(int n, int batch, int precision, int direction, const char* cache_path,
                   int* best_variant);

/* Same for a mixed plan of `count` cubic grids of edges dims[g]. */
int fft3d_autotune_mixed(int count, const int* dims, int direction, const char* cache_path,
                         int* best_variant);

/*
 * ---------------------------------------------------------------------------
 * Plane-wave Hartree energy, the use of the 3D FFT in plane-wave DFT that the
 * paper accelerates (sections "Introduction" and "Results"; the formulas are
 * the standard Gaussian-and-plane-wave ones, which the paper does not print).
 * Cubic periodic cell of side L (bohr), volume Omega = L^3, n^3 grid,
 * G = (2 pi / L) m with m_d = k_d for k_d < n/2 and k_d - n otherwise, G = 0
 * excluded (neutralising background).  With F = forward transform (Eq. 1,
 * unnormalised) and s = Omega 4 pi / (n^6 (2 pi / L)^2):
 *   E_H = (Omega/2) sum_{G!=0} 4 pi |F(rho)(G)/n^3|^2 / |G|^2
 *       = (s/2) sum_{m!=0} |F(rho)(m)|^2 / |m|^2,
 *   dE_H/drho = Re F^H( s F(rho) / |m|^2 ).
 * The energy and seed kernels each run one wave of the blocks the device
 * holds at once: the first call of each of the four entry points in a
 * process asks the runtime for that kernel's occupancy (with the call's
 * device current), so make it before any stream capture.  Later calls
 * allocate nothing, never synchronise and are capturable (the energy: a
 * memset of its counters and one kernel; the seed: one kernel).
 * ---------------------------------------------------------------------------
 */

/* Bytes of device workspace fft3d_hartree_energy needs (0 on bad args). */
size_t fft3d_hartree_workspace_bytes(int n, int batch);

/*
 * energy[b] = E_H of grid b, for `batch` spectra rhohat = F(rho) (device,
 * complex64, batch * n^3 points, 8-byte aligned).  Each term formed in FP32
 * (relative error below 6 * 2^-24), eight at a time summed in FP32, those
 * sums accumulated in FP64 in an order fixed by (n, batch) and the device
 * (bit-reproducible from call to call).  energy: DEVICE array of `batch`
 * doubles.
 * workspace: DEVICE buffer of at least fft3d_hartree_workspace_bytes(n,
 * batch) bytes, owned by the caller; it may be reused by later calls on the
 * same stream.  Asynchronous on `stream`.
 */
int fft3d_hartree_energy(const void* rhohat, int n, int batch, double L,
                         double* energy, void* workspace, size_t workspace_bytes,
                         void* stream);

/*
 * Backward seed of E_H: seed[b] = grad_energy[b] * s * rhohat[b] / |m|^2
 * (0 at m = 0), complex64, so that Re F^H(seed) (fft3d with
 * FFT3D_INVERSE, unnormalised) is grad_energy[b] * dE_H/drho.
 * grad_energy: DEVICE array of `batch` doubles.  All pointers device,
 * 8-byte aligned.
 */
int fft3d_hartree_seed(const void* rhohat, int n, int batch, double L,
                       const double* grad_energy, void* seed, void* stream);

/*
 * The same two steps on HALF spectra, for real densities (n even): rhohat_half
 * and seed_half are the half spectra kx = 0 .. n/2 of fft3d_real_execute's
 * layout (batch * n * n * (n/2 + 1) complex64 points, index
 * (kz*n + ky)*(n/2 + 1) + kx).  Since F(rho)(-k) = conj F(rho)(k) for a
 * real rho, the energy counts every point with 0 < kx < n/2 twice (its
 * mirror is not stored) and the points kx = 0, n/2 once: the same E_H as
 * fft3d_hartree_energy on the full spectrum, from about half the reads.
 * The seed is Hermitian as well, so the real inverse transform of
 * seed_half (fft3d_real_execute, FFT3D_INVERSE, unnormalised) is
 * grad_energy[b] * dE_H/drho.  workspace: as for fft3d_hartree_energy (its
 * size covers both).  FFT3D_ERR_INVALID_ARG for odd n.
 */
int fft3d_hartree_energy_half(const void* rhohat_half, int n, int batch, double L,
                              double* energy, void* workspace, size_t workspace_bytes,
                              void* stream);
int fft3d_hartree_seed_half(const void* rhohat_half, int n, int batch, double L,
                            const double* grad_energy, void* seed_half, void* stream);

/* out[i] = (re[i], 0) for i < count (device float -> complex64). */
int fft3d_real_to_complex(const float* re, void* out, int64_t count, void* stream);

/* re[i] = Re in[i] for i < count (device complex64 -> float). */
int fft3d_complex_to_real(const void* in, float* re, int64_t count, void* stream);

/*
 * ---------------------------------------------------------------------------
 * Real grids (a real density, the setting of the paper's plane-wave DFT
 * application, section "Introduction").  For a real grid f, Eq. 1 gives
 * F(-k) = conj(F(k)) (indices modulo n), so the forward transform returns the
 * HALF spectrum kx = 0 .. n/2 and the inverse takes one.
 *
 * Layouts: a real grid is n^3 floats, index (z*n + y)*n + x; a half spectrum
 * is n*n*(n/2 + 1) complex64 points, index (kz*n + ky)*(n/2 + 1) + kx; grids
 * of a batch are packed back to back.
 *
 * Forward: out = the half spectrum of F(in) (unnormalised, or scaled per
 * norm).  Inverse: out = Re of the inverse transform of the Hermitian
 * extension of the half spectrum `in` (bins above n/2 taken as conj(X(-k)));
 * for a half spectrum of a real grid that is n^3 times the grid (norm NONE),
 * and for any other input the imaginary parts of the self-mirrored bins
 * (kx, ky, kz each 0 or n/2) drop out.  `in` is not modified.
 *
 * At n = 16, 32, 64 and 128 in FP32 the transforms run as dedicated kernels:
 * each real row of n points is transformed as n/2 complex points and split
 * into its half spectrum (the even and odd samples' transforms,
 * X[k] = E[k] + W_n^k O[k]),
 * so the y and z transforms run on n/2 (+ 1) columns; at n = 16 and 32 one
 * block transforms a whole grid, at 64 and 128 one pass runs over the real
 * grids and one over the half spectra; each grid's error is relative to
 * itself.
 * Elsewhere two grids of the batch share one complex transform (c = a + i b;
 * the pair is separated with the symmetry above), so a grid's rounding error
 * is relative to the larger of its pair; cost per pair: a packing pass, one
 * complex transform of the plan's precision, a separating pass.
 * ---------------------------------------------------------------------------
 */
typedef struct fft3d_real_plan_s* fft3d_real_plan;

/*
 * Plan `batch` real transforms of n^3 grids.
 *   n         : even and fft3d_size_supported (FFT3D_ERR_UNSUPPORTED_SIZE
 *               otherwise).
 *   batch     : 1 .. 2^24 grids.
 *   precision : as for fft3d_plan_create (tensor-core kinds at n = 64, 128).
 *   direction : FFT3D_FORWARD (real -> half spectrum) or FFT3D_INVERSE
 *               (half spectrum -> real).
 *   norm      : fft3d_norm (1/n^3 or 1/sqrt(n^3) on the output).
 * Validates its arguments before touching the GPU.  Owns its device memory,
 * allocated here and freed by fft3d_real_plan_destroy: at n = 64 and 128
 * in FP32 a schedule, counters and (forward) batch * n * n/2 complex64
 * points of workspace, at n = 16 and 32 a status word only; elsewhere a complex plan of ceil(batch/2) grids and a workspace
 * of ceil(batch/2) * n^3 complex64 points.  The environment variable
 * FFT3D_REAL_PATH=pairs selects the pair scheme everywhere (for testing).
 */
int fft3d_real_plan_create(int n, int batch, int precision, int direction, int norm,
                           fft3d_real_plan* out_plan);

/*
 * Transform every grid of the plan.  `in` and `out` are DEVICE pointers,
 * 16-byte aligned, not overlapping (forward: in = real grids, out = half
 * spectra; inverse: the other way round).  Asynchronous on `stream`,
 * allocates nothing, capturable in a CUDA graph (one kernel at n = 16 and
 * 32, a counter reset and one kernel at n = 64 and 128 in FP32; elsewhere a packing
 * or rebuilding kernel, the complex plan's launch, a separating or splitting
 * kernel).  A plan may run
 * on one stream at a time.
 */
int fft3d_real_execute(fft3d_real_plan plan, const void* in, void* out, void* stream);

/* As fft3d_get_device_status, for the plan's complex transform. */
int fft3d_real_get_device_status(fft3d_real_plan plan, void* stream);

/* Release the plan's complex plan and workspace.  NULL is accepted. */
int fft3d_real_plan_destroy(fft3d_real_plan plan);

/* Largest batch fft3d_execute_noalloc accepts. */
#define FFT3D_NOALLOC_MAX_BATCH 4096

/*
 * The batched cubic transform for callers that cannot allocate device
 * memory when they need it -- for example a solver loop whose framework
 * hands out all device memory up front and forbids cudaMalloc later (it can
 * synchronise the device and can fail under memory pressure).  The paper has
 * no counterpart; this is a deployment convenience.
 *
 * Computes what a plan from fft3d_plan_create(n, n, n, batch, FFT3D_FP32,
 * direction, norm) followed by fft3d_execute(plan, in, out, stream) computes,
 * with the same kernels, but creates no plan and calls no cudaMalloc,
 * cudaFree or other allocating routine.  The kernels' scratch (work
 * counters, ticket schedule, twiddle table, status word) lives in one
 * file-scope device array of 160 KiB that every GPU which loads this library
 * holds until the process exits.
 *   n         : edge, one of 16, 32, 48, 64, 80, 96, 128.
 *   batch     : 1 .. FFT3D_NOALLOC_MAX_BATCH grids; larger batches return
 *               FFT3D_ERR_EXCEEDS_STATIC_SCRATCH.
 *   direction, norm, in, out, stream : as for fft3d_plan_create/execute.
 * Each call enqueues two kernels on `stream`: a set-up kernel that clears
 * the counters and the status word and writes the schedule and twiddle
 * table (computed on the host, passed as kernel parameters), then the
 * transform; nothing is copied between host and device.  The first call on
 * a device looks up the array's device address (and the kernel's
 * occupancy) with that device current; make that first call before any
 * stream capture.  Every call on a device shares the one array and rewrites
 * it, so calls whose work overlaps on the GPU -- on different streams, or
 * from different host threads -- race.  Host threads are serialised inside
 * the call.  A bounded wait that times out is recorded in the array's
 * status word; fft3d_noalloc_get_device_status reads it.
 */
int fft3d_execute_noalloc(int n, int batch, int direction, int norm,
                          const void* in, void* out, void* stream);

/*
 * Status of the last fft3d_execute_noalloc call on the current device:
 * synchronises `stream` (the stream of that call), then reads and clears the
 * status word in the library's device array.  Returns FFT3D_SUCCESS (also
 * when no call has run on this device), FFT3D_ERR_DEVICE_TIMEOUT (a bounded
 * inter-block wait ran out; that call's outputs are undefined) or
 * FFT3D_ERR_CUDA.  Allocates nothing.
 */
int fft3d_noalloc_get_device_status(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFT3D_H */
