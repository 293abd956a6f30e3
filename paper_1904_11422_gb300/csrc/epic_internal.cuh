// epic_internal.cuh -- plan layout and kernel launchers shared by the .cu files
// of libepic.so.  Not part of the public ABI (include/epic.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/epic.h"

namespace epic {

// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum.
// The attribute belongs to the function, not to a plan, so it is never set to
// one plan's need: a later, smaller plan would then lower it under the launches
// (and captured graphs) of a larger one.  Each launch still asks for its own size.
template <class Fn>
cudaError_t allow_max_smem(Fn fn) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  return e;
}

// Device-side error word values (written by kernels, read by epic_sync).
enum : int { kDevOk = 0, kDevTimeout = 1, kDevBadIndex = 2, kDevOffGrid = 3 };

// Per-CTA channel spans: CTA b of an imaging launch owns the work units
// [b*W, min((b+1)*W, C*T)) of the channel-major (c, t) index u = c*T + t.
struct WorkSplit {
  int ctas;        // CTAs of the launch
  long long units; // C * T
  long long W;     // units per CTA
  int T;
  int spans;       // partial-image slots per CTA used by this call (ctas * spans fits the workspace)
};

// The split of an imaging call: units u = c*T + t (channel-major) in equal
// contiguous ranges, one per CTA (at most `cap` CTAs, or the plan's own cap),
// no CTA left empty; spans = the most channels any CTA touches.  split_fits
// says whether the split's (CTA, span) slots fit the plan's workspace.
int spans_needed(const WorkSplit& ws);
struct Plan;
WorkSplit split_work_cap(const Plan& p, int T, int cap);
WorkSplit split_work(const Plan& p, int T);
bool split_fits(const Plan& p, const WorkSplit& ws);

// Gather tables of a gridder (see epic_gather.cu).
enum : int { kLayoutFft64 = 0, kLayoutFft32 = 1, kLayoutPair64 = 3, kLayoutFft128 = 4,
             kLayoutPairQ = 5, kLayoutPairD = 6, kLayoutFft64Q = 7 };
// Layouts whose table set 4 c + q gathers the 128 x 128 grid of channel c folded
// into the 64 x 64 field H_q of output-parity subset q.
__host__ __device__ inline bool layout_folded(int layout) { return layout == kLayoutPairQ || layout == kLayoutFft64Q; }
// Position of entry k of lane `lane` in the (warp, slot) range starting at
// `base`.  The FFT kernels' layouts (kFft64, kFft32, kFft64Q) walk entries two at
// a time and store each lane's entries 2j and 2j + 1 side by side, so that one
// 32-bit load fetches both antennas and one 8-byte load both weights:
// base + 64 (k / 2) + 2 lane + k % 2 (base and every trip count are even).  The
// other layouts keep entry k of every lane together: base + 32 k + lane.
__host__ __device__ inline bool layout_paired(int layout) {
  return layout == kLayoutFft64 || layout == kLayoutFft32 || layout == kLayoutFft64Q;
}
__host__ __device__ inline size_t entry_pos(int layout, size_t base, int k, int lane) {
  return layout_paired(layout) ? base + 64 * (size_t)(k >> 1) + 2 * lane + (k & 1) : base + 32 * (size_t)k + lane;
}
struct GatherTables {
  int layout = 0, threads = 0;
  int max_chan_entries = 0;      // padded entries of the largest channel
  int* d_cnt = nullptr;          // [C][warps][slots] trip count of (warp, slot); 8 slots, 16 at N = 128
  int* d_base = nullptr;         // [C][warps][slots] first entry of (warp, slot) within the channel
  int* d_chan_off = nullptr;     // [C+1] first entry of each channel
  uint16_t* d_task = nullptr;    // [C][threads] task of each thread ([C][threads][4] pairs for kLayoutPair64)
  uint16_t* d_ent_a = nullptr;   // [entries] antenna index (0 for padding)
  float* d_ent_w = nullptr;      // [entries] kernel weight (0 for padding)
};

struct Plan {
  // descriptor copy
  int A, P, C, N, S, xform, subtract;
  int vq = 1;  // virtual channels per channel: 4 for the tensor path at N = 128 (output-parity subsets)
  int dec = 1; // 2 for the tensor path at N = 32: a 64 x 64 transform of the zero-padded grid, even pixels kept
  double cell_lambda, sigma;
  int device, sm_count;

  // plan constants, generated on the GPU in FP64 (Sec. 3.2)
  double* d_ant_xy = nullptr;   // [A][2]
  double* d_freq = nullptr;     // [C]
  double* d_gains = nullptr;    // [C][A][P][2] (or null)
  double* d_delays = nullptr;   // [A][P] (or null)
  int* d_box = nullptr;         // [C][A][2] kernel box origin (i0, j0)
  double* d_wx = nullptr;       // [C][A][S] normalised 1-D kernel factors along x
  double* d_wy = nullptr;       // [C][A][S] along y
  float2* d_coef = nullptr;     // [C][A][P] calibration coefficient k (FP32)
  double2* d_coef64 = nullptr;  // [C][A][P] the same in FP64
  double2* d_dphase = nullptr;  // [C][A][P] delay phase exp(-2 pi i nu tau) alone (FP64)
  float* d_kx2 = nullptr;       // [C][A][N] |FT of w_x|^2 per output column
  float* d_ky2 = nullptr;       // [C][A][N] |FT of w_y|^2 per output row
  float* d_beam = nullptr;      // [C][N][N] kernel imprint (1/A) sum_a |W_a|^2
  int* d_csr_ptr = nullptr;     // [C][N*N+1] gather table: cell -> entries
  int2* d_csr_ent = nullptr;    // [C][A*S*S] (antenna, weight bits), antenna order
  float2* d_twiddle = nullptr;  // [N] exp(+2 pi i m / N)
  uint16_t* d_fmat = nullptr;   // tensor path: real DFT matrix, hi/lo 16-bit, shared-memory image (64 KB)
  float* d_dscale = nullptr;    // FP16 tensor path: [C * vq][4] power-of-two scales (fields, stage 1, squares)
  int* d_status = nullptr;      // device error word
  GatherTables gt;              // gridder's lane-interleaved gather tables

  // imaging launch shape and its workspace (partial images per CTA span)
  int ctas = 0, threads = 0, spans = 0, ent_in_smem = 0;
  unsigned unpack_warps = 0;  // FP32 64 x 64: the four warps that unpack each next sample early (0: none)
  int ctas_use = 0;  // CTAs an imaging launch may use (0: ctas); set by the batch autotuner
  size_t smem = 0;
  float* d_part = nullptr;      // [ctas][spans][4][N][N]
  float2* d_xbuf = nullptr;     // N = 128 FP32 path: row exchange between the two CTAs of each cluster
  int* d_part_auto = nullptr;   // [ctas][spans][A][4] exact integer self powers
  size_t device_bytes = 0, workspace_bytes = 0;

  // optional per-launch timing (epic_timing_enable)
  struct Timed {
    int kind;
    cudaEvent_t start, stop;
  };
  bool timing = false;
  std::vector<std::string> kinds;
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<long long> kind_launches;
  std::vector<double> kind_ms;

  // epic_grad workspace (FP32 plans of the fft_image kernel: N = 32 with A <= 128,
  // N = 64 and folded N = 128 with A <= 512)
  bool grad_ok = false;
  float2* d_gcoef = nullptr;     // [C][A][P] coefficients g * delay phase of the call
  double2* d_gcoef64 = nullptr;  // [C][A][P] the same in FP64
  float* d_gimage = nullptr;     // [C][4][N][N] forward image of the call
  float* d_resid = nullptr;      // [C][2][N][N] R = 2 (I - M) for XX, YY
  double* d_loss_part = nullptr; // [C] per-channel loss
  float2* d_gpart = nullptr;     // [ctas][spans][A][P] per-CTA sums of conj(e~) D

  // staging for epic_image_host
  uint8_t* d_stage_in = nullptr;
  size_t stage_in_bytes = 0;
  float* d_stage_out = nullptr;

  // epic_image_host_async: two staging slots used alternately, a stream for the
  // input copies and one for the result copies, and per slot the events that
  // order each buffer's reuse (input copied, imaged, result copied back)
  struct HostPipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t copied[2] = {}, computed[2] = {}, returned[2] = {};
    uint8_t* d_in[2] = {};
    size_t in_bytes = 0;  // capacity of each input slot
    float* d_out[2] = {};
    int slot = 0;
  } pipe;
};

// ---- launchers (each returns cudaGetLastError() of its launch) -------------
cudaError_t launch_plan_terms(Plan& p, cudaStream_t s);
cudaError_t launch_build_csr(Plan& p, cudaStream_t s);
cudaError_t launch_twiddles(Plan& p, cudaStream_t s);
cudaError_t launch_beam(Plan& p, cudaStream_t s);
cudaError_t launch_postprocess(const Plan& p, const float* d_in, float* d_out, int flags, float floor,
                               cudaStream_t s);
// Builds p.gt from the per-cell table (two launches, synchronous).
cudaError_t build_gather_tables(Plan& p, int layout, int threads, size_t* bytes);
void free_gather_tables(GatherTables& g);
// Waits for and releases the streams, events and buffers of epic_image_host_async.
void free_host_pipe(Plan& p);

// FP32 FFT path: the fused unpack + calibrate + grid + FFT + products kernel.
// Sets p.threads, p.smem, p.ent_in_smem and returns the resident CTAs per SM.
cudaError_t fft_image_config(Plan& p, int* ctas_per_sm);
cudaError_t launch_fft_image(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws,
                             cudaStream_t s);

// The same path on 128 x 128 grids, run by clusters of two CTAs (epic_fft128.cu).
// Sets p.threads, p.smem, p.ent_in_smem and returns the co-resident clusters;
// an imaging launch's WorkSplit then counts clusters.
size_t fft128_smem_need(int A, int P);
size_t fft128_xbuf_elems(int clusters, int P);  // float2 of the clusters' exchange buffers
int fft128_max_ant();
cudaError_t fft128_config(Plan& p, int* clusters);
cudaError_t launch_fft128_image_ws(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                                   int* part_auto, cudaStream_t s);

// What one block-end reduction needs of a plan and of its call's split.
struct ReduceArgs {
  int T, C, A, N, vq, dec, ctas, spans, subtract, accumulate;
  long long W;
  const float* part;
  const int* part_auto;
  const double2* coef64;
  const float* kx2;
  const float* ky2;
  float* out;
};

// One imaging problem of the tensor-core kernel: a plan's tables and the split
// of one call over its units (CTA-sized spans of W units, each span an "item").
struct DftJob {
  const uint8_t* volts;
  const float2* coef;
  const int* cnt;
  const int* base;
  const int* off;
  const uint16_t* task;
  const uint16_t* ent_a;
  const float* ent_w;
  const float4* dscale;
  float* part;
  int* part_auto;
  int* status;
  long long W, units;
  int T, C, A, spans, q128, ent_in_smem;
  int first_item, n_items;  // a batch's items [first_item, first_item + n_items) are this job's spans
  // batch only: the job's block-end reduction, run in the same launch as items
  // [red_first, red_first + n_red) of the queue (numbered after every imaging
  // item), each `red_rows` rows of one virtual channel; done[cv] counts
  // the imaging items that have written their partial image of virtual channel cv
  ReduceArgs red;
  int* done;
  int red_first, n_red, red_rows;
};
// A batch's work list: the items of several jobs (jobs ordered by first_item),
// claimed one at a time by the CTAs of one persistent launch.
struct DftQueue {
  const DftJob* jobs;
  int n_jobs, n_items;  // all items: imaging items first, then reduction items
  int n_image_items;
  int* head;  // the next unclaimed item; zero when the launch starts
  // failure test only: reduction items wait for this many signals more than can
  // come, for at most wait_ns (0: the normal one-second limit, no extra)
  int test_extra = 0;
  unsigned long long wait_ns = 0;
};

// Pixels of one row per thread in the reduction items of a batch launch.
constexpr int kBatchReducePix = 2;
// The job of one call of a tensor-core plan (its first_item is 0).
DftJob dft_job(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part, int* part_auto);
// Shared memory of a persistent batch launch whose jobs have at most A_lay
// antennas and max_entries gather entries held in shared memory.
size_t dft_batch_smem(int A_lay, int max_entries);
// One persistent launch of `ctas` CTAs that image every item of q (device
// memory: q.jobs, q.head, which must be 0); all jobs share the transform xform.
cudaError_t launch_dft_batch(int xform, const DftQueue& q, int A_lay, int max_entries, const uint16_t* fmat,
                             const float2* twiddle, int ctas, cudaStream_t s);

// Tensor-core path (DFT-by-GEMM on tcgen05; N = 64, two polarisations).
size_t dft_smem_need(int A, int max_entries);
cudaError_t launch_dft_tables(Plan& p, cudaStream_t s);
cudaError_t dft_image_config(Plan& p, int* ctas_per_sm);
// test_wait_ns > 0: the first mbarrier wait of every CTA waits on a barrier
// that nothing arrives at, for that long, and takes the time-out path (tests).
cudaError_t launch_dft_image(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                             int* part_auto, cudaStream_t s, unsigned long long test_wait_ns = 0);

// Gradient of the image-plane loss (epic_grad), FP32 FFT path at N = 64.
cudaError_t launch_grad_coef(Plan& p, const float* d_gains, cudaStream_t s);
cudaError_t launch_fft_image_coef(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, const float2* coef,
                                  cudaStream_t s);
cudaError_t launch_reduce_coef(Plan& p, int T, const WorkSplit& ws, const double2* coef64, float* d_out,
                               cudaStream_t s);
cudaError_t launch_residual(Plan& p, const float* d_model, float* d_loss, cudaStream_t s);
cudaError_t launch_adjoint(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, cudaStream_t s);
cudaError_t launch_grad_reduce(Plan& p, int T, const WorkSplit& ws, const float* d_gains, float* d_grad,
                               cudaStream_t s);
size_t adjoint_smem_need(const Plan& p);
int adjoint_max_ant(int N);

// Block end: sum the CTA partials of every channel in a fixed order, remove the
// autocorrelation term, write or accumulate the output.
cudaError_t launch_reduce(Plan& p, int T, const WorkSplit& ws, float* d_out, int accumulate,
                          cudaStream_t s);
cudaError_t launch_zero(float* d_out, size_t n, cudaStream_t s);
cudaError_t image_launches(Plan& p, const uint8_t* d_volts, int n_time, float* d_out, int accumulate,
                           cudaStream_t s);

// The same two launches with the partial-image workspace passed explicitly
// (used by the entry point that allocates nothing and takes its workspace from
// a static device array).
cudaError_t launch_fft_image_ws(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                                int* part_auto, cudaStream_t s);
cudaError_t launch_reduce_ws(const Plan& p, int T, const WorkSplit& ws, const float* part, const int* part_auto,
                             float* d_out, int accumulate, cudaStream_t s);

cudaError_t launch_debug_unpack(const uint8_t* d_in, size_t n, int8_t* d_out, cudaStream_t s);
cudaError_t launch_debug_grid(Plan& p, const uint8_t* d_volts, int T, int t, int c, int pol,
                              float* d_grid, cudaStream_t s);
// The pre-square image Y of one (t, c, pol) through the imaging kernel's line
// transforms (FP32 plans, N = 32 or 64); d_y [N][N][2].
cudaError_t launch_debug_transform(Plan& p, const uint8_t* d_volts, int T, int t, int c, int pol, float* d_y,
                                   cudaStream_t s);

// ---- small device helpers shared by the kernels ----------------------------
// Sec. 3.2: one byte = 4-bit real (high nibble) + 4-bit imaginary (low nibble),
// both two's complement.
__device__ __forceinline__ int nib_hi(unsigned b) { return (int)((b >> 4) & 15u) - (int)((b >> 3) & 16u); }
__device__ __forceinline__ int nib_lo(unsigned b) { return (int)(b & 15u) - (int)((b << 1) & 16u); }

__host__ __device__ __forceinline__ long long span_first_unit(const WorkSplit& ws, int b) {
  return (long long)b * ws.W;
}

}  // namespace epic

// The opaque handle of include/epic.h.
struct epic_plan {
  epic::Plan p;
};
