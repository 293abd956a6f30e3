// epic_api.cu -- the C ABI declared in include/epic.h: validation, plan
// lifetime, and the launch sequence of one imaging call.
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "epic_internal.cuh"

using epic::Plan;

namespace {

constexpr double kC0 = 299792458.0;
constexpr int kMaxAntFft = 2048;

bool is_finite(double x) { return std::isfinite(x); }

// The same FP64 operations, in the same order and each rounded on its own, as
// the device-side plan kernel (this file is compiled with -ffp-contract=off).
double cell_coord(double pos_m, double freq_hz, double cell_lambda, int N) {
  const double lambda = kC0 / freq_hz;
  return pos_m / (lambda * cell_lambda) + 0.5 * (double)N;
}

constexpr size_t kSmemOptin = 232448;  // opt-in shared memory per CTA on sm_100/sm_103 (227 KB)

// FP32 path on 128 x 128 grids: four folded 64 x 64 problems per channel run by
// the 64 x 64 kernel, or clusters of two CTAs that split one 128 x 128 problem.
// Folding repeats the gather four times but runs the cheaper 64 x 64 transforms;
// measured on the station array (A S^2 = 6 400 entries per channel) folding took
// 10.3 ms against 11.5 ms, on 1 024 antennas (25 600 entries) 10.4 ms against
// 8.2 ms, which puts the crossover near 10 000 entries per channel.  Arrays too
// large for the clusters are always folded.
bool fft128_fold(int A, int S) {
  return (long long)A * S * S <= 10000 || A > epic::fft128_max_ant() ||
         epic::fft128_smem_need(A, 2) > kSmemOptin;
}

bool grid_supported(int xform, int N, int P, int A, int S) {
  if (xform == EPIC_XFORM_FFT_FP32) {
    if (N == 128 && !fft128_fold(A, S)) return A <= epic::fft128_max_ant() && epic::fft128_smem_need(A, P) <= kSmemOptin;
    return (N == 32 || N == 64 || N == 128) && A <= kMaxAntFft;
  }
  // tensor path: 64 x 64 or 128 x 128 grids of two polarisations, up to 1024
  // antennas (gather entries in shared memory when they fit, else read from L2)
  (void)S;
  return (N == 32 || N == 64 || N == 128) && P == 2 && A <= 1024 && epic::dft_smem_need(A, 0) <= kSmemOptin;
}

// A named range on the profiler's timeline for the life of an entry-point call
// (NVTX: a no-op unless a profiling tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

epic_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return EPIC_OK;
  if (e == cudaErrorMemoryAllocation) return EPIC_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return EPIC_ERR_NO_DEVICE;
  return EPIC_ERR_CUDA;
}

template <class T>
cudaError_t alloc(T** ptr, size_t count, size_t* total) {
  *ptr = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * count);
  if (e == cudaSuccess) *total += sizeof(T) * count;
  else (void)cudaGetLastError();  // a failed allocation must not be reported again by a later launch
  return e;
}

void free_plan(Plan& p) {
  for (const Plan::Timed& t : p.pending) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (cudaEvent_t e : p.event_pool) cudaEventDestroy(e);
  p.pending.clear();
  p.event_pool.clear();
  void* ptrs[] = {p.d_ant_xy, p.d_freq, p.d_gains, p.d_delays, p.d_box, p.d_wx, p.d_wy, p.d_coef, p.d_coef64,
                  p.d_kx2, p.d_ky2, p.d_csr_ptr, p.d_csr_ent, p.d_twiddle, p.d_status, p.d_part, p.d_part_auto,
                  p.d_stage_in, p.d_stage_out, p.d_fmat, p.d_dphase, p.d_gcoef, p.d_gcoef64, p.d_gimage,
                  p.d_resid, p.d_loss_part, p.d_gpart, p.d_beam, p.d_xbuf, p.d_dscale};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  epic::free_gather_tables(p.gt);
  epic::free_host_pipe(p);
}


cudaEvent_t take_event(Plan& p) {
  if (!p.event_pool.empty()) {
    cudaEvent_t e = p.event_pool.back();
    p.event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int kind_index(Plan& p, const char* name) {
  for (size_t k = 0; k < p.kinds.size(); ++k)
    if (p.kinds[k] == name) return (int)k;
  p.kinds.emplace_back(name);
  p.kind_launches.push_back(0);
  p.kind_ms.push_back(0.0);
  return (int)p.kinds.size() - 1;
}

// Runs launch(), bracketed by events on s when the plan records timing.
template <class F>
cudaError_t timed(Plan& p, const char* name, cudaStream_t s, F&& launch) {
  if (!p.timing) return launch();
  Plan::Timed t{kind_index(p, name), take_event(p), take_event(p)};
  cudaEventRecord(t.start, s);
  cudaError_t e = launch();
  cudaEventRecord(t.stop, s);
  p.pending.push_back(t);
  return e;
}

cudaError_t drain_timing(Plan& p) {
  for (const Plan::Timed& t : p.pending) {
    cudaError_t e = cudaEventSynchronize(t.stop);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.start, t.stop);
    p.kind_launches[t.kind] += 1;
    p.kind_ms[t.kind] += ms;
    p.event_pool.push_back(t.start);
    p.event_pool.push_back(t.stop);
  }
  p.pending.clear();
  return cudaSuccess;
}

}  // namespace

namespace epic {
// Largest number of channels any CTA of a split touches.
int spans_needed(const epic::WorkSplit& ws) {
  int worst = 1;
  for (int b = 0; b < ws.ctas; ++b) {
    const long long u0 = (long long)b * ws.W;
    const long long u1 = (u0 + ws.W < ws.units ? u0 + ws.W : ws.units) - 1;
    const int n = (int)(u1 / ws.T - u0 / ws.T) + 1;
    if (n > worst) worst = n;
  }
  return worst;
}

// Work units u = c*T + t (channel-major) split into equal contiguous ranges,
// one per CTA (at most `cap` CTAs), with no CTA left empty.
epic::WorkSplit split_work_cap(const Plan& p, int T, int cap) {
  epic::WorkSplit ws;
  ws.T = T;
  ws.units = (long long)p.C * p.vq * T;
  long long ctas = cap < ws.units ? cap : ws.units;
  ws.W = (ws.units + ctas - 1) / ctas;
  ws.ctas = (int)((ws.units + ws.W - 1) / ws.W);
  ws.spans = spans_needed(ws);
  return ws;
}

epic::WorkSplit split_work(const Plan& p, int T) { return split_work_cap(p, T, p.ctas_use > 0 ? p.ctas_use : p.ctas); }

bool split_fits(const Plan& p, const epic::WorkSplit& ws) {
  return (long long)ws.ctas * ws.spans <= (long long)p.ctas * p.spans;
}

// The launches of one imaging call (image kernel, then the block-end reduction),
// shared by epic_image and the batch graphs.  No timing, no allocation.
cudaError_t image_launches(Plan& p, const uint8_t* d_volts, int n_time, float* d_out, int accumulate, cudaStream_t s) {
  const size_t out_n = (size_t)p.C * 4 * p.N * p.N;
  if (n_time == 0) return accumulate ? cudaSuccess : launch_zero(d_out, out_n, s);
  const WorkSplit ws = split_work(p, n_time);
  if (!split_fits(p, ws)) return cudaErrorInvalidConfiguration;
  cudaError_t e = (p.xform == EPIC_XFORM_FFT_FP32) ? launch_fft_image(p, d_volts, n_time, ws, s)
                                                   : launch_dft_image(p, d_volts, n_time, ws, p.d_part, p.d_part_auto, s);
  if (e != cudaSuccess) return e;
  return launch_reduce(p, n_time, ws, d_out, accumulate, s);
}
}  // namespace epic

using epic::split_fits;
using epic::split_work;

extern "C" {

const char* epic_status_string(int s) {
  switch (s) {
    case EPIC_OK: return "EPIC_OK";
    case EPIC_ERR_INVALID_ARG: return "EPIC_ERR_INVALID_ARG";
    case EPIC_ERR_OFFGRID: return "EPIC_ERR_OFFGRID";
    case EPIC_ERR_UNSUPPORTED: return "EPIC_ERR_UNSUPPORTED";
    case EPIC_ERR_OOM: return "EPIC_ERR_OOM";
    case EPIC_ERR_CUDA: return "EPIC_ERR_CUDA";
    case EPIC_ERR_TIMEOUT: return "EPIC_ERR_TIMEOUT";
    case EPIC_ERR_NO_DEVICE: return "EPIC_ERR_NO_DEVICE";
    case EPIC_ERR_INTERNAL: return "EPIC_ERR_INTERNAL";
    default: return "EPIC_ERR_UNKNOWN";
  }
}

epic_status epic_plan_validate(const epic_plan_desc* d) {
  if (!d || !d->ant_xy_m || !d->chan_freq_hz) return EPIC_ERR_INVALID_ARG;
  if (d->n_ant < 1 || d->n_chan < 1 || (d->n_pol != 1 && d->n_pol != 2)) return EPIC_ERR_INVALID_ARG;
  if (d->n_chan > (1 << 20)) return EPIC_ERR_INVALID_ARG;
  const int N = d->grid_n, S = d->kernel_support;
  if (N < 8 || N > 4096 || (N & (N - 1)) != 0) return EPIC_ERR_INVALID_ARG;
  if (S < 1 || S > 15 || (S % 2) == 0 || S >= N) return EPIC_ERR_INVALID_ARG;
  if (!is_finite(d->cell_lambda) || d->cell_lambda <= 0.0) return EPIC_ERR_INVALID_ARG;
  if (S > 1 && (!is_finite(d->kernel_sigma_cells) || d->kernel_sigma_cells <= 0.0)) return EPIC_ERR_INVALID_ARG;
  if (d->xform < EPIC_XFORM_FFT_FP32 || d->xform > EPIC_XFORM_DFT_FP16) return EPIC_ERR_INVALID_ARG;
  if (d->subtract_autos != 0 && d->subtract_autos != 1) return EPIC_ERR_INVALID_ARG;
  const int A = d->n_ant, P = d->n_pol, C = d->n_chan;
  for (int k = 0; k < 2 * A; ++k)
    if (!is_finite(d->ant_xy_m[k])) return EPIC_ERR_INVALID_ARG;
  for (int c = 0; c < C; ++c)
    if (!is_finite(d->chan_freq_hz[c]) || d->chan_freq_hz[c] <= 0.0) return EPIC_ERR_INVALID_ARG;
  if (d->gains)
    for (long long k = 0; k < 2LL * C * A * P; ++k)
      if (!is_finite(d->gains[k])) return EPIC_ERR_INVALID_ARG;
  if (d->delays_s)
    for (int k = 0; k < A * P; ++k)
      if (!is_finite(d->delays_s[k])) return EPIC_ERR_INVALID_ARG;
  // every kernel box inside the grid, in every channel (reading R7: no wrap)
  for (int c = 0; c < C; ++c)
    for (int a = 0; a < A; ++a) {
      const double u = cell_coord(d->ant_xy_m[2 * a], d->chan_freq_hz[c], d->cell_lambda, N);
      const double v = cell_coord(d->ant_xy_m[2 * a + 1], d->chan_freq_hz[c], d->cell_lambda, N);
      if (!is_finite(u) || !is_finite(v) || std::fabs(u) > 1e9 || std::fabs(v) > 1e9) return EPIC_ERR_OFFGRID;
      const long long i0 = (long long)std::floor(u + 0.5) - (S - 1) / 2;
      const long long j0 = (long long)std::floor(v + 0.5) - (S - 1) / 2;
      if (i0 < 0 || j0 < 0 || i0 + S > N || j0 + S > N) return EPIC_ERR_OFFGRID;
    }
  if (!grid_supported(d->xform, N, P, A, S)) return EPIC_ERR_UNSUPPORTED;
  return EPIC_OK;
}

epic_status epic_plan_create(const epic_plan_desc* d, epic_plan** out) {
  Range range("epic_plan_create");
  if (!out) return EPIC_ERR_INVALID_ARG;
  *out = nullptr;
  epic_status st = epic_plan_validate(d);
  if (st != EPIC_OK) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return from_cuda(e);
  epic_plan* h = new (std::nothrow) epic_plan();
  if (!h) return EPIC_ERR_OOM;
  Plan& p = h->p;
  p.A = d->n_ant; p.P = d->n_pol; p.C = d->n_chan; p.N = d->grid_n; p.S = d->kernel_support;
  p.xform = d->xform; p.subtract = d->subtract_autos;
  p.cell_lambda = d->cell_lambda;
  p.sigma = p.S > 1 ? d->kernel_sigma_cells : 1.0;
  p.device = dev;
  cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev);

  const size_t A = p.A, P = p.P, C = p.C, N = p.N, S = p.S;
  size_t total = 0;
  auto fail = [&](cudaError_t err) {
    free_plan(p);
    delete h;
    return from_cuda(err);
  };
#define EPIC_TRY(x)                   \
  do {                                \
    cudaError_t err_ = (x);           \
    if (err_ != cudaSuccess) return fail(err_); \
  } while (0)
  EPIC_TRY(alloc(&p.d_ant_xy, 2 * A, &total));
  EPIC_TRY(alloc(&p.d_freq, C, &total));
  if (d->gains) EPIC_TRY(alloc(&p.d_gains, 2 * C * A * P, &total));
  if (d->delays_s) EPIC_TRY(alloc(&p.d_delays, A * P, &total));
  EPIC_TRY(alloc(&p.d_box, 2 * C * A, &total));
  EPIC_TRY(alloc(&p.d_wx, C * A * S, &total));
  EPIC_TRY(alloc(&p.d_wy, C * A * S, &total));
  EPIC_TRY(alloc(&p.d_coef, C * A * P, &total));
  EPIC_TRY(alloc(&p.d_coef64, C * A * P, &total));
  EPIC_TRY(alloc(&p.d_dphase, C * A * P, &total));
  EPIC_TRY(alloc(&p.d_kx2, C * A * N, &total));
  EPIC_TRY(alloc(&p.d_ky2, C * A * N, &total));
  EPIC_TRY(alloc(&p.d_beam, C * N * N, &total));
  EPIC_TRY(alloc(&p.d_csr_ptr, C * (N * N + 1), &total));
  EPIC_TRY(alloc(&p.d_csr_ent, C * A * S * S, &total));
  EPIC_TRY(alloc(&p.d_twiddle, N, &total));
  EPIC_TRY(alloc(&p.d_status, 1, &total));

  EPIC_TRY(cudaMemcpy(p.d_ant_xy, d->ant_xy_m, sizeof(double) * 2 * A, cudaMemcpyHostToDevice));
  EPIC_TRY(cudaMemcpy(p.d_freq, d->chan_freq_hz, sizeof(double) * C, cudaMemcpyHostToDevice));
  if (d->gains) EPIC_TRY(cudaMemcpy(p.d_gains, d->gains, sizeof(double) * 2 * C * A * P, cudaMemcpyHostToDevice));
  if (d->delays_s) EPIC_TRY(cudaMemcpy(p.d_delays, d->delays_s, sizeof(double) * A * P, cudaMemcpyHostToDevice));
  EPIC_TRY(cudaMemset(p.d_status, 0, sizeof(int)));

  EPIC_TRY(epic::launch_plan_terms(p, 0));
  EPIC_TRY(epic::launch_twiddles(p, 0));
  EPIC_TRY(epic::launch_build_csr(p, 0));
  EPIC_TRY(epic::launch_beam(p, 0));
  EPIC_TRY(cudaDeviceSynchronize());
  int status = 0, nnz_last = 0;
  EPIC_TRY(cudaMemcpy(&status, p.d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status == epic::kDevOffGrid) {
    free_plan(p);
    delete h;
    return EPIC_ERR_OFFGRID;
  }
  // every antenna contributes S*S entries to every channel's gather table
  for (size_t c = 0; c < C; ++c) {
    EPIC_TRY(cudaMemcpy(&nnz_last, p.d_csr_ptr + c * (N * N + 1) + N * N, sizeof(int), cudaMemcpyDeviceToHost));
    if ((size_t)nnz_last != A * S * S) return fail(cudaErrorUnknown);
  }

  int per_sm = 0;
  size_t gt_bytes = 0;
  int clusters = 0;  // N = 128: the imaging launch counts clusters of two CTAs
  if (p.xform == EPIC_XFORM_FFT_FP32 && p.N == 128 && fft128_fold(p.A, p.S)) {
    p.vq = 4;
    EPIC_TRY(epic::build_gather_tables(p, epic::kLayoutFft64Q, 512, &gt_bytes));
    total += gt_bytes;
    EPIC_TRY(epic::fft_image_config(p, &per_sm));
  } else if (p.xform == EPIC_XFORM_FFT_FP32 && p.N == 128) {
    EPIC_TRY(epic::build_gather_tables(p, epic::kLayoutFft128, 1024, &gt_bytes));
    total += gt_bytes;
    EPIC_TRY(epic::fft128_config(p, &clusters));
    if (clusters < 1) return fail(cudaErrorInvalidConfiguration);
  } else if (p.xform == EPIC_XFORM_FFT_FP32) {
    EPIC_TRY(epic::build_gather_tables(p, p.N == 64 ? epic::kLayoutFft64 : epic::kLayoutFft32,
                                       p.N == 64 ? 512 : 128, &gt_bytes));
    total += gt_bytes;
    EPIC_TRY(epic::fft_image_config(p, &per_sm));
  } else {
    // N = 128: four virtual channels per channel, one per output-parity subset;
    // N = 32: the 64 x 64 transform of the zero-padded grid, even pixels kept
    p.vq = p.N == 128 ? 4 : 1;
    p.dec = p.N == 32 ? 2 : 1;
    const int layout = p.N == 128 ? epic::kLayoutPairQ : p.N == 32 ? epic::kLayoutPairD : epic::kLayoutPair64;
    EPIC_TRY(epic::build_gather_tables(p, layout, 512, &gt_bytes));
    total += gt_bytes;
    EPIC_TRY(alloc(&p.d_fmat, (size_t)4 * 128 * 128 / 2, &total));
    if (p.xform == EPIC_XFORM_DFT_FP16X3 || p.xform == EPIC_XFORM_DFT_FP16)
      EPIC_TRY(alloc(&p.d_dscale, (size_t)4 * p.C * p.vq, &total));
    EPIC_TRY(epic::launch_dft_tables(p, 0));
    EPIC_TRY(cudaDeviceSynchronize());
    EPIC_TRY(epic::dft_image_config(p, &per_sm));
  }
  if (clusters == 0 && per_sm < 1) return fail(cudaErrorInvalidConfiguration);
  p.ctas = clusters > 0 ? clusters : p.sm_count * per_sm;
  p.spans = (p.C * p.vq + p.ctas - 1) / p.ctas + 2;
  size_t before = total;
  const size_t Ns = p.vq == 4 ? N / 2 : N * p.dec;  // side of a partial image
  EPIC_TRY(alloc(&p.d_part, (size_t)p.ctas * p.spans * 4 * Ns * Ns, &total));
  EPIC_TRY(alloc(&p.d_part_auto, (size_t)p.ctas * p.spans * A * 4, &total));
  if (p.xform == EPIC_XFORM_FFT_FP32 && p.N == 128 && p.vq == 1)
    EPIC_TRY(alloc(&p.d_xbuf, epic::fft128_xbuf_elems(p.ctas, p.P), &total));
  p.workspace_bytes = total - before;
  // epic_grad: FP32 FFT plans imaged by the fft_image kernel (32 x 32, 64 x 64,
  // and 128 x 128 folded into four 64 x 64 problems), one antenna per thread of
  // the adjoint (at most 128 antennas at 32 x 32, 512 otherwise)
  if (p.xform == EPIC_XFORM_FFT_FP32 && (p.N != 128 || p.vq == 4) && p.A <= epic::adjoint_max_ant(p.N) &&
      epic::adjoint_smem_need(p) <= kSmemOptin) {
    EPIC_TRY(alloc(&p.d_gcoef, C * A * P, &total));
    EPIC_TRY(alloc(&p.d_gcoef64, C * A * P, &total));
    EPIC_TRY(alloc(&p.d_gimage, C * 4 * N * N, &total));
    EPIC_TRY(alloc(&p.d_resid, C * 2 * N * N, &total));
    EPIC_TRY(alloc(&p.d_loss_part, C, &total));
    EPIC_TRY(alloc(&p.d_gpart, (size_t)p.ctas * p.spans * A * P, &total));
    EPIC_TRY(cudaMemset(p.d_resid, 0, sizeof(float) * C * 2 * N * N));
    p.grad_ok = true;
  }
  p.device_bytes = total;
#undef EPIC_TRY
  *out = h;
  return EPIC_OK;
}

epic_status epic_plan_destroy(epic_plan* h) {
  if (!h) return EPIC_OK;
  cudaDeviceSynchronize();
  free_plan(h->p);
  delete h;
  return EPIC_OK;
}

epic_status epic_plan_query(const epic_plan* h, epic_plan_info* info) {
  if (!h || !info) return EPIC_ERR_INVALID_ARG;
  const Plan& p = h->p;
  info->n_ant = p.A; info->n_pol = p.P; info->n_chan = p.C; info->grid_n = p.N;
  info->kernel_support = p.S; info->xform = p.xform; info->subtract_autos = p.subtract;
  info->device = p.device; info->ctas = p.ctas; info->threads_per_cta = p.threads;
  const size_t out_bytes = sizeof(float) * 4 * p.C * p.N * p.N;
  info->device_bytes = p.device_bytes + p.stage_in_bytes + (p.d_stage_out ? out_bytes : 0) + 2 * p.pipe.in_bytes +
                       (p.pipe.d_out[0] ? 2 * out_bytes : 0);
  info->workspace_bytes = p.workspace_bytes;
  // integer self powers stay exact in int32 per CTA and the unit index in int64
  info->max_time = (1LL << 24);
  info->cluster_dim = (p.xform == EPIC_XFORM_FFT_FP32 && p.N == 128 && p.vq == 1) ? 2 : 1;
  info->transform_n = p.vq == 4 ? p.N / 2 : (p.xform != EPIC_XFORM_FFT_FP32 ? 64 : p.N);
  info->transforms_per_image = p.vq;
  info->unpack_warps = p.unpack_warps;
  return EPIC_OK;
}

epic_status epic_image(epic_plan* h, const uint8_t* d_volts, int n_time, float* d_out, int accumulate,
                       void* stream) {
  Range range("epic_image");
  if (!h || !d_out || n_time < 0 || n_time > (1 << 24) || (accumulate != 0 && accumulate != 1))
    return EPIC_ERR_INVALID_ARG;
  if (n_time > 0 && !d_volts) return EPIC_ERR_INVALID_ARG;
  Plan& p = h->p;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t out_n = (size_t)p.C * 4 * p.N * p.N;
  if (n_time == 0) return accumulate ? EPIC_OK : from_cuda(epic::launch_zero(d_out, out_n, s));
  const epic::WorkSplit ws = split_work(p, n_time);
  if (!split_fits(p, ws)) return EPIC_ERR_UNSUPPORTED;  // a CTA cap below the plan's needs more slots
  cudaError_t e = (p.xform == EPIC_XFORM_FFT_FP32)
                      ? timed(p, "fft_image", s, [&] { return epic::launch_fft_image(p, d_volts, n_time, ws, s); })
                      : timed(p, "dft_image", s, [&] {
                          return epic::launch_dft_image(p, d_volts, n_time, ws, p.d_part, p.d_part_auto, s);
                        });
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(timed(p, "reduce", s, [&] { return epic::launch_reduce(p, n_time, ws, d_out, accumulate, s); }));
}

epic_status epic_image_host(epic_plan* h, const uint8_t* h_volts, int n_time, float* h_out, int accumulate,
                            void* stream) {
  Range range("epic_image_host");
  if (!h || !h_out || n_time < 0 || n_time > (1 << 24) || (accumulate != 0 && accumulate != 1))
    return EPIC_ERR_INVALID_ARG;
  if (n_time > 0 && !h_volts) return EPIC_ERR_INVALID_ARG;
  Plan& p = h->p;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t in_bytes = (size_t)n_time * p.C * p.A * p.P;
  const size_t out_bytes = sizeof(float) * (size_t)p.C * 4 * p.N * p.N;
  if (in_bytes > p.stage_in_bytes) {
    if (p.d_stage_in) cudaFree(p.d_stage_in);
    p.d_stage_in = nullptr;
    p.stage_in_bytes = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p.d_stage_in), in_bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return from_cuda(e);
    }
    p.stage_in_bytes = in_bytes;
  }
  if (!p.d_stage_out) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p.d_stage_out), out_bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return from_cuda(e);
    }
  }
  cudaError_t e = cudaSuccess;
  if (in_bytes) e = cudaMemcpyAsync(p.d_stage_in, h_volts, in_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && accumulate) e = cudaMemcpyAsync(p.d_stage_out, h_out, out_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return from_cuda(e);
  epic_status st = epic_image(h, p.d_stage_in, n_time, p.d_stage_out, accumulate, stream);
  if (st != EPIC_OK) return st;
  e = cudaMemcpyAsync(h_out, p.d_stage_out, out_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

epic_status epic_sync(epic_plan* h, void* stream) {
  if (!h) return EPIC_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaSuccess && h->p.pipe.d2h) e = cudaStreamSynchronize(h->p.pipe.d2h);  // epic_image_host_async results
  if (e != cudaSuccess) return from_cuda(e);
  int status = 0;
  e = cudaMemcpy(&status, h->p.d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  if (status == epic::kDevOk) return EPIC_OK;
  cudaMemset(h->p.d_status, 0, sizeof(int));
  return status == epic::kDevTimeout ? EPIC_ERR_TIMEOUT : EPIC_ERR_CUDA;
}

epic_status epic_grad(epic_plan* h, const uint8_t* d_volts, int n_time, const float* d_gains,
                      const float* d_model, float* d_grad, float* d_loss, void* stream) {
  Range range("epic_grad");
  if (!h || !d_volts || !d_gains || !d_model || !d_grad || !d_loss || n_time < 1 || n_time > (1 << 24))
    return EPIC_ERR_INVALID_ARG;
  Plan& p = h->p;
  if (!p.grad_ok) return EPIC_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const epic::WorkSplit ws = split_work(p, n_time);
  if (!split_fits(p, ws)) return EPIC_ERR_UNSUPPORTED;
  cudaError_t e = epic::launch_grad_coef(p, d_gains, s);
  if (e == cudaSuccess)
    e = timed(p, "fft_image", s, [&] { return epic::launch_fft_image_coef(p, d_volts, n_time, ws, p.d_gcoef, s); });
  if (e == cudaSuccess)
    e = timed(p, "reduce", s, [&] { return epic::launch_reduce_coef(p, n_time, ws, p.d_gcoef64, p.d_gimage, s); });
  if (e == cudaSuccess) e = epic::launch_residual(p, d_model, d_loss, s);
  if (e == cudaSuccess) e = timed(p, "adjoint", s, [&] { return epic::launch_adjoint(p, d_volts, n_time, ws, s); });
  if (e == cudaSuccess) e = epic::launch_grad_reduce(p, n_time, ws, d_gains, d_grad, s);
  return from_cuda(e);
}

epic_status epic_postprocess(const epic_plan* h, const float* d_in, float* d_out, int flags, float beam_floor,
                             void* stream) {
  if (!h || !d_in || !d_out || (flags & ~(EPIC_POST_STOKES | EPIC_POST_BEAM)) != 0 || !(beam_floor > 0.f))
    return EPIC_ERR_INVALID_ARG;
  if ((flags & EPIC_POST_STOKES) && h->p.P != 2) return EPIC_ERR_INVALID_ARG;
  return from_cuda(epic::launch_postprocess(h->p, d_in, d_out, flags, beam_floor,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

epic_status epic_debug_unpack(const uint8_t* d_in, size_t n, int8_t* d_out, void* stream) {
  if (n > 0 && (!d_in || !d_out)) return EPIC_ERR_INVALID_ARG;
  return from_cuda(epic::launch_debug_unpack(d_in, n, d_out, reinterpret_cast<cudaStream_t>(stream)));
}

epic_status epic_debug_grid(epic_plan* h, const uint8_t* d_volts, int n_time, int t, int c, int p, float* d_grid,
                            void* stream) {
  if (!h || !d_volts || !d_grid || n_time < 1 || t < 0 || t >= n_time || c < 0 || c >= h->p.C || p < 0 ||
      p >= h->p.P)
    return EPIC_ERR_INVALID_ARG;
  return from_cuda(epic::launch_debug_grid(h->p, d_volts, n_time, t, c, p, d_grid,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

epic_status epic_debug_transform(epic_plan* h, const uint8_t* d_volts, int n_time, int t, int c, int p, float* d_y,
                                 void* stream) {
  if (!h || !d_volts || !d_y || n_time < 1 || t < 0 || t >= n_time || c < 0 || c >= h->p.C || p < 0 ||
      p >= h->p.P)
    return EPIC_ERR_INVALID_ARG;
  if (h->p.xform != EPIC_XFORM_FFT_FP32 || (h->p.N != 32 && h->p.N != 64)) return EPIC_ERR_UNSUPPORTED;
  return from_cuda(epic::launch_debug_transform(h->p, d_volts, n_time, t, c, p, d_y,
                                                reinterpret_cast<cudaStream_t>(stream)));
}

epic_status epic_debug_image_timeout(epic_plan* h, const uint8_t* d_volts, int n_time, long long wait_ns,
                                     void* stream) {
  if (!h || !d_volts || n_time < 1 || n_time > (1 << 24) || wait_ns < 1000 || wait_ns > 1000000000LL)
    return EPIC_ERR_INVALID_ARG;
  Plan& p = h->p;
  if (p.xform == EPIC_XFORM_FFT_FP32) return EPIC_ERR_UNSUPPORTED;
  const epic::WorkSplit ws = split_work(p, n_time);
  if (!split_fits(p, ws)) return EPIC_ERR_UNSUPPORTED;
  return from_cuda(epic::launch_dft_image(p, d_volts, n_time, ws, p.d_part, p.d_part_auto,
                                          reinterpret_cast<cudaStream_t>(stream), (unsigned long long)wait_ns));
}

epic_status epic_timing_enable(epic_plan* h, int enable) {
  if (!h || (enable != 0 && enable != 1)) return EPIC_ERR_INVALID_ARG;
  Plan& p = h->p;
  cudaError_t e = drain_timing(p);
  for (size_t k = 0; k < p.kinds.size(); ++k) {
    p.kind_launches[k] = 0;
    p.kind_ms[k] = 0.0;
  }
  p.timing = enable != 0;
  return from_cuda(e);
}

epic_status epic_timing_read(epic_plan* h, epic_kernel_time* out, int capacity, int* count) {
  if (!h || !count || capacity < 0 || (capacity > 0 && !out)) return EPIC_ERR_INVALID_ARG;
  Plan& p = h->p;
  cudaError_t e = drain_timing(p);
  if (e != cudaSuccess) return from_cuda(e);
  *count = (int)p.kinds.size();
  for (int k = 0; k < capacity && k < (int)p.kinds.size(); ++k) {
    std::memset(out[k].kernel, 0, sizeof(out[k].kernel));
    std::strncpy(out[k].kernel, p.kinds[k].c_str(), sizeof(out[k].kernel) - 1);
    out[k].launches = p.kind_launches[k];
    out[k].total_ms = p.kind_ms[k];
  }
  return EPIC_OK;
}

}  // extern "C"
