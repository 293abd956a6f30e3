/*
 * epic.h -- C ABI of the GB300 E-field direct imager (MOFF / EPIC).
 *
 * The library images channelised antenna voltages the way Eq. (5) of Kent et
 * al. (arxiv 1904.11422) defines it:
 *
 *     I(l,m) = < | FT{ W * E' }(l,m) |^2 >
 *
 * i.e. unpack 4+4-bit complex samples (Sec. 3.2), apply per-antenna gains and
 * delay compensation (Sec. 3.2, Fig. 2), grid every antenna through its
 * illumination kernel W onto a 0.5-wavelength aperture grid (Sec. 3.2-3.3),
 * spatially Fourier transform each channel and polarisation (Eq. (5), "inverse
 * FT" in Sec. 3.2), form XX, YY, XY (YX = conj XY), accumulate over the block
 * (Sec. 2.1, Sec. 3.2) and optionally remove the autocorrelation term (Sec.
 * 3.2, last paragraph; Fig. 2 "Remove Autocorrelations").
 *
 * Conventions shared by every entry point:
 *   - Plain C types only.  A "stream" argument is a cudaStream_t passed as
 *     void*; NULL means the legacy default stream.
 *   - d_* pointers are device memory owned by the caller; h_* pointers are
 *     host memory owned by the caller.  A plan owns its own device constants
 *     and workspace and frees them in epic_plan_destroy.
 *   - Calls that take a stream are asynchronous and stream-ordered.  Argument
 *     errors are returned synchronously, before anything is launched.
 *     Launch failures return EPIC_ERR_CUDA.
 *   - A plan may be used from one stream at a time (its workspace is shared
 *     by all of its calls).
 *   - No entry point falls back to a CPU implementation: without a usable
 *     CUDA device, calls that need one return EPIC_ERR_NO_DEVICE.
 *
 * Geometry (fixed by the plan; Sec. 3.2 and the readings stated here):
 *   - cell size d = cell_lambda wavelengths of each channel;
 *   - antenna a sits at u = x_a / (lambda_c d) + N/2, v = y_a / (lambda_c d)
 *     + N/2 cells; its S x S kernel box starts at floor(u + 1/2) - (S-1)/2;
 *   - kernel: Gaussian exp(-r^2 / (2 sigma^2)) sampled at cell centres, then
 *     normalised to sum 1 (S = 1: a single unit weight);
 *   - calibration coefficient k = g * exp(-2 pi i nu tau);
 *   - output pixel (column i, row j) is direction l = (i - N/2)/(N d),
 *     m = (j - N/2)/(N d); the transform uses exp(+2 pi i (...)) and no 1/N^2.
 */
#ifndef EPIC_H
#define EPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EPIC_OK = 0,
  EPIC_ERR_INVALID_ARG = 1, /* a pointer, size or flag is out of range        */
  EPIC_ERR_OFFGRID = 2,     /* an antenna's kernel box leaves the N x N grid   */
  EPIC_ERR_UNSUPPORTED = 3, /* valid but not supported (grid size, transform)  */
  EPIC_ERR_OOM = 4,         /* a device allocation failed                       */
  EPIC_ERR_CUDA = 5,        /* a CUDA call or launch failed                     */
  EPIC_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up               */
  EPIC_ERR_NO_DEVICE = 7,   /* no usable CUDA device                            */
  EPIC_ERR_INTERNAL = 8     /* a plan invariant does not hold (debug checks)    */
} epic_status;

/* How the 2-D spatial transform of Eq. (5) is computed. */
typedef enum {
  EPIC_XFORM_FFT_FP32 = 0,   /* shared-memory radix-8 FFT, FP32                 */
  EPIC_XFORM_DFT_BF16X3 = 1, /* DFT-by-GEMM on tcgen05, BF16 hi+lo (3 products) */
  EPIC_XFORM_DFT_FP16X3 = 2, /* DFT-by-GEMM on tcgen05, FP16 hi+lo (3 products) */
  EPIC_XFORM_DFT_BF16 = 3,   /* DFT-by-GEMM on tcgen05, plain BF16              */
  EPIC_XFORM_DFT_FP16 = 4    /* DFT-by-GEMM on tcgen05, plain FP16              */
} epic_xform;

/* Everything a plan needs.  epic_plan_create copies every array; the caller
 * may free them when it returns. */
typedef struct {
  int n_ant;                 /* antennas, >= 1                                   */
  int n_pol;                 /* polarisations: 1 (X) or 2 (X, Y)                 */
  int n_chan;                /* channels, >= 1                                   */
  int grid_n;                /* grid side N (power of two, see epic_plan_validate) */
  int kernel_support;        /* kernel box side S, odd, 1 <= S <= 15, S < N      */
  double cell_lambda;        /* grid cell in wavelengths, > 0 (0.5 = lambda/2)   */
  double kernel_sigma_cells; /* Gaussian sigma in cells, > 0 (used when S > 1)   */
  const double* ant_xy_m;    /* host [n_ant][2]: x (east), y (north) in metres
                                from the array centre                            */
  const double* chan_freq_hz;/* host [n_chan]: channel centre frequencies, > 0   */
  const double* gains;       /* host [n_chan][n_ant][n_pol][2] (re, im) or NULL
                                for unit gains                                   */
  const double* delays_s;    /* host [n_ant][n_pol] seconds, or NULL for zero    */
  int xform;                 /* an epic_xform                                    */
  int subtract_autos;        /* 1: remove sum_a P_a |W_a(l,m)|^2; 0: raw images */
} epic_plan_desc;

typedef struct epic_plan epic_plan;

/* Read-only facts about a plan, for callers that size buffers or report. */
typedef struct {
  int n_ant, n_pol, n_chan, grid_n, kernel_support, xform, subtract_autos;
  int device;                /* CUDA device the plan lives on                    */
  int ctas;                  /* CTAs of one imaging launch                        */
  int threads_per_cta;       /* threads per CTA of the imaging launch            */
  size_t device_bytes;       /* device memory held by the plan                   */
  size_t workspace_bytes;    /* of which per-call scratch (partial images)       */
  long long max_time;        /* largest n_time accepted by one epic_image call   */
  int cluster_dim;           /* CTAs per thread-block cluster of the imaging launch
                                (2: a 128 x 128 grid split over two SMs), else 1  */
  int transform_n;           /* side of the 2-D transforms the imaging kernel runs */
  int transforms_per_image;  /* transforms per (sample, channel, polarisation):
                                4 when a 128 x 128 grid is folded into 64 x 64
                                parity problems, else 1                          */
  unsigned unpack_warps;     /* FP32 path at 64 x 64: bit w set for the four warps
                                that unpack each next sample while the others
                                still grid (chosen from the gather tables), or 0 */
} epic_plan_info;

/* Host-only check of a descriptor, no CUDA call (the same checks that
 * epic_plan_create makes before touching the device).  Returns EPIC_OK,
 * EPIC_ERR_INVALID_ARG (NULL pointer, non-positive or non-finite value, even
 * or too large support), EPIC_ERR_OFFGRID (some antenna's box leaves the grid
 * in some channel) or EPIC_ERR_UNSUPPORTED (a grid size or transform this
 * build does not implement: the FP32 FFT path takes N = 32, 64 or 128 with at
 * most 2048 antennas (a 128 x 128 grid runs on clusters of two CTAs when the
 * array has more than 10 000 gather entries per channel, n_ant x S^2, and at
 * most 1024 antennas, otherwise as four folded 64 x 64 problems); the
 * tensor-core paths take N = 32, 64 or 128 (a 128 x 128 grid is transformed as
 * four 64 x 64 parity sub-problems, a 32 x 32 grid as one zero-padded 64 x 64
 * problem), two polarisations and at most 1024 antennas). */
epic_status epic_plan_validate(const epic_plan_desc* desc);

/* Creates a plan on the current CUDA device: validates desc, copies its
 * arrays, and generates in FP64 on the GPU (Sec. 3.2) each antenna's cell
 * coordinates, kernel weights, calibration coefficient and kernel power
 * spectrum |W_a|^2, plus the per-cell gather table of the gridder.  Blocks
 * until the plan is ready.  *out receives the plan, or NULL on error. */
epic_status epic_plan_create(const epic_plan_desc* desc, epic_plan** out);

/* Frees a plan and all device memory it holds (synchronises the device).
 * NULL is accepted. */
epic_status epic_plan_destroy(epic_plan* plan);

/* Fills *info. */
epic_status epic_plan_query(const epic_plan* plan, epic_plan_info* info);

/* Images one block of n_time samples (Eq. (5), accumulated over the block).
 *   d_volts  device [n_time][n_chan][n_ant][n_pol] bytes, one 4+4-bit complex
 *            sample each (real part in the high nibble, imaginary part in the
 *            low nibble, 4-bit two's complement).
 *   n_time   0 <= n_time <= info.max_time.  n_time = 0 images nothing (the
 *            output is zeroed when accumulate = 0).
 *   d_out    device [n_chan][4][N][N] float: XX, YY, Re XY, Im XY with
 *            XY = sum_t Y_X conj(Y_Y); rows are m, columns l.  With one
 *            polarisation, planes 1-3 are written as zeros.
 *   accumulate 0: d_out = image; 1: d_out += image.
 * With subtract_autos the per-antenna term is removed per call, so images are
 * additive over consecutive blocks.  Deterministic: the same inputs give
 * bit-identical outputs on the same device.  Uses the plan's workspace, so
 * calls on one plan must be ordered (one stream, or synchronised streams);
 * different plans may run concurrently. */
epic_status epic_image(epic_plan* plan, const uint8_t* d_volts, int n_time, float* d_out,
                       int accumulate, void* stream);

/* The same imaging from host buffers: copies h_volts (host [n_time][n_chan]
 * [n_ant][n_pol] bytes, pinned or pageable) to a plan-owned device staging
 * buffer, images it, copies the [n_chan][4][N][N] result to h_out (which is
 * read first when accumulate = 1) and waits for the stream.  Synchronous. */
epic_status epic_image_host(epic_plan* plan, const uint8_t* h_volts, int n_time, float* h_out,
                            int accumulate, void* stream);

/* Streaming form of epic_image_host for page-locked (pinned) host buffers:
 * enqueues the call and returns.  The input is copied to one of two plan-owned
 * device slots on a plan-owned copy stream, imaged on `stream` once it has
 * landed, and the [n_chan][4][N][N] result is copied to h_out on a second
 * plan-owned copy stream; consecutive calls alternate slots, so the input copy
 * of one call overlaps the imaging of the previous one.  h_volts must stay
 * unchanged and h_out untouched until epic_sync(plan, stream) returns, which
 * waits for every enqueued call and reports device errors.  Calls on one plan
 * must use one stream (as for epic_image).  Images equal epic_image's bit for
 * bit.  Returns EPIC_ERR_INVALID_ARG if h_volts (when n_time > 0) or h_out is
 * not page-locked host memory. */
epic_status epic_image_host_async(epic_plan* plan, const uint8_t* h_volts, int n_time, float* h_out,
                                  int accumulate, void* stream);

/* Size of the static device array that epic_image_noalloc takes its scratch
 * space from (32 MiB, held on every GPU that loads the library until exit). */
#define EPIC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* epic_image for callers that must not allocate device memory while they run:
 * for example a real-time streaming loop, where an allocation can stall on
 * device-wide synchronisation and break the block's time budget, or a host
 * application that accounts for all device memory through its own allocator.
 * (The paper has no counterpart; it is an interface addition.)
 * Same arguments, layouts and results as epic_image (FP32 FFT plans only;
 * otherwise EPIC_ERR_UNSUPPORTED), computed by the same kernels with the same
 * work split and summation order, so the images equal epic_image's bit for
 * bit.  The per-call scratch (partial images and self powers) comes from one
 * static device array of EPIC_NOALLOC_SCRATCH_BYTES instead of the plan's
 * workspace, and no call allocates anything.
 *   - Scratch of a call: partial images slots x 4 x Ns^2 floats and self
 *     powers slots x n_ant x 4 ints, each rounded up to a multiple of 256
 *     bytes, where Ns is the side of a partial image (N, or N/2 when
 *     info.transforms_per_image = 4) and slots = (CTAs or clusters of the
 *     call's split) x (channels the busiest of them touches), at most
 *     info.ctas x the plan's span count; the two together must fit in
 *     EPIC_NOALLOC_SCRATCH_BYTES, else the call returns EPIC_ERR_UNSUPPORTED
 *     before anything is launched.  The need never exceeds the partial-image
 *     part of info.workspace_bytes and can be smaller for short blocks.
 *   - Plans imaged by two-CTA clusters (info.cluster_dim = 2) also use the
 *     row-exchange buffer the plan allocated when it was created.
 *   - The plan's device must be the current device (else EPIC_ERR_INVALID_ARG).
 *   - The first call with a device current looks up the array's device address
 *     (cudaGetSymbolAddress, which may load the library's device code), and
 *     looks it up again when the device's context has changed since (after
 *     cudaDeviceReset); make that first call before any stream capture and
 *     before the time-critical loop.
 *   - Every call, from every plan and stream, shares the one array: calls that
 *     overlap on the GPU race and corrupt each other's results.  Order them on
 *     one stream or synchronise between them.  The array keeps the previous
 *     call's contents; each call writes every slot it reads, so nothing needs
 *     clearing. */
epic_status epic_image_noalloc(epic_plan* plan, const uint8_t* d_volts, int n_time, float* d_out,
                               int accumulate, void* stream);

/* Gradient of an image-plane calibration loss with respect to the complex
 * per-antenna gains, for real-time gain calibration (the gain multiplication of
 * Fig. 2, solved for by the EPICal block the paper plans in Sec. 6):
 *     L = sum_c sum_{pp in XX, YY} sum_pix (I_pp(pix) - M_pp(pix))^2
 * where I is the plan's image of the block (autocorrelations removed when the
 * plan removes them) computed with calibration coefficients
 * k = g exp(-2 pi i nu tau): g from d_gains, tau the plan's delays (the plan's
 * own gains are not used).
 *   d_volts  device [n_time][n_chan][n_ant][n_pol] bytes as in epic_image, n_time >= 1
 *   d_gains  device [n_chan][n_ant][n_pol][2] float (re, im)
 *   d_model  device [n_chan][2][N][N] float: M_XX, M_YY (M_YY unused for one pol)
 *   d_grad   device [n_chan][n_ant][n_pol][2] float: dL/dRe g, dL/dIm g
 *            (= 2 dL/d conj(g))
 *   d_loss   device float: L
 * The gridded fields are recomputed in a second pass over the block rather than
 * stored (forward image, residual R = 2 (I - M), then per sample the conjugate
 * transform of R . Y degridded onto each antenna).  FP32 FFT plans with
 * N = 32 and at most 128 antennas, N = 64 and at most 512, or N = 128 folded
 * into four 64 x 64 problems (info.transforms_per_image = 4) and at most 512;
 * others (tensor-core plans, 128 x 128 grids on two-CTA clusters) return
 * EPIC_ERR_UNSUPPORTED.  Uses the plan's workspace; asynchronous. */
epic_status epic_grad(epic_plan* plan, const uint8_t* d_volts, int n_time, const float* d_gains,
                      const float* d_model, float* d_grad, float* d_loss, void* stream);

/* Post-processing flags of epic_postprocess. */
#define EPIC_POST_STOKES 1  /* planes -> pseudo-Stokes I, Q, U, V                     */
#define EPIC_POST_BEAM 2    /* divide by the image of the illumination kernels        */

/* Post-processes accumulated images (layout of epic_image's output):
 *   EPIC_POST_STOKES: pseudo-Stokes planes of linear feeds (Sec. 4.3: straight
 *     linear combinations of the coherency products): I = XX + YY,
 *     Q = XX - YY, U = XY + YX = 2 Re XY, V = -i (XY - YX) = 2 Im XY, with
 *     YX = conj XY.  Needs a two-polarisation plan.
 *   EPIC_POST_BEAM: every plane divided by the channel's kernel imprint
 *     B(l,m) = (1/n_ant) sum_a |W_a(l,m)|^2 (Sec. 3.2, last paragraph: the
 *     image of the pre-generated gridding kernels, removed after the fact);
 *     pixels with B < beam_floor are set to 0.  B = 1 at the zero frequency.
 * Both flags together apply the Stokes step first.  d_in and d_out are device
 * [n_chan][4][N][N] float and may be the same buffer.  beam_floor > 0. */
epic_status epic_postprocess(const epic_plan* plan, const float* d_in, float* d_out, int flags,
                             float beam_floor, void* stream);

/* A batch: several imaging problems (arrays of different antenna counts, grid
 * sizes and channel counts, each with its own plan) run by one graph launch. */
typedef struct epic_batch epic_batch;

/* Captures the imaging of n_plans plans (distinct plans, 1..64) into one CUDA
 * graph, so that one launch images every array (the paper runs one pipeline per
 * array; batching several is this library's addition, for arrays of uneven
 * antenna count, grid size and channel count on one GPU).
 * d_volts[i], n_time[i], d_out[i] are plan i's arguments as in epic_image
 * (accumulate = 0); the pointers are baked into the graph and must stay valid
 * while the batch exists (their contents may change between launches).
 *   - Tensor-core plans of one transform form a family, imaged by ONE persistent
 *     launch of one CTA per SM: every plan's call is cut into time tiles (W
 *     consecutive (channel, sample) units), listed in a device work list
 *     (largest tiles first), and claimed by the CTAs one at a time; each plan's
 *     partial images are then reduced by its own small kernel.  The batch owns
 *     these partial images.
 *   - FP32 plans run their own imaging kernel and reduction, each plan on its
 *     own graph branch so that the arrays overlap on the SMs.
 * tune = 1 runs the autotuner first: it times candidate graphs (for FP32 plans
 * each plan's CTA count, i.e. its time-tile length: all SMs, shares
 * proportional to the plans' work, halved and quartered caps; for a tensor-core
 * family its members' tile length: 1, 2, 3 or 4 tiles per SM and plan) and
 * keeps the fastest; this launches the imaging kernels several times on
 * `stream` and overwrites d_out.  chosen_ctas (optional, [n_plans]) receives
 * each plan's CTA cap (FP32) or tile count cap (tensor core) in the graph.
 * Synchronous.  Results equal epic_image's exactly when tune = 0 (every tile is
 * the span one CTA of a single call images), and up to the summation order of
 * the partial images (FP32 rounding) when tune = 1.  FP32 plans use their own
 * workspace: a plan in a batch must not run other calls (epic_image,
 * epic_grad, another batch) concurrently with a launch.  A bounded wait that
 * gives up inside a family's launch is reported by epic_sync on the plan whose
 * tile was being imaged. */
epic_status epic_batch_create(epic_plan* const* plans, int n_plans, const uint8_t* const* d_volts,
                              const int* n_time, float* const* d_out, int tune, int* chosen_ctas,
                              void* stream, epic_batch** out);

/* One launch of the batch's graph on stream (asynchronous). */
epic_status epic_batch_launch(epic_batch* batch, void* stream);

/* Debug: the failure path of a batch's bounded-spin reduction claims.  (No
 * counterpart in the paper: the test hook of the library's own failure
 * detection.)  Runs, outside the batch's graph, the persistent launch of every
 * tensor-core family whose reductions run in the launch, with each reduction
 * item waiting for one completion signal more than its imaging items send,
 * limited to wait_ns (1 000 .. 1 000 000 000).  The imaging items complete; every
 * reduction item gives up, sets its plan's device status to a time-out and skips
 * its rows (the outputs are left unspecified).  The next epic_sync of a member
 * plan returns EPIC_ERR_TIMEOUT and clears the status; the batch and its plans
 * are usable as before.  EPIC_ERR_UNSUPPORTED when no family of the batch reduces
 * in its launch. */
epic_status epic_debug_batch_timeout(epic_batch* batch, long long wait_ns, void* stream);

/* Frees the batch (synchronises the device); the plans are not destroyed. */
epic_status epic_batch_destroy(epic_batch* batch);

/* Waits for the stream and reports any device-side error recorded by the
 * plan's kernels since the previous call (EPIC_ERR_TIMEOUT, EPIC_ERR_CUDA). */
epic_status epic_sync(epic_plan* plan, void* stream);

/* Human-readable name of a status code (static storage). */
const char* epic_status_string(int status);

/* Debug: unpacks n bytes (Sec. 3.2 format above) into d_out [n][2] int8 as
 * (real, imaginary).  Needs no plan. */
epic_status epic_debug_unpack(const uint8_t* d_in, size_t n, int8_t* d_out, void* stream);

/* Debug: the gridded, calibrated field G = W * E' (Eq. (5)) of sample t,
 * channel c, polarisation p of d_volts (layout as in epic_image, n_time
 * samples), as d_grid [N][N][2] float (row y, column x, re/im), computed with
 * the imaging kernels' own gather code. */
epic_status epic_debug_grid(epic_plan* plan, const uint8_t* d_volts, int n_time, int t, int c,
                            int p, float* d_grid, void* stream);

/* Debug: the pre-square image Y = FT{W * E'} (Eq. (5) before squaring) of sample
 * t, channel c, polarisation p, as d_y [N][N][2] float (row m, column l, re/im;
 * pixel N/2 is the zero frequency), computed with the imaging kernel's own
 * line transforms and shared-memory layouts on the field that epic_debug_grid
 * returns.  FP32 FFT plans with N = 32 or 64 (else EPIC_ERR_UNSUPPORTED). */
epic_status epic_debug_transform(epic_plan* plan, const uint8_t* d_volts, int n_time, int t, int c, int p,
                                 float* d_y, void* stream);

/* Debug: copies the plan's gridding tables to the host and checks them: every
 * antenna, cell and entry index the imaging kernels dereference lies within
 * the plan's sizes, each (warp, slot) range tiles its table set, and every
 * lane's entry list equals the one re-derived from the per-cell table (the
 * antennas whose kernel box covers the cell, in antenna order, folded with
 * signs on folded grids), followed by weight-0 padding.  Writes a one-line
 * summary or the first violated invariant to report (report_len bytes, may be
 * NULL).  Returns EPIC_OK or EPIC_ERR_INTERNAL.  Synchronous. */
epic_status epic_debug_check_plan(const epic_plan* plan, char* report, size_t report_len);

/* Debug: the failure path of the tensor-core kernel's bounded waits.  (No
 * counterpart in the paper: the test hook of the library's own failure
 * detection.)  Runs the imaging kernel of a tensor-core plan over d_volts
 * (layout as in epic_image, 1 <= n_time <= info.max_time) with the first
 * mbarrier wait of every CTA made on a barrier that nothing ever arrives at,
 * limited to wait_ns (1 000 .. 1 000 000 000).  Every CTA gives up on that
 * wait, sets the plan's device status to a time-out, waits (bounded, one second)
 * for the tensor-core products it has already issued, releases its tensor memory
 * and returns; no output is written.  The next epic_sync(plan, stream) returns
 * EPIC_ERR_TIMEOUT and clears the status, after which the plan and the device
 * are usable as before.  EPIC_ERR_UNSUPPORTED for FP32 plans. */
epic_status epic_debug_image_timeout(epic_plan* plan, const uint8_t* d_volts, int n_time, long long wait_ns,
                                     void* stream);

/* Debug: the FP32 FMA rate the GPU sustains, measured by a kernel of
 * independent dependent-FMA chains filling every SM (2 flop per FMA).  One
 * warm-up launch, then one timed launch of `iterations` (1 .. 2^32) loop trips
 * of 128 FMAs per thread, CUDA events on `stream`; *tflops receives TFLOP/s.
 * Synchronous.  The denominator check of the FP32 path's roofline, whose peak
 * is derived as SMs x 128 FP32 lanes x 2 flop x SM clock. */
epic_status epic_debug_fma_rate(long long iterations, double* tflops, void* stream);

/* Device time per kernel kind of a plan's launches, for benchmarks. */
typedef struct {
  char kernel[32];      /* kernel kind, e.g. "fft_image", "reduce"              */
  long long launches;   /* launches recorded since timing was enabled          */
  double total_ms;      /* summed device time of those launches (CUDA events)  */
} epic_kernel_time;

/* enable = 1: from now on every launch the plan makes is bracketed by CUDA
 * events on its stream; enable = 0: stop recording.  Both clear the counters.
 * Recording costs two event records per launch. */
epic_status epic_timing_enable(epic_plan* plan, int enable);

/* Waits for every recorded launch, then writes up to capacity entries to out
 * (one per kernel kind seen) and the number of kinds to *count. */
epic_status epic_timing_read(epic_plan* plan, epic_kernel_time* out, int capacity, int* count);

#ifdef __cplusplus
}
#endif

#endif /* EPIC_H */
