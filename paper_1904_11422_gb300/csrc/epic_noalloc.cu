// epic_noalloc.cu -- epic_image_noalloc: the imaging call for callers that must
// not allocate device memory while they run.
//
// Some callers may not call cudaMalloc (or anything that allocates) once they
// are running: a real-time streaming loop that must finish each block within its
// time budget cannot risk an allocation, which can stall on device-wide
// synchronisation; an application that owns its whole device-memory budget
// through its own allocator may forbid allocations outside it.  This entry point
// runs the same two kernels as epic_image, with the same work split, but takes
// their scratch space (the per-CTA partial images and self powers) from one
// file-scope static device array instead of the plan's workspace, and calls
// nothing that allocates.  (Plans imaged by two-CTA clusters keep using the
// exchange buffer they allocated when they were created.)
//
// The array is EPIC_NOALLOC_SCRATCH_BYTES (32 MiB); every GPU that loads this
// library holds it until the process exits.  Host code cannot use the array's
// name as a device address, so its address is looked up with
// cudaGetSymbolAddress by the first call made with a device current, and again
// whenever that device's current context has changed since (for example after
// cudaDeviceReset, which unloads the library's device code).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "epic_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[EPIC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
struct ScratchAddr {
  unsigned long long ctx_id = 0;  // the context the address belongs to (0: none yet)
  void* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Unique id of the calling thread's current context (driver entry points
// resolved through the runtime, so the library links no driver library).
cudaError_t current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorNotSupported;
    g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
    g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the static scratch array on the current device dev.
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  // cudaSetDevice of the current device binds its primary context to this
  // thread if no context is current yet (it allocates nothing)
  cudaError_t e = cudaSetDevice(dev);
  unsigned long long id = 0;
  if (e == cudaSuccess) e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  ScratchAddr& s = g_scratch[dev];
  if (s.ctx_id != id || !s.ptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    s.ptr = ptr;
    s.ctx_id = id;
  }
  *out = s.ptr;
  return cudaSuccess;
}

epic_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return EPIC_OK;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return EPIC_ERR_NO_DEVICE;
  return EPIC_ERR_CUDA;
}

}  // namespace

extern "C" epic_status epic_image_noalloc(epic_plan* h, const uint8_t* d_volts, int n_time, float* d_out,
                                          int accumulate, void* stream) {
  if (!h || !d_out || n_time < 0 || n_time > (1 << 24) || (accumulate != 0 && accumulate != 1))
    return EPIC_ERR_INVALID_ARG;
  if (n_time > 0 && !d_volts) return EPIC_ERR_INVALID_ARG;
  const epic::Plan& p = h->p;
  if (p.xform != EPIC_XFORM_FFT_FP32) return EPIC_ERR_UNSUPPORTED;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  if (dev != p.device) return EPIC_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t out_n = (size_t)p.C * 4 * p.N * p.N;
  if (n_time == 0) return accumulate ? EPIC_OK : status_of(epic::launch_zero(d_out, out_n, s));

  // The split of epic_image (same CTAs, same unit ranges), so both entry points
  // sum in the same order and give the same bits.
  const epic::WorkSplit ws = epic::split_work(p, n_time);
  if (!epic::split_fits(p, ws)) return EPIC_ERR_UNSUPPORTED;

  // Scratch of this call: partial images [ctas][spans][4][Ns][Ns] float, then
  // self powers [ctas][spans][A][4] int, each rounded up to 256 bytes.  Every
  // slot the reduction reads is written by the imaging kernel of the same call
  // first, so nothing needs clearing; what the previous call left in the array
  // is never read.
  const size_t Ns = p.vq == 4 ? p.N / 2 : (size_t)p.N * p.dec;  // side of a partial image
  const size_t slots = (size_t)ws.ctas * ws.spans;
  const size_t part_bytes = align256(sizeof(float) * slots * 4 * Ns * Ns);
  const size_t auto_bytes = align256(sizeof(int) * slots * p.A * 4);
  if (part_bytes + auto_bytes > (size_t)EPIC_NOALLOC_SCRATCH_BYTES) return EPIC_ERR_UNSUPPORTED;

  void* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return status_of(e);
  float* part = static_cast<float*>(base);
  int* part_auto = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + part_bytes);

  e = epic::launch_fft_image_ws(p, d_volts, n_time, ws, part, part_auto, s);
  if (e != cudaSuccess) return status_of(e);
  return status_of(epic::launch_reduce_ws(p, n_time, ws, part, part_auto, d_out, accumulate, s));
}
