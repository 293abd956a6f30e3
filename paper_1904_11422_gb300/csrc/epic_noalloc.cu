// epic_noalloc.cu -- epic_image_noalloc: the imaging call for callers that must
// not allocate device memory while they run.
//
// Some callers may not call cudaMalloc (or anything that allocates) once they
// are running: a real-time streaming loop that must finish each block within its
// time budget cannot risk an allocation, which can stall on device-wide
// synchronisation; an application that owns its whole device-memory budget
// through its own allocator may forbid allocations outside it.  This entry point
// runs the same two kernels as epic_image, but takes their scratch space (the
// per-CTA partial images and self powers) from one file-scope static device
// array instead of the plan's workspace, and calls nothing that allocates.
//
// The array is EPIC_NOALLOC_SCRATCH_BYTES (32 MiB); every GPU that loads this
// library holds it until the process exits.  Its device address is looked up
// with cudaGetSymbolAddress once per device, by the first call made with that
// device current (host code cannot use the array's name as a device address).
#include <mutex>

#include "epic_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[EPIC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the static scratch array on the current device.
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
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
  const size_t Ns = p.vq == 4 ? p.N / 2 : (size_t)p.N * p.dec;  // side of a partial image
  const size_t part_bytes = align256(sizeof(float) * (size_t)p.ctas * p.spans * 4 * Ns * Ns);
  const size_t auto_bytes = align256(sizeof(int) * (size_t)p.ctas * p.spans * p.A * 4);
  if (part_bytes + auto_bytes > (size_t)EPIC_NOALLOC_SCRATCH_BYTES) return EPIC_ERR_UNSUPPORTED;
  const size_t out_n = (size_t)p.C * 4 * p.N * p.N;
  if (n_time == 0) return accumulate ? EPIC_OK : status_of(epic::launch_zero(d_out, out_n, s));

  // The same split of the (c, t) units over the plan's CTAs as epic_image, so
  // both entry points sum in the same order.
  epic::WorkSplit ws;
  ws.T = n_time;
  ws.units = (long long)p.C * p.vq * n_time;
  const long long ctas = p.ctas < ws.units ? p.ctas : ws.units;
  ws.W = (ws.units + ctas - 1) / ctas;
  ws.ctas = (int)((ws.units + ws.W - 1) / ws.W);
  ws.spans = p.spans;

  // Partial images [ctas][spans][4][N][N] float, then self powers
  // [ctas][spans][A][4] int.  Every slot the reduction reads is written by the
  // imaging kernel of the same call first, so nothing needs clearing; what the
  // previous call left in the array is never read.
  // (sized above for the plan's largest launch, p.ctas CTAs, whatever n_time is)

  void* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return status_of(e);
  float* part = static_cast<float*>(base);
  int* part_auto = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + part_bytes);

  e = epic::launch_fft_image_ws(p, d_volts, n_time, ws, part, part_auto, s);
  if (e != cudaSuccess) return status_of(e);
  return status_of(epic::launch_reduce_ws(p, n_time, ws, part, part_auto, d_out, accumulate, s));
}
