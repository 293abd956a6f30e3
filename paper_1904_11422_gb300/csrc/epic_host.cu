// epic_host.cu -- epic_image_host_async: imaging from page-locked host buffers
// with the transfers of consecutive calls overlapping the imaging.
//
// A streaming imager (Sec. 3.1: gulps of voltages arriving back to back) spends
// a block's host-to-device copy and its result copy outside the kernels when
// every call waits for its own transfers.  Here a call only enqueues work: the
// input goes to one of two device staging slots on the plan's input-copy stream,
// the imaging runs on the caller's stream once that copy has landed, and the
// images return to the host on the plan's result-copy stream.  Slots alternate
// between calls, so the input copy of call i + 1 runs while call i is imaged.
// Events order every reuse of a slot: its input is overwritten only after the
// imaging of the call two back has read it, and its output only after that
// call's images have been copied out.  The kernels are the same as epic_image's,
// so the images are identical bit for bit.
#include "epic_internal.cuh"

namespace {

bool pinned(const void* ptr) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

epic_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return EPIC_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? EPIC_ERR_OOM : EPIC_ERR_CUDA;
}

}  // namespace

namespace epic {

void free_host_pipe(Plan& p) {
  Plan::HostPipe& q = p.pipe;
  if (q.h2d) cudaStreamSynchronize(q.h2d);
  if (q.d2h) cudaStreamSynchronize(q.d2h);
  for (int k = 0; k < 2; ++k) {
    if (q.copied[k]) cudaEventDestroy(q.copied[k]);
    if (q.computed[k]) cudaEventDestroy(q.computed[k]);
    if (q.returned[k]) cudaEventDestroy(q.returned[k]);
    if (q.d_in[k]) cudaFree(q.d_in[k]);
    if (q.d_out[k]) cudaFree(q.d_out[k]);
  }
  if (q.h2d) cudaStreamDestroy(q.h2d);
  if (q.d2h) cudaStreamDestroy(q.d2h);
  q = Plan::HostPipe();
}

}  // namespace epic

extern "C" epic_status epic_image_host_async(epic_plan* h, const uint8_t* h_volts, int n_time, float* h_out,
                                             int accumulate, void* stream) {
  if (!h || !h_out || n_time < 0 || n_time > (1 << 24) || (accumulate != 0 && accumulate != 1))
    return EPIC_ERR_INVALID_ARG;
  if (n_time > 0 && (!h_volts || !pinned(h_volts))) return EPIC_ERR_INVALID_ARG;
  if (!pinned(h_out)) return EPIC_ERR_INVALID_ARG;
  epic_plan_info info{};
  epic_status st = epic_plan_query(h, &info);
  if (st != EPIC_OK) return st;
  const size_t in_bytes = (size_t)n_time * info.n_chan * info.n_ant * info.n_pol;
  const size_t out_bytes = sizeof(float) * (size_t)info.n_chan * 4 * info.grid_n * info.grid_n;
  epic::Plan::HostPipe& q = h->p.pipe;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;

  if (!q.h2d) {  // first call: streams, events and the output slots
    e = cudaStreamCreateWithFlags(&q.h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q.d2h, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&q.copied[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.computed[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.returned[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&q.d_out[k]), out_bytes);
    }
    if (e != cudaSuccess) {
      epic::free_host_pipe(h->p);
      return status_of(e);
    }
  }
  if (in_bytes > q.in_bytes) {  // grow both input slots (rare): wait until neither is in use
    e = cudaDeviceSynchronize();
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      if (q.d_in[k]) cudaFree(q.d_in[k]);
      q.d_in[k] = nullptr;
    }
    q.in_bytes = 0;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(reinterpret_cast<void**>(&q.d_in[k]), in_bytes);
    if (e != cudaSuccess) {
      for (int k = 0; k < 2; ++k) {
        if (q.d_in[k]) cudaFree(q.d_in[k]);
        q.d_in[k] = nullptr;
      }
      return status_of(e);
    }
    q.in_bytes = in_bytes;
  }

  const int k = q.slot;
  q.slot ^= 1;
  // 1. input (and, to accumulate, the current output) into slot k, once the
  //    call that last used the slot has been imaged and its images copied out
  e = cudaStreamWaitEvent(q.h2d, q.computed[k], 0);
  if (e == cudaSuccess && in_bytes) e = cudaMemcpyAsync(q.d_in[k], h_volts, in_bytes, cudaMemcpyHostToDevice, q.h2d);
  if (e == cudaSuccess && accumulate) {
    // h_out may be the previous call's destination: wait for every result copy
    e = cudaStreamWaitEvent(q.h2d, q.returned[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q.h2d, q.returned[k ^ 1], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q.d_out[k], h_out, out_bytes, cudaMemcpyHostToDevice, q.h2d);
  }
  if (e == cudaSuccess) e = cudaEventRecord(q.copied[k], q.h2d);
  // 2. imaging on the caller's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, q.copied[k], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, q.returned[k], 0);
  if (e != cudaSuccess) return status_of(e);
  st = epic_image(h, q.d_in[k], n_time, q.d_out[k], accumulate, stream);
  if (st != EPIC_OK) return st;
  e = cudaEventRecord(q.computed[k], s);
  // 3. images back to the host
  if (e == cudaSuccess) e = cudaStreamWaitEvent(q.d2h, q.computed[k], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, q.d_out[k], out_bytes, cudaMemcpyDeviceToHost, q.d2h);
  if (e == cudaSuccess) e = cudaEventRecord(q.returned[k], q.d2h);
  return status_of(e);
}
