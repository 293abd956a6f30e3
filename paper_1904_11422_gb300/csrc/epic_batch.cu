// epic_batch.cu -- many imaging problems in one graph launch.
//
// A batch holds several plans (arrays of different antenna counts, grid sizes
// and channel counts) with their input and output buffers.  All their launches
// are captured once into a CUDA graph, each plan on its own branch so that the
// arrays run concurrently on the SMs, and epic_batch_launch replays the graph
// with a single launch call.  An optional autotuner chooses each plan's CTA
// count (how many SMs its persistent imaging kernel spreads over, i.e. its
// time-tile length) by timing candidate graphs.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <new>
#include <vector>

#include "epic_internal.cuh"

struct epic_batch {
  std::vector<epic_plan*> plans;
  std::vector<const uint8_t*> volts;
  std::vector<int> n_time;
  std::vector<float*> outs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // capture stream (the legacy default stream cannot be captured)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> ctas;  // CTA cap of each plan in the captured graph
};

namespace {

epic_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return EPIC_OK;
  if (e == cudaErrorMemoryAllocation) return EPIC_ERR_OOM;
  return EPIC_ERR_CUDA;
}

void drop_graph(epic_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Captures every plan's imaging launches with the given CTA caps (on the batch's
// own capture stream).
cudaError_t capture(epic_batch* b, const std::vector<int>& caps) {
  cudaStream_t s0 = b->cap;
  drop_graph(b);
  std::vector<int> saved(b->plans.size());
  for (size_t i = 0; i < b->plans.size(); ++i) {
    saved[i] = b->plans[i]->p.ctas_use;
    b->plans[i]->p.ctas_use = caps[i];
  }
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = cudaEventRecord(b->fork, s0);
    for (size_t i = 0; i < b->plans.size() && le == cudaSuccess; ++i) {
      le = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
      if (le == cudaSuccess)
        le = epic::image_launches(b->plans[i]->p, b->volts[i], b->n_time[i], b->outs[i], 0, b->streams[i]);
      if (le == cudaSuccess) le = cudaEventRecord(b->joins[i], b->streams[i]);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(s0, b->joins[i], 0);
    }
    e = cudaStreamEndCapture(s0, &b->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  for (size_t i = 0; i < b->plans.size(); ++i) b->plans[i]->p.ctas_use = saved[i];
  if (e == cudaSuccess) b->ctas = caps;
  return e;
}

// Average milliseconds of one graph launch (after one warm-up launch).
cudaError_t time_graph(epic_batch* b, cudaStream_t s, int reps, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  *ms = t / reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

// A cap is usable when the split it gives fits the plan's partial-image slots.
bool cap_fits(const epic::Plan& p, int T, int cap) {
  if (T == 0) return true;
  epic::WorkSplit ws;
  ws.T = T;
  ws.units = (long long)p.C * p.vq * T;
  const long long ctas = cap < ws.units ? cap : ws.units;
  ws.W = (ws.units + ctas - 1) / ctas;
  ws.ctas = (int)((ws.units + ws.W - 1) / ws.W);
  int worst = 1;
  for (int b = 0; b < ws.ctas; ++b) {
    const long long u0 = (long long)b * ws.W;
    const long long u1 = (u0 + ws.W < ws.units ? u0 + ws.W : ws.units) - 1;
    worst = std::max(worst, (int)(u1 / T - u0 / T) + 1);
  }
  return (long long)ws.ctas * worst <= (long long)p.ctas * p.spans;
}

}  // namespace

extern "C" {

epic_status epic_batch_create(epic_plan* const* plans, int n_plans, const uint8_t* const* d_volts,
                              const int* n_time, float* const* d_out, int tune, int* chosen_ctas, void* stream,
                              epic_batch** out) {
  if (!out) return EPIC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!plans || !d_volts || !n_time || !d_out || n_plans < 1 || n_plans > 64 || (tune != 0 && tune != 1))
    return EPIC_ERR_INVALID_ARG;
  for (int i = 0; i < n_plans; ++i) {
    if (!plans[i] || !d_out[i] || n_time[i] < 0 || n_time[i] > (1 << 24) || (n_time[i] > 0 && !d_volts[i]))
      return EPIC_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return EPIC_ERR_INVALID_ARG;  // one workspace per plan
  }
  epic_batch* b = new (std::nothrow) epic_batch();
  if (!b) return EPIC_ERR_OOM;
  b->plans.assign(plans, plans + n_plans);
  b->volts.assign(d_volts, d_volts + n_plans);
  b->n_time.assign(n_time, n_time + n_plans);
  b->outs.assign(d_out, d_out + n_plans);
  cudaStream_t s0 = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  b->streams.resize(n_plans, nullptr);
  b->joins.resize(n_plans, nullptr);
  for (int i = 0; i < n_plans && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
  }
  std::vector<int> caps(n_plans);
  for (int i = 0; i < n_plans; ++i) caps[i] = plans[i]->p.ctas;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = capture(b, caps);
  if (e == cudaSuccess && tune) {
    // Autotuner: start from every plan on all its CTAs; try CTA shares
    // proportional to each plan's work, then halve / quarter each plan's cap in
    // turn, keeping whatever lowers the measured time of the whole graph.
    float best = 0.f;
    e = time_graph(b, s0, 3, &best);
    std::vector<int> best_caps = caps;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double total = 0.0;
    std::vector<double> work(n_plans);
    for (int i = 0; i < n_plans; ++i) {
      const epic::Plan& p = plans[i]->p;
      work[i] = (double)p.C * n_time[i] * p.N * p.N * (p.xform == EPIC_XFORM_FFT_FP32 ? 1.0 : 0.7);
      total += work[i];
    }
    std::vector<std::vector<int>> trials;
    if (total > 0.0) {
      std::vector<int> prop(n_plans);
      for (int i = 0; i < n_plans; ++i)
        prop[i] = std::max(1, std::min(plans[i]->p.ctas, (int)(sms * work[i] / total + 0.5)));
      trials.push_back(prop);
    }
    for (int i = 0; i < n_plans; ++i)
      for (int div : {2, 4}) {
        std::vector<int> t = best_caps;
        t[i] = std::max(1, t[i] / div);
        trials.push_back(t);
      }
    for (const auto& t : trials) {
      if (e != cudaSuccess) break;
      bool ok = true;
      for (int i = 0; i < n_plans; ++i) ok = ok && cap_fits(plans[i]->p, n_time[i], t[i]);
      if (!ok) continue;
      e = capture(b, t);
      float ms = 0.f;
      if (e == cudaSuccess) e = time_graph(b, s0, 3, &ms);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_caps = t;
      }
    }
    if (e == cudaSuccess) e = capture(b, best_caps);
  }
  if (e != cudaSuccess) {
    epic_batch_destroy(b);
    return status_of(e);
  }
  if (chosen_ctas)
    for (int i = 0; i < n_plans; ++i) chosen_ctas[i] = b->ctas[i];
  *out = b;
  return EPIC_OK;
}

epic_status epic_batch_launch(epic_batch* b, void* stream) {
  if (!b || !b->exec) return EPIC_ERR_INVALID_ARG;
  nvtxRangePushA("epic_batch_launch");
  const epic_status st = status_of(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
  nvtxRangePop();
  return st;
}

epic_status epic_batch_destroy(epic_batch* b) {
  if (!b) return EPIC_OK;
  cudaDeviceSynchronize();
  drop_graph(b);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t ev : b->joins)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return EPIC_OK;
}

}  // extern "C"
