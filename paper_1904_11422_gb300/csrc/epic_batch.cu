// epic_batch.cu -- many imaging problems in one graph launch.
//
// A batch holds several plans (arrays of different antenna counts, grid sizes
// and channel counts) with their input and output buffers.  All their launches
// are captured once into a CUDA graph, and epic_batch_launch replays the graph
// with a single launch call.
//
// Plans on the tensor-core path that share a transform form one family: their
// calls are cut into items (a time tile: W consecutive (channel, sample) units
// of one plan, the span one CTA of a single call would image) and listed in one
// device work list; a single persistent launch of one CTA per SM claims items
// from it (an atomic counter, largest items first) until none is left, so the
// ragged arrays -- 32 x 32, 64 x 64 and 128 x 128 grids, any antenna count --
// share every SM.  Each plan's partial images are then summed by its own
// reduction.  FP32 plans run their own imaging kernel and reduction, each plan
// on its own graph branch so that the arrays overlap on the SMs.
//
// An optional autotuner times candidate graphs: for the FP32 plans each plan's
// CTA count (its time-tile length), for a tensor-core family the tile length of
// every member (items per plan = 1, 2, 3 or 4 times the SM count).
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <new>
#include <vector>

#include "epic_internal.cuh"
#include "epic_reduce.cuh"

// One tensor-core family of a batch: its members (plan indices), the
// batch-owned partial images of each member (sized for the finest tiling the
// tuner tries), the device work list and claim counter, and the tiling in the
// captured graph.
struct TensorFamily {
  int xform = 0;
  std::vector<int> members;
  std::vector<float*> part;
  std::vector<int*> part_auto;
  std::vector<epic::WorkSplit> ws;  // each member's split (its items) in the captured graph
  epic::DftJob* d_jobs = nullptr;
  int* d_head = nullptr;
  int* d_done = nullptr;            // per member and virtual channel: imaging items that have signalled
  int n_done = 0, n_image_items = 0, n_items = 0;
  int A_lay = 0, max_ent = 0, ctas = 0;
  int mult = 1;  // items per member: mult x the plan's CTA count (its split's cap)
  // reductions as items of the same launch (waiting on the completion counters),
  // or as each member's own reduction kernel after it
  bool inkernel = true;
};

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
  std::vector<TensorFamily> families;
  std::vector<int> family_of;  // plan -> family index, -1 for FP32 plans
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

// Per-unit cost of a tensor-core plan's items, for ordering the work list
// (largest items first): the transform, plus the gather's padded entries of its
// largest (virtual) channel relative to the station array's 12 000.
double unit_cost(const epic::Plan& p) { return 1.0 + 0.5 * p.gt.max_chan_entries / 12000.0; }

// Splits every member of a family into mult x (its CTA count) items, writes the
// work list (largest items first) to the device, and records the splits.
cudaError_t prepare_family(epic_batch* b, TensorFamily& f, int mult, bool inkernel) {
  const size_t n = f.members.size();
  std::vector<int> order(n);
  for (size_t k = 0; k < n; ++k) order[k] = (int)k;
  std::vector<epic::WorkSplit> ws(n);
  std::vector<double> item_cost(n);
  for (size_t k = 0; k < n; ++k) {
    const epic::Plan& p = b->plans[f.members[k]]->p;
    ws[k] = epic::split_work_cap(p, b->n_time[f.members[k]], mult * p.ctas);
    item_cost[k] = (double)ws[k].W * unit_cost(p);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return item_cost[x] > item_cost[y]; });
  std::vector<epic::DftJob> jobs(n);
  int first = 0, done_off = 0;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (size_t j = 0; j < n; ++j) {
    const int k = order[j];
    const epic::Plan& p = b->plans[f.members[k]]->p;
    epic::DftJob job = epic::dft_job(p, b->volts[f.members[k]], b->n_time[f.members[k]], ws[k], f.part[k],
                                     f.part_auto[k]);
    // gather entries in shared memory when the family's layout holds them
    job.ent_in_smem = (p.gt.max_chan_entries <= f.max_ent &&
                       epic::dft_batch_smem(f.A_lay, f.max_ent) <= (size_t)optin) ? 1 : 0;
    job.first_item = first;
    job.n_items = b->n_time[f.members[k]] > 0 ? ws[k].ctas : 0;
    first += job.n_items;
    // its block-end reduction, in pieces of whole rows of one virtual channel
    // whose staging (A float4 + A x rows floats) fits the kernel's 128 KB of
    // operand slabs, which are idle once a CTA has no imaging item left
    const int L = p.vq == 4 ? p.N / 2 : p.N;
    const int rows = epic::reduce_rows_per_piece(L, 512 * epic::kBatchReducePix, p.A, 128 * 1024);
    job.red = epic::ReduceArgs{b->n_time[f.members[k]], p.C, p.A, p.N, p.vq, p.dec, ws[k].ctas, ws[k].spans,
                               p.subtract, 0, ws[k].W, f.part[k], f.part_auto[k], p.d_coef64, p.d_kx2,
                               p.d_ky2, b->outs[f.members[k]]};
    job.done = f.d_done + done_off;
    done_off += p.C * p.vq;
    job.red_rows = rows;
    job.n_red = (inkernel && job.n_items > 0) ? p.C * p.vq * (L / rows) : 0;
    jobs[j] = job;
  }
  f.n_image_items = first;
  for (size_t j = 0; j < n; ++j) {
    jobs[j].red_first = first;
    first += jobs[j].n_red;
  }
  f.n_items = first;
  f.ws = ws;
  f.mult = mult;
  f.inkernel = inkernel;
  return cudaMemcpy(f.d_jobs, jobs.data(), sizeof(epic::DftJob) * n, cudaMemcpyHostToDevice);
}

// The launches of one family: reset the claim and completion counters, then
// one persistent launch that images every member's time tiles and reduces every
// member's channels (a member with no samples gets its output zeroed).
// test_wait_ns > 0 (failure test): every reduction item waits for one signal
// more than can come, for at most test_wait_ns.
cudaError_t family_launches(epic_batch* b, const TensorFamily& f, cudaStream_t s,
                            unsigned long long test_wait_ns = 0) {
  const float2* twiddle = nullptr;
  for (int i : f.members)
    if (b->plans[i]->p.N == 128) twiddle = b->plans[i]->p.d_twiddle;
  cudaError_t e = cudaMemsetAsync(f.d_head, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.d_done, 0, sizeof(int) * f.n_done, s);
  if (e == cudaSuccess && f.n_items > 0) {
    const epic::DftQueue q{f.d_jobs, (int)f.members.size(), f.n_items, f.n_image_items, f.d_head,
                           test_wait_ns ? 1 : 0, test_wait_ns};
    e = epic::launch_dft_batch(f.xform, q, f.A_lay, f.max_ent, b->plans[f.members[0]]->p.d_fmat, twiddle,
                               std::min(f.ctas, f.n_items), s);
  }
  for (size_t k = 0; k < f.members.size() && e == cudaSuccess; ++k) {
    const int i = f.members[k];
    const epic::Plan& p = b->plans[i]->p;
    if (b->n_time[i] == 0)
      e = epic::launch_zero(b->outs[i], (size_t)p.C * 4 * p.N * p.N, s);
    else if (!f.inkernel)
      e = epic::launch_reduce_ws(p, b->n_time[i], f.ws[k], f.part[k], f.part_auto[k], b->outs[i], 0, s);
  }
  return e;
}

// Captures the batch (on its own capture stream): every FP32 plan's imaging
// launches with the given CTA caps on a branch of its own, every tensor-core
// family's launches on the branch of its first member.
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
      const int fam = b->family_of[i];
      if (fam >= 0 && b->families[fam].members[0] != (int)i) continue;  // imaged by its family's launch
      le = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
      if (le == cudaSuccess)
        le = fam >= 0 ? family_launches(b, b->families[fam], b->streams[i])
                      : epic::image_launches(b->plans[i]->p, b->volts[i], b->n_time[i], b->outs[i], 0,
                                             b->streams[i]);
      if (le == cudaSuccess) le = cudaEventRecord(b->joins[i], b->streams[i]);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(s0, b->joins[i], 0);
    }
    e = cudaStreamEndCapture(s0, &b->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  for (size_t i = 0; i < b->plans.size(); ++i) b->plans[i]->p.ctas_use = saved[i];
  if (e == cudaSuccess) {
    b->ctas = caps;
    for (const TensorFamily& f : b->families)
      for (size_t k = 0; k < f.members.size(); ++k) b->ctas[f.members[k]] = f.mult * b->plans[f.members[k]]->p.ctas;
  }
  return e;
}

// Groups the tensor-core plans by transform and allocates each family's work
// list, claim counter and partial images (for up to kMaxMult x each plan's
// CTA count items).
constexpr int kMaxMult = 4;
cudaError_t make_families(epic_batch* b) {
  b->family_of.assign(b->plans.size(), -1);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const epic::Plan& p = b->plans[i]->p;
    if (p.xform == EPIC_XFORM_FFT_FP32) continue;
    int fam = -1;
    for (size_t g = 0; g < b->families.size(); ++g)
      if (b->families[g].xform == p.xform) fam = (int)g;
    if (fam < 0) {
      b->families.emplace_back();
      b->families.back().xform = p.xform;
      fam = (int)b->families.size() - 1;
    }
    b->family_of[i] = fam;
    b->families[fam].members.push_back((int)i);
  }
  for (TensorFamily& f : b->families) {
    f.ctas = sms;  // one CTA per SM (each holds all 512 tensor-memory columns)
    for (int i : f.members) f.n_done += b->plans[i]->p.C * b->plans[i]->p.vq;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&f.d_jobs), sizeof(epic::DftJob) * f.members.size());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&f.d_head), sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&f.d_done), sizeof(int) * f.n_done);
    if (e != cudaSuccess) return e;
    for (int i : f.members) {
      const epic::Plan& p = b->plans[i]->p;
      f.A_lay = std::max(f.A_lay, p.A);
      if (p.ent_in_smem) f.max_ent = std::max(f.max_ent, p.gt.max_chan_entries);
      size_t slots = 0;
      if (b->n_time[i] > 0)
        for (int m = 1; m <= kMaxMult; ++m) {
          const epic::WorkSplit ws = epic::split_work_cap(p, b->n_time[i], m * p.ctas);
          slots = std::max(slots, (size_t)ws.ctas * ws.spans);
        }
      const size_t Ns = p.vq == 4 ? p.N / 2 : (size_t)p.N * p.dec;
      float* part = nullptr;
      int* pa = nullptr;
      if (slots) {
        e = cudaMalloc(reinterpret_cast<void**>(&part), sizeof(float) * slots * 4 * Ns * Ns);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&pa), sizeof(int) * slots * p.A * 4);
      }
      f.part.push_back(part);
      f.part_auto.push_back(pa);
      if (e != cudaSuccess) return e;
    }
    // the shared-memory layout must fit: drop entry tables to L2, largest first
    int dev2 = 0, optin = 0;
    cudaGetDevice(&dev2);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev2);
    while (f.max_ent > 0 && epic::dft_batch_smem(f.A_lay, f.max_ent) > (size_t)optin) {
      int next = 0;
      for (int i : f.members) {
        const int me = b->plans[i]->p.gt.max_chan_entries;
        if (b->plans[i]->p.ent_in_smem && me < f.max_ent) next = std::max(next, me);
      }
      f.max_ent = next;
    }
    if (epic::dft_batch_smem(f.A_lay, f.max_ent) > (size_t)optin) return cudaErrorInvalidConfiguration;
    e = prepare_family(b, f, 1, true);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void free_families(epic_batch* b) {
  for (TensorFamily& f : b->families) {
    if (f.d_jobs) cudaFree(f.d_jobs);
    if (f.d_head) cudaFree(f.d_head);
    if (f.d_done) cudaFree(f.d_done);
    for (float* q : f.part)
      if (q) cudaFree(q);
    for (int* q : f.part_auto)
      if (q) cudaFree(q);
  }
  b->families.clear();
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
  if (e == cudaSuccess) e = make_families(b);
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
    // FP32 plans: CTA counts (tensor-core families keep their own launch)
    double total = 0.0;
    std::vector<double> work(n_plans, 0.0);
    for (int i = 0; i < n_plans; ++i) {
      const epic::Plan& p = plans[i]->p;
      if (b->family_of[i] >= 0) continue;
      work[i] = (double)p.C * n_time[i] * p.N * p.N;
      total += work[i];
    }
    std::vector<std::vector<int>> trials;
    int n_fp32 = 0;
    for (int i = 0; i < n_plans; ++i) n_fp32 += b->family_of[i] < 0;
    if (total > 0.0 && n_fp32 > 1) {
      std::vector<int> prop = best_caps;
      for (int i = 0; i < n_plans; ++i)
        if (b->family_of[i] < 0) prop[i] = std::max(1, std::min(plans[i]->p.ctas, (int)(sms * work[i] / total + 0.5)));
      trials.push_back(prop);
    }
    for (int i = 0; i < n_plans; ++i)
      for (int div : {2, 4}) {
        if (b->family_of[i] >= 0) continue;
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
    // tensor-core families, one at a time: the tile length of every member
    // (items per plan = mult x its CTA count) and where the reductions run
    for (TensorFamily& f : b->families) {
      int best_mult = f.mult;
      bool best_ik = f.inkernel;
      for (int m = 1; m <= kMaxMult && e == cudaSuccess; ++m)
        for (int ik = 1; ik >= 0 && e == cudaSuccess; --ik) {
          if (m == best_mult && (ik != 0) == best_ik) continue;  // the configuration timed already
          e = prepare_family(b, f, m, ik != 0);
          if (e == cudaSuccess) e = capture(b, best_caps);
          float ms = 0.f;
          if (e == cudaSuccess) e = time_graph(b, s0, 3, &ms);
          if (e == cudaSuccess && ms < best) {
            best = ms;
            best_mult = m;
            best_ik = ik != 0;
          }
        }
      if (e == cudaSuccess) e = prepare_family(b, f, best_mult, best_ik);
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

epic_status epic_debug_batch_timeout(epic_batch* b, long long wait_ns, void* stream) {
  if (!b || wait_ns < 1000 || wait_ns > 1000000000LL) return EPIC_ERR_INVALID_ARG;
  bool any = false;
  for (const TensorFamily& f : b->families) any = any || (f.inkernel && f.n_items > f.n_image_items);
  if (!any) return EPIC_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (const TensorFamily& f : b->families) {
    if (!(f.inkernel && f.n_items > f.n_image_items)) continue;
    const cudaError_t e = family_launches(b, f, s, (unsigned long long)wait_ns);
    if (e != cudaSuccess) return status_of(e);
  }
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
  free_families(b);
  delete b;
  return EPIC_OK;
}

}  // extern "C"
