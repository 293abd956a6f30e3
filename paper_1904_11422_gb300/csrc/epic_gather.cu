// epic_gather.cu -- plan-time gather tables of the gridders.
//
// The gridding of Eq. (5) (W * E') is done as a gather: every grid cell sums
// w * e over the antennas whose kernel box covers it (the per-cell table built
// by build_csr_kernel, antenna order).  An imaging kernel thread owns 8 cells
// ("slots"), or 16 on 128 x 128 grids; the 32 threads of a warp walk their k-th
// entries in lock step.
// This file lays those entries out for that walk: for warp w and slot s the
// trip count K_ws is the largest cell count among the warp's 32 cells (rounded
// up to even for the FFT kernel, which walks entries two at a time to keep two
// independent load chains in flight), and entry
// k of lane l sits at base_ws + 32 k + l (the FFT kernel's layouts: at
// base_ws + 64 (k / 2) + 2 l + k % 2, a lane's two entries of a step side by side,
// see entry_pos), cells with fewer entries padded with
// weight-0 entries of antenna 0 (adding +0 leaves every sum unchanged, and the
// real entries keep their antenna order, so the results are the same as a
// per-cell loop).  Loads are coalesced and the loop has no divergence.
//
// Cell layouts (thread task t, slot s -> cell (y, x)):
//   kFft64: y = t / 8, x = t % 8 + 8 s   (the FFT kernel's row layout, N = 64)
//   kFft32: y = t / 4, x = t % 4 + 4 s   (N = 32)
//   kFft128: y = t / 8, x = t % 8 + 8 s, s < 16 (N = 128; 1024 tasks, the
//            two CTAs of a cluster: tasks 512 r + i belong to CTA r)
//   kPair64: four load-balanced cell pairs per thread (tensor path, see deal_pairs)
//   kPairQ: the same over the 64 x 64 field H_q that the tensor path transforms
//           for output-parity subset q of a 128 x 128 grid: H_q(y, x) sums the
//           four grid cells (y + 64 u, x + 64 s), u, s in {0, 1}, with sign
//           (-1)^(alpha s + beta u) (alpha = q & 1, beta = q >> 1); its entry
//           list is the four cells' lists in (u, s) order, weights signed.  One
//           table set per virtual channel 4 c + q.
//   kFft64Q: the kFft64 row layout over the folded fields H_q (the FP32 path's
//           128 x 128 grids run as four 64 x 64 problems), trip counts even.
//   kPairD: the same over a 64 x 64 field holding a 32 x 32 grid in its cells
//           y, x < 32 (zero elsewhere): the tensor path's transform of 32 x 32
//           grids, whose even output pixels are the 32-point transform.
#include "epic_internal.cuh"

namespace epic {

namespace {

// Cell (y, x) of slot s of thread `task` in the FFT row layouts (kFft64, kFft64Q,
// kFft128: eight threads per row; kFft32: four).
__device__ __forceinline__ int2 cell_of(int layout, int task, int s) {
  if (layout == kLayoutFft32) return make_int2(task >> 2, (task & 3) + 4 * s);
  return make_int2(task >> 3, (task & 7) + 8 * s);
}

// Grid cell of field cell (y, x), or -1 where the field is zero (kLayoutPairD
// outside the 32 x 32 grid); not used by the folded layouts.
__device__ __forceinline__ int field_cell(int layout, int N, int y, int x) {
  if (layout == kLayoutPairD) return (y < N && x < N) ? y * N + x : -1;
  return y * N + x;
}

// Entries of cell (y, x) of the gathered field: a grid cell, or for a folded layout
// the four grid cells folded into H_q(y, x).
__device__ __forceinline__ int field_count(int layout, const int* ptr, int N, int y, int x) {
  if (!layout_folded(layout)) {
    const int cell = field_cell(layout, N, y, x);
    return cell < 0 ? 0 : ptr[cell + 1] - ptr[cell];
  }
  int n = 0;
  for (int us = 0; us < 4; ++us) {
    const int cell = (y + 64 * (us >> 1)) * N + x + 64 * (us & 1);
    n += ptr[cell + 1] - ptr[cell];
  }
  return n;
}

// kLayoutPair64 / kLayoutPairQ / kLayoutPairD: the 2048 cell pairs
// (y, 2r..2r+1) of a 64 x 64 field, dealt four per thread.  Slot s of a thread
// is cell (s & 1) of its pair s >> 1, and a warp's gather costs, per slot, the
// largest entry count over its 32 lanes, so a warp costs
//   sum over its four pair slots j of (max K(cell 0) + max K(cell 1)),
// and the block's slowest warp sets the time.  The pairs are ranked by
// (K(cell 0), K(cell 1)) (descending, ties by index) and cut into blocks of 32
// consecutive ranks, whose lanes then hold near-equal counts; the blocks are
// dealt to the warps largest cost first, each to the cheapest warp with a free
// pair slot, and then blocks of the costliest warp are swapped with cheaper
// blocks of other warps while that lowers the largest warp cost.  Warp 0
// starts with a cost of head entries: its first lane issues the tensor-core
// products and is held about as long as they run, which the kernel measured at
// about the time of 8 (hi + lo transforms, 48 MMA instructions per sample) or 4
// (plain, 16) gathered entries per lane.  pair_of[t*4 + j] receives pair index
// y*32 + r.  smem: keys [2048], perm [2048], bcost [64], bslot [64].
__device__ void deal_pairs(int layout, const int* ptr, int N, int tid, int head, int* keys, int* perm,
                           int* bcost, int* bslot, int* pair_of) {
  for (int q = tid; q < 2048; q += 512) {
    const int y = q >> 5, r = q & 31;
    keys[q] = field_count(layout, ptr, N, y, 2 * r) * 8192 + field_count(layout, ptr, N, y, 2 * r + 1);
  }
  __syncthreads();
  for (int q = tid; q < 2048; q += 512) {
    const int L = keys[q];
    int rank = 0;
    for (int j = 0; j < 2048; ++j) rank += (keys[j] > L) || (keys[j] == L && j < q);
    perm[rank] = q;
  }
  __syncthreads();
  constexpr int nw = 16, nb = 64;  // warps, blocks
  if (tid < nb) {
    int m0 = 0, m1 = 0;
    for (int l = 0; l < 32; ++l) {
      const int k = keys[perm[32 * tid + l]];
      m0 = max(m0, k / 8192);
      m1 = max(m1, k % 8192);
    }
    bcost[tid] = m0 + m1;
    bslot[tid] = -1;
  }
  __syncthreads();
  if (tid == 0) {
    int wcost[16], wfill[16];
    for (int w = 0; w < 16; ++w) wcost[w] = wfill[w] = 0;
    wcost[0] = head;
    for (int it = 0; it < nb; ++it) {  // largest block first, to the cheapest warp with room
      int b = -1;
      for (int k = 0; k < nb; ++k)
        if (bslot[k] < 0 && (b < 0 || bcost[k] > bcost[b])) b = k;
      int w = -1;
      for (int x = 0; x < nw; ++x)
        if (wfill[x] < 4 && (w < 0 || wcost[x] < wcost[w])) w = x;
      bslot[b] = 4 * w + wfill[w]++;
      wcost[w] += bcost[b];
    }
    for (int round = 0; round < 256; ++round) {  // swaps that lower the costliest warp
      int wm = 0;
      for (int x = 1; x < nw; ++x)
        if (wcost[x] > wcost[wm]) wm = x;
      int best = wcost[wm], bi = -1, bk = -1;
      for (int i = 0; i < nb; ++i) {
        if (bslot[i] / 4 != wm) continue;
        for (int k = 0; k < nb; ++k) {
          const int w = bslot[k] / 4;
          if (w == wm || bcost[k] >= bcost[i]) continue;
          const int nm = max(wcost[wm] - bcost[i] + bcost[k], wcost[w] - bcost[k] + bcost[i]);
          if (nm < best) {
            best = nm;
            bi = i;
            bk = k;
          }
        }
      }
      if (bi < 0) break;
      const int wk = bslot[bk] / 4, d = bcost[bi] - bcost[bk];
      wcost[wm] -= d;
      wcost[wk] += d;
      const int t = bslot[bi];
      bslot[bi] = bslot[bk];
      bslot[bk] = t;
    }
  }
  __syncthreads();
  for (int b = 0; b < nb; ++b) {  // block b to the lanes of warp bslot / 4, pair slot bslot % 4
    const int w = bslot[b] / 4, j = bslot[b] % 4;
    if (tid >> 5 == w) pair_of[tid * 4 + j] = perm[32 * b + (tid & 31)];
  }
  __syncthreads();
}

// One CTA of nt threads per channel.  fill = 0: only the padded entry count of
// the channel (tot[c]); fill = 1: also every table.
__global__ void gather_tables_kernel(int layout, int head, int N, int nnz, int fill, const int* __restrict__ csr_ptr,
                                     const int2* __restrict__ csr_ent, const int* __restrict__ chan_off,
                                     int* __restrict__ tot, int* __restrict__ cnt_out, int* __restrict__ base_out,
                                     uint16_t* __restrict__ task_out, uint16_t* __restrict__ ent_a,
                                     float* __restrict__ ent_w) {
  extern __shared__ int sh[];
  const int nt = blockDim.x, warps = nt / 32;
  const int ns = layout == kLayoutFft128 ? 16 : 8;  // slots per thread
  int* kws = sh;                 // [warps * ns]
  int* bws = kws + warps * ns;   // [warps * ns]
  const bool pairs = layout == kLayoutPair64 || layout == kLayoutPairQ || layout == kLayoutPairD;
  int* keys = bws + warps * ns;  // [2048] (pairs only)
  int* perm = keys + 2048;       // [2048] (pairs only)
  int* pair_of = perm + 2048;    // [4 nt] (pairs only)
  int* bcost = pair_of + 4 * nt; // [64] (pairs only)
  int* bslot = bcost + 64;       // [64] (pairs only)
  // table set (channel, or virtual channel 4 c + q) and the grid channel it reads
  const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int cg = layout_folded(layout) ? c >> 2 : c;
  const int alpha = c & 1, beta = (c >> 1) & 1;  // folded layouts only
  const int* ptr = csr_ptr + (size_t)cg * (N * N + 1);

  int task = tid;
  int2 cells[16];
  if (pairs) {
    deal_pairs(layout, ptr, N, tid, head, keys, perm, bcost, bslot, pair_of);
    for (int s = 0; s < 8; ++s) {
      const int q = pair_of[tid * 4 + (s >> 1)];
      cells[s] = make_int2(q >> 5, 2 * (q & 31) + (s & 1));
    }
  } else {
    for (int s = 0; s < ns; ++s) cells[s] = cell_of(layout, task, s);
  }
  int cnt[16], beg[16];
  for (int s = 0; s < ns; ++s) {
    const int2 yx = cells[s];
    const int cell = layout_folded(layout) ? -1 : field_cell(layout, N, yx.x, yx.y);
    beg[s] = cell < 0 ? 0 : ptr[cell];
    cnt[s] = field_count(layout, ptr, N, yx.x, yx.y);
    // FFT layouts: trip count rounded up to even (that kernel walks entries in pairs)
    const int kmax = __reduce_max_sync(0xffffffffu, cnt[s]);
    const int k = (layout == kLayoutFft64 || layout == kLayoutFft32 || layout == kLayoutFft128 ||
                   layout == kLayoutFft64Q)
                      ? ((kmax + 1) & ~1)
                      : kmax;
    if (lane == 0) kws[w * ns + s] = k;
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int q = 0; q < warps * ns; ++q) {
      bws[q] = run;
      run += 32 * kws[q];
    }
    if (!fill) tot[c] = run;
  }
  __syncthreads();
  if (!fill) return;
  const size_t off = (size_t)chan_off[c];
  for (int q = tid; q < warps * ns; q += nt) {
    cnt_out[(size_t)c * warps * ns + q] = kws[q];
    base_out[(size_t)c * warps * ns + q] = bws[q];
  }
  if (pairs) {
    for (int j = 0; j < 4; ++j) task_out[((size_t)c * nt + tid) * 4 + j] = (uint16_t)pair_of[tid * 4 + j];
  } else {
    task_out[(size_t)c * nt + tid] = (uint16_t)task;
  }
  const int2* ent = csr_ent + (size_t)cg * nnz;
  for (int s = 0; s < ns; ++s) {
    const int K = kws[w * ns + s];
    if (layout_folded(layout)) {
      // the four source cells' entries in (u, s) order, weights signed, then padding
      int k = 0;
      for (int us = 0; us < 4; ++us) {
        const int u = us >> 1, sx = us & 1;
        const int cell = (cells[s].x + 64 * u) * N + cells[s].y + 64 * sx;
        const int b0 = ptr[cell], n = ptr[cell + 1] - b0;
        const bool neg = ((alpha * sx + beta * u) & 1) != 0;
        for (int i = 0; i < n; ++i, ++k) {
          const size_t idx = off + entry_pos(layout, (size_t)bws[w * ns + s], k, lane);
          const int2 e = ent[b0 + i];
          ent_a[idx] = (uint16_t)e.x;
          ent_w[idx] = neg ? -__int_as_float(e.y) : __int_as_float(e.y);
        }
      }
      for (; k < K; ++k) {
        const size_t idx = off + entry_pos(layout, (size_t)bws[w * ns + s], k, lane);
        ent_a[idx] = 0;
        ent_w[idx] = 0.f;
      }
      continue;
    }
    for (int k = 0; k < K; ++k) {
      const size_t idx = off + entry_pos(layout, (size_t)bws[w * ns + s], k, lane);
      if (k < cnt[s]) {
        const int2 e = ent[beg[s] + k];
        ent_a[idx] = (uint16_t)e.x;
        ent_w[idx] = __int_as_float(e.y);
      } else {
        ent_a[idx] = 0;
        ent_w[idx] = 0.f;
      }
    }
  }
}

}  // namespace

cudaError_t build_gather_tables(Plan& p, int layout, int threads, size_t* total_bytes) {
  GatherTables& g = p.gt;
  g.layout = layout;
  g.threads = threads;
  const int warps = threads / 32;
  const int ns = layout == kLayoutFft128 ? 16 : 8;
  const int nnz = p.A * p.S * p.S;
  const bool pairs = layout == kLayoutPair64 || layout == kLayoutPairQ || layout == kLayoutPairD;
  const int nsets = layout_folded(layout) ? 4 * p.C : p.C;  // table sets (virtual channels)
  // warp 0's head start in the tensor path's deal (its lane 0 issues the products)
  const bool x3 = p.xform == EPIC_XFORM_DFT_BF16X3 || p.xform == EPIC_XFORM_DFT_FP16X3;
  const int head = pairs ? (x3 ? 8 : 4) : 0;
  const size_t smem = sizeof(int) * (2 * (size_t)warps * ns +
                                     (pairs ? 2 * 2048 + 4 * (size_t)threads + 128 : 0));
  int* d_tot = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_tot), sizeof(int) * nsets);
  if (e != cudaSuccess) return e;
  gather_tables_kernel<<<nsets, threads, smem>>>(layout, head, p.N, nnz, 0, p.d_csr_ptr, p.d_csr_ent, nullptr, d_tot,
                                               nullptr, nullptr, nullptr, nullptr, nullptr);
  e = cudaGetLastError();
  std::vector<int> tot(nsets);
  if (e == cudaSuccess) e = cudaMemcpy(tot.data(), d_tot, sizeof(int) * nsets, cudaMemcpyDeviceToHost);
  cudaFree(d_tot);
  if (e != cudaSuccess) return e;
  std::vector<int> off(nsets + 1, 0);
  g.max_chan_entries = 0;
  for (int c = 0; c < nsets; ++c) {
    off[c + 1] = off[c] + tot[c];
    if (tot[c] > g.max_chan_entries) g.max_chan_entries = tot[c];
  }
  const size_t total = (size_t)off[nsets];
  size_t bytes = 0;
  auto grab = [&](void** ptr, size_t b) {
    cudaError_t err = cudaMalloc(ptr, b > 0 ? b : 16);
    if (err == cudaSuccess) bytes += b;
    return err;
  };
  if ((e = grab(reinterpret_cast<void**>(&g.d_chan_off), sizeof(int) * (nsets + 1))) != cudaSuccess) return e;
  if ((e = grab(reinterpret_cast<void**>(&g.d_cnt), sizeof(int) * (size_t)nsets * warps * ns)) != cudaSuccess) return e;
  if ((e = grab(reinterpret_cast<void**>(&g.d_base), sizeof(int) * (size_t)nsets * warps * ns)) != cudaSuccess) return e;
  const size_t per_thread = pairs ? 4 : 1;
  if ((e = grab(reinterpret_cast<void**>(&g.d_task), sizeof(uint16_t) * (size_t)nsets * threads * per_thread)) !=
      cudaSuccess)
    return e;
  if ((e = grab(reinterpret_cast<void**>(&g.d_ent_a), sizeof(uint16_t) * total)) != cudaSuccess) return e;
  if ((e = grab(reinterpret_cast<void**>(&g.d_ent_w), sizeof(float) * total)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(g.d_chan_off, off.data(), sizeof(int) * (nsets + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  gather_tables_kernel<<<nsets, threads, smem>>>(layout, head, p.N, nnz, 1, p.d_csr_ptr, p.d_csr_ent, g.d_chan_off,
                                               nullptr, g.d_cnt, g.d_base, g.d_task, g.d_ent_a, g.d_ent_w);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  *total_bytes = bytes;
  return e;
}

void free_gather_tables(GatherTables& g) {
  void* ptrs[] = {g.d_cnt, g.d_base, g.d_chan_off, g.d_ent_a, g.d_ent_w, g.d_task};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  g = GatherTables();
}

}  // namespace epic
