// epic_check.cu -- epic_debug_check_plan: the plan's gridding tables checked on
// the host against invariants derived independently of the code that built them.
//
// The imaging kernels index the field array E and the grid by the antenna and
// cell numbers these tables hold, and walk each (warp, slot) for a trip count
// the tables give, so every index the kernels dereference is checked here
// against the plan's sizes.  Beyond bounds, each lane's entry list is re-derived
// from the per-cell table (Eq. (5): the cell sums w * e over the antennas whose
// kernel box covers it, in antenna order) with plain loops, and must match the
// built list entry for entry, with weight-0 padding of antenna 0 after it.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "epic_internal.cuh"

namespace {

struct Entry {
  int a;
  uint32_t wbits;
};

}  // namespace

extern "C" epic_status epic_debug_check_plan(const epic_plan* h, char* report, size_t report_len) {
  if (!h) return EPIC_ERR_INVALID_ARG;
  const epic::Plan& p = h->p;
  const epic::GatherTables& g = p.gt;
  auto say = [&](const char* fmt, ...) {
    if (report && report_len) {
      va_list ap;
      va_start(ap, fmt);
      vsnprintf(report, report_len, fmt, ap);
      va_end(ap);
    }
  };
  const int A = p.A, C = p.C, N = p.N, S = p.S, NN = N * N, nnz = A * S * S;
  const int layout = g.layout, threads = g.threads, warps = threads / 32;
  const bool folded = epic::layout_folded(layout);
  const bool pairs = layout == epic::kLayoutPair64 || layout == epic::kLayoutPairQ || layout == epic::kLayoutPairD;
  const bool even = !pairs;  // the FFT kernels walk entries two at a time
  const int ns = layout == epic::kLayoutFft128 ? 16 : 8;
  const int nsets = folded ? 4 * C : C;
  const int field = (layout == epic::kLayoutPairD || folded) ? 64 : N;  // side of the gathered field

  std::vector<int> ptr((size_t)C * (NN + 1)), off(nsets + 1), cnt((size_t)nsets * warps * ns),
      base((size_t)nsets * warps * ns);
  std::vector<int2> csr((size_t)C * nnz);
  cudaError_t e = cudaMemcpy(ptr.data(), p.d_csr_ptr, sizeof(int) * ptr.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(csr.data(), p.d_csr_ent, sizeof(int2) * csr.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(off.data(), g.d_chan_off, sizeof(int) * off.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), g.d_cnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(base.data(), g.d_base, sizeof(int) * base.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    say("copying the tables failed: %s", cudaGetErrorString(e));
    return EPIC_ERR_CUDA;
  }
  const size_t total = off[nsets] >= 0 ? (size_t)off[nsets] : 0;
  std::vector<uint16_t> ea(total), task((size_t)nsets * threads * (pairs ? 4 : 1));
  std::vector<float> ew(total);
  if (total) e = cudaMemcpy(ea.data(), g.d_ent_a, sizeof(uint16_t) * total, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && total) e = cudaMemcpy(ew.data(), g.d_ent_w, sizeof(float) * total, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(task.data(), g.d_task, sizeof(uint16_t) * task.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    say("copying the tables failed: %s", cudaGetErrorString(e));
    return EPIC_ERR_CUDA;
  }

  // 1. per-cell table: row pointers, antennas in range and increasing within a
  //    cell, weights positive and finite, every antenna's S x S box present
  for (int c = 0; c < C; ++c) {
    const int* pc = &ptr[(size_t)c * (NN + 1)];
    if (pc[0] != 0 || pc[NN] != nnz) return say("channel %d: cell table holds %d entries, not %d", c, pc[NN], nnz), EPIC_ERR_INTERNAL;
    std::vector<int> per_ant(A, 0);
    for (int cell = 0; cell < NN; ++cell) {
      if (pc[cell + 1] < pc[cell]) return say("channel %d: row pointers decrease at cell %d", c, cell), EPIC_ERR_INTERNAL;
      for (int k = pc[cell]; k < pc[cell + 1]; ++k) {
        const int2 en = csr[(size_t)c * nnz + k];
        float w;
        std::memcpy(&w, &en.y, sizeof w);
        if (en.x < 0 || en.x >= A) return say("channel %d cell %d: antenna %d out of range", c, cell, en.x), EPIC_ERR_INTERNAL;
        if (k > pc[cell] && csr[(size_t)c * nnz + k - 1].x >= en.x)
          return say("channel %d cell %d: antennas not in increasing order", c, cell), EPIC_ERR_INTERNAL;
        if (!(w > 0.f) || !std::isfinite(w)) return say("channel %d cell %d: weight %g", c, cell, (double)w), EPIC_ERR_INTERNAL;
        ++per_ant[en.x];
      }
    }
    for (int a = 0; a < A; ++a)
      if (per_ant[a] != S * S) return say("channel %d: antenna %d covers %d cells, not %d", c, a, per_ant[a], S * S), EPIC_ERR_INTERNAL;
  }

  // 2. table sets: offsets, and the (warp, slot) ranges tile each set in order
  int largest = 0;
  for (int q = 0; q < nsets; ++q) {
    const int tot = off[q + 1] - off[q];
    if (off[q] < 0 || tot < 0) return say("set %d: bad offsets", q), EPIC_ERR_INTERNAL;
    largest = tot > largest ? tot : largest;
    int run = 0;
    for (int ws = 0; ws < warps * ns; ++ws) {
      const int K = cnt[(size_t)q * warps * ns + ws], B = base[(size_t)q * warps * ns + ws];
      if (K < 0 || B != run || (even && (K & 1)))
        return say("set %d (warp, slot) %d: trip count %d, first entry %d, expected %d", q, ws, K, B, run), EPIC_ERR_INTERNAL;
      run += 32 * K;
    }
    if (run != tot) return say("set %d: slots cover %d of %d entries", q, run, tot), EPIC_ERR_INTERNAL;
  }
  if (largest != g.max_chan_entries)
    return say("largest set holds %d entries, the plan sized for %d", largest, g.max_chan_entries), EPIC_ERR_INTERNAL;

  // 3. each thread's cells: the FFT row layouts by position, the pair layouts a
  //    permutation of the field's 2048 cell pairs per set
  for (int q = 0; q < nsets && pairs; ++q) {
    std::vector<char> seen(2048, 0);
    for (int i = 0; i < 4 * threads; ++i) {
      const int pr = task[(size_t)q * threads * 4 + i];
      if (pr >= 2048 || seen[pr]) return say("set %d: cell pair %d dealt twice or out of range", q, pr), EPIC_ERR_INTERNAL;
      seen[pr] = 1;
    }
  }

  // 4. every lane's entries, re-derived from the per-cell table
  std::vector<Entry> want;
  long long real = 0, padded = 0;
  for (int q = 0; q < nsets; ++q) {
    const int c = folded ? q >> 2 : q, alpha = q & 1, beta = (q >> 1) & 1;
    const int* pc = &ptr[(size_t)c * (NN + 1)];
    const int2* ec = &csr[(size_t)c * nnz];
    for (int t = 0; t < threads; ++t) {
      const int w = t >> 5, lane = t & 31;
      for (int s = 0; s < ns; ++s) {
        int y, x;
        if (pairs) {
          const int pr = task[((size_t)q * threads + t) * 4 + (s >> 1)];
          y = pr >> 5;
          x = 2 * (pr & 31) + (s & 1);
        } else if (layout == epic::kLayoutFft32) {
          y = t >> 2;
          x = (t & 3) + 4 * s;
        } else {
          y = t >> 3;
          x = (t & 7) + 8 * s;
        }
        if (y >= field || x >= field) return say("set %d thread %d slot %d: cell (%d, %d) outside the field", q, t, s, y, x), EPIC_ERR_INTERNAL;
        want.clear();
        auto add_cell = [&](int cy, int cx, bool neg) {
          const int cell = cy * N + cx;
          for (int k = pc[cell]; k < pc[cell + 1]; ++k)
            want.push_back({ec[k].x, (uint32_t)ec[k].y ^ (neg ? 0x80000000u : 0u)});
        };
        if (folded) {
          for (int us = 0; us < 4; ++us) {
            const int u = us >> 1, sx = us & 1;
            add_cell(y + 64 * u, x + 64 * sx, ((alpha * sx + beta * u) & 1) != 0);
          }
        } else if (y < N && x < N) {
          add_cell(y, x, false);
        }
        const size_t slot = (size_t)q * warps * ns + w * ns + s;
        const int K = cnt[slot];
        if ((int)want.size() > K) return say("set %d thread %d slot %d: %d entries, trip count %d", q, t, s, (int)want.size(), K), EPIC_ERR_INTERNAL;
        for (int k = 0; k < K; ++k) {
          const size_t idx = (size_t)off[q] + epic::entry_pos(layout, (size_t)base[slot], k, lane);
          uint32_t wb;
          std::memcpy(&wb, &ew[idx], sizeof wb);
          if (ea[idx] >= A) return say("set %d entry %zu: antenna %d out of range", q, idx, (int)ea[idx]), EPIC_ERR_INTERNAL;
          if (k < (int)want.size()) {
            if (ea[idx] != want[k].a || wb != want[k].wbits)
              return say("set %d thread %d slot %d entry %d: (%d, %08x), expected (%d, %08x)", q, t, s, k, (int)ea[idx], wb,
                         want[k].a, want[k].wbits), EPIC_ERR_INTERNAL;
            ++real;
          } else {
            if (ea[idx] != 0 || wb != 0u)
              return say("set %d thread %d slot %d entry %d: padding is not (0, +0)", q, t, s, k), EPIC_ERR_INTERNAL;
            ++padded;
          }
        }
      }
    }
  }
  const long long expect_real = (long long)nsets * nnz;
  if (real != expect_real) return say("%lld real entries in the tables, expected %lld", real, expect_real), EPIC_ERR_INTERNAL;
  say("ok: %d channels, %d table sets, %lld entries (%lld padding), every index in range", C, nsets, real + padded, padded);
  return EPIC_OK;
}
