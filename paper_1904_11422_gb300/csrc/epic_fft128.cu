// epic_fft128.cu -- the FP32 imaging path on 128 x 128 grids: one fused kernel
// that unpacks, calibrates, grids, transforms and squares (Eq. (5), Sec. 3.2),
// run by clusters of two CTAs on neighbouring SMs.
//
// A 128 x 128 grid of two polarisations is 256 KB in FP32, more than one CTA's
// shared memory, and a whole channel's image accumulators (XX, YY, Re XY, Im XY)
// are another 256 KB.  The pair splits both:
//   * CTA r grids and row-transforms the rows y in [64 r, 64 r + 64) of both
//     polarisations, in its own shared memory (128 KB);
//   * the row outputs in the other CTA's columns go to a small exchange buffer
//     in global memory (L2) instead of the own row buffer; after a cluster
//     barrier (release / acquire at cluster scope), CTA r column-transforms the
//     columns k in [64 r, 64 r + 64), reading its own rows from shared memory
//     and the other CTA's rows from the exchange buffer;
//   * the squared and cross-multiplied outputs of its columns are accumulated
//     in tensor memory (TMEM, 128 KB per CTA: 512 threads x 64 FP32 values),
//     which stays resident for the cluster's whole span of samples.
// The exchange buffer is double-buffered by sample parity: a CTA writes sample
// u + 2 only after the barrier of sample u + 1, which the other CTA reaches after
// reading sample u.  Fine-grained distributed shared memory was measured to move
// only about 11 bytes per clock per SM for this pattern (loads or stores), a
// quarter of the kernel's time; through L2 the same 64 KB per sample and CTA
// costs far less.  Both CTAs of a cluster walk the same units, so they reach
// every barrier the same number of times.
//
// Line transforms: 128 = 16 x 8 (Cooley-Tukey).  A line is held by 8 threads,
// thread n1 holding elements n1 + 8 n2 (n2 = 0..15); it takes the 16-point DFT
// over n2, multiplies by exp(+2 pi i n1 k2 / 128), exchanges through 128 words
// of shared memory, and finishes with two 8-point DFTs, after which thread q
// holds outputs (2q + h) + 16 k1 (h = 0, 1; k1 = 0..7).  The XOR layouts below
// were checked (on the host, for every access pattern of the kernel) to need one
// shared-memory wavefront per half-warp.
#include "epic_internal.cuh"
#include "epic_ptx.cuh"

namespace epic {

namespace {

using namespace ptx;

constexpr int kN = 128, kRows = 64, kThreads = 512, kWarps = 16, kSlots = 16;
constexpr int kMaxAnt = 1024;
constexpr int kMaxK = kMaxAnt / kThreads;
constexpr uint32_t kTmemCols = 256;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }

// 4- and 8-point DFTs with the exp(+2 pi i nk/n) kernel, natural order in and out.
__device__ __forceinline__ void dft4(float2& y0, float2& y1, float2& y2, float2& y3) {
  const float2 s02 = cadd(y0, y2), d02 = csub(y0, y2);
  const float2 s13 = cadd(y1, y3), d13 = mul_i(csub(y1, y3));
  y0 = cadd(s02, s13);
  y2 = csub(s02, s13);
  y1 = cadd(d02, d13);
  y3 = csub(d02, d13);
}
__device__ __forceinline__ void dft8(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4, float2& x5,
                                     float2& x6, float2& x7) {
  const float h = 0.70710678118654752f;  // 1/sqrt(2)
  float2 a0 = cadd(x0, x4), a1 = cadd(x1, x5), a2 = cadd(x2, x6), a3 = cadd(x3, x7);
  float2 b0 = csub(x0, x4);
  const float2 t1 = csub(x1, x5);
  float2 b1 = make_float2(h * (t1.x - t1.y), h * (t1.x + t1.y));   // * exp(+i pi/4)
  float2 b2 = mul_i(csub(x2, x6));                                 // * exp(+i pi/2)
  const float2 t3 = csub(x3, x7);
  float2 b3 = make_float2(-h * (t3.x + t3.y), h * (t3.x - t3.y));  // * exp(+3i pi/4)
  dft4(a0, a1, a2, a3);
  dft4(b0, b1, b2, b3);
  x0 = a0; x2 = a1; x4 = a2; x6 = a3;
  x1 = b0; x3 = b1; x5 = b2; x7 = b3;
}

// 16-point DFT: 8-point DFTs of the even and odd elements, then one radix-2
// step with exp(+2 pi i k / 16).
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = x[2 * i];
    o[i] = x[2 * i + 1];
  }
  dft8(e[0], e[1], e[2], e[3], e[4], e[5], e[6], e[7]);
  dft8(o[0], o[1], o[2], o[3], o[4], o[5], o[6], o[7]);
  float2 t[8];
  t[0] = o[0];
  t[1] = cmul(o[1], make_float2(c1, s1));
  t[2] = make_float2(h * (o[2].x - o[2].y), h * (o[2].x + o[2].y));
  t[3] = cmul(o[3], make_float2(s1, c1));
  t[4] = mul_i(o[4]);
  t[5] = cmul(o[5], make_float2(-s1, c1));
  t[6] = make_float2(-h * (o[6].x + o[6].y), h * (o[6].x - o[6].y));
  t[7] = cmul(o[7], make_float2(-c1, s1));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = cadd(e[k], t[k]);
    x[k + 8] = csub(e[k], t[k]);
  }
}

// Exchange slot of value k2 of thread n1 in the 128-word scratch line `line`.
__device__ __forceinline__ int xpos(int line, int k2, int n1) { return ((k2 << 3) | (n1 ^ (k2 >> 1))) ^ ((line & 1) << 3); }
// Stored column of output k in local row yl of the row buffer.
__device__ __forceinline__ int cpos(int yl, int k) { return k ^ (2 * (yl & 7) + (yl & 1)); }
// Output index held as value s by thread q after a line transform.
__host__ __device__ constexpr int kidx(int q, int s) { return 2 * q + (s >> 3) + 16 * (s & 7); }

// One 128-point line transform (see the file comment); `line_buf` is the
// 128-word exchange line of this group of 8 threads.
__device__ __forceinline__ void fft_line128(float2 (&v)[16], const float2* __restrict__ tw, float2* line_buf,
                                            int line, int n1) {
  dft16(v);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw[(n1 * k2) & (kN - 1)]);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) line_buf[xpos(line, k2, n1)] = v[k2];
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int m = 0; m < 8; ++m) v[8 * h + m] = line_buf[xpos(line, 2 * n1 + h, m)];
  __syncwarp();
  dft8(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
  dft8(v[8], v[9], v[10], v[11], v[12], v[13], v[14], v[15]);
}

struct F128Smem {
  size_t R, tw, wst, coef, E, autos, ent_a, ent_w, taddr, total;
};

template <int P>
__host__ __device__ inline F128Smem f128_layout(int A, int max_entries, int ent_in_smem) {
  F128Smem L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) & ~(size_t)15;
    return at;
  };
  L.R = take(sizeof(float2) * P * kRows * kN);
  L.tw = take(sizeof(float2) * kN);
  L.wst = take(sizeof(int) * 2 * kWarps * kSlots);
  L.coef = take(sizeof(float2) * A * P);
  L.E = take((P == 2 ? 16 : 8) * (size_t)A);
  L.autos = take(sizeof(int4) * A);
  L.ent_a = take(ent_in_smem ? sizeof(uint16_t) * (size_t)max_entries : 0);
  L.ent_w = take(ent_in_smem ? sizeof(float) * (size_t)max_entries : 0);
  L.taddr = take(16);
  L.total = o;
  return L;
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
    fft128_image_kernel(const uint8_t* __restrict__ volts, int T, int C, int A, long long W, long long units,
                        int spans, const float2* __restrict__ coef, const int* __restrict__ g_cnt,
                        const int* __restrict__ g_base, const int* __restrict__ g_off,
                        const uint16_t* __restrict__ g_ent_a, const float* __restrict__ g_ent_w, int max_entries,
                        int ent_in_smem, const float2* __restrict__ twiddle, float* __restrict__ part,
                        int* __restrict__ part_auto, float2* __restrict__ xbuf) {
  constexpr int NN = kN * kN, HALF = kN / 2;
  constexpr int NPL = (P == 2) ? 4 : 1;

  extern __shared__ __align__(16) unsigned char smem[];
  const F128Smem L = f128_layout<P>(A, max_entries, ent_in_smem);
  float2* Rbuf = reinterpret_cast<float2*>(smem + L.R);   // [P][64 local rows][128]
  float2* tw_s = reinterpret_cast<float2*>(smem + L.tw);
  int* cnt_s = reinterpret_cast<int*>(smem + L.wst);      // [warps][16] trip counts
  int* base_s = cnt_s + kWarps * kSlots;                  // [warps][16] first entries
  float2* coef_s = reinterpret_cast<float2*>(smem + L.coef);
  float4* E4 = reinterpret_cast<float4*>(smem + L.E);
  float2* E2 = reinterpret_cast<float2*>(smem + L.E);
  int4* auto_s = reinterpret_cast<int4*>(smem + L.autos);
  uint16_t* enta_s = reinterpret_cast<uint16_t*>(smem + L.ent_a);
  float* entw_s = reinterpret_cast<float*>(smem + L.ent_w);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + L.taddr);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int line = tid >> 3, n1 = tid & 7;  // row pass: local row; column pass: local column
  const uint32_t rank = cluster_ctarank();
  const long long cluster = blockIdx.x >> 1;

  const long long u0 = cluster * W;
  const long long u1 = min(u0 + W, units);
  if (u0 >= u1) return;  // the same for both CTAs of the cluster
  const int c_first = (int)(u0 / T);

  for (int m = tid; m < kN; m += kThreads) tw_s[m] = twiddle[m];
  if (warp == 0) {
    tmem_alloc(smem_u32(taddr_s), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // lane quarter of this warp, and its 64 accumulator columns (4 planes x 16)
  const uint32_t tacc = *taddr_s + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)(warp >> 2);
  // exchange buffers of this cluster: [parity][writer rank][P][64 columns][8 j][8 m1]
  // holding the writer's row y = 64 rank + m1 + 8 j in the reader's column 64 (1 - rank) + k
  constexpr size_t kXSlab = (size_t)P * kRows * kRows;  // float2 per (parity, writer)
  float2* xb = xbuf + (size_t)cluster * 4 * kXSlab;

  // unit u = (channel cu, sample tu), stepped without 64-bit divisions
  unsigned raw[kMaxK] = {}, raw_next[kMaxK] = {};
  int cu = c_first, tu = (int)(u0 - (long long)c_first * T);
  auto load_raw = [&](int c, int t, unsigned (&dst)[kMaxK]) {
    const uint8_t* base = volts + ((size_t)t * C + c) * (size_t)A * P;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      const int a = tid + k * kThreads;
      if (a < A) {
        if constexpr (P == 2)
          dst[k] = __ldg(reinterpret_cast<const unsigned short*>(base) + a);
        else
          dst[k] = __ldg(base + a);
      }
    }
  };
  load_raw(cu, tu, raw);

  auto zero_acc = [&]() {
    uint32_t z[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) z[s] = 0u;
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) tmem_st16(tacc + 16u * pl, z);
    tmem_wait_st();
  };

  const int kglob = (int)rank * kRows + line;  // column of the column pass
  auto flush = [&](int c) {
    const int slot = c - c_first;
    float* dst = part + (size_t)(cluster * spans + slot) * 4 * NN;
    const int col = (kglob + HALF) & (kN - 1);  // pixel N/2 is the zero frequency (reading R4)
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) {
      float a[16];
      tmem_ld16(tacc + 16u * pl, a);
      tmem_wait_ld();
#pragma unroll
      for (int s = 0; s < 16; ++s) dst[(size_t)pl * NN + ((kidx(n1, s) + HALF) & (kN - 1)) * kN + col] = a[s];
    }
    if (rank == 0) {
      int4* pa = reinterpret_cast<int4*>(part_auto) + (size_t)(cluster * spans + slot) * A;
      for (int a = tid; a < A; a += kThreads) pa[a] = auto_s[a];
    }
  };

  // 1. unpack, calibrate, exact integer self powers (kept by CTA 0)
  auto unpack = [&](const unsigned (&rw)[kMaxK]) {
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      const int a = tid + k * kThreads;
      if (a < A) {
        const int xr = nib_hi(rw[k] & 0xffu), xi = nib_lo(rw[k] & 0xffu);
        const float2 kx = coef_s[a * P];
        const float2 ex = make_float2(kx.x * xr - kx.y * xi, kx.x * xi + kx.y * xr);
        int4 au = auto_s[a];
        au.x += xr * xr + xi * xi;
        if constexpr (P == 2) {
          const int yr = nib_hi(rw[k] >> 8), yi = nib_lo(rw[k] >> 8);
          const float2 ky = coef_s[a * P + 1];
          const float2 ey = make_float2(ky.x * yr - ky.y * yi, ky.x * yi + ky.y * yr);
          E4[a] = make_float4(ex.x, ex.y, ey.x, ey.y);
          au.y += yr * yr + yi * yi;
          au.z += xr * yr + xi * yi;
          au.w += xi * yr - xr * yi;
        } else {
          E2[a] = ex;
        }
        if (rank == 0) auto_s[a] = au;
      }
    }
  };

  int cur_c = -1, eoff = 0;
  bool have_next = false;
  const uint16_t* ent_a = g_ent_a;
  const float* ent_w = g_ent_w;

  for (long long u = u0; u < u1; ++u) {
    const int c = cu;
    int cn = cu, tn = tu + 1;  // the next unit
    if (tn == T) {
      tn = 0;
      ++cn;
    }
    if (c != cur_c) {
      if (cur_c >= 0) flush(cur_c);
      zero_acc();
      cur_c = c;
      const int* cnt_g = g_cnt + (size_t)c * 2 * kWarps * kSlots + rank * kWarps * kSlots;
      const int* base_g = g_base + (size_t)c * 2 * kWarps * kSlots + rank * kWarps * kSlots;
      if (tid < kWarps * kSlots) {
        cnt_s[tid] = cnt_g[tid];
        base_s[tid] = base_g[tid];
      }
      for (int k = tid; k < A * P; k += kThreads) coef_s[k] = coef[(size_t)c * A * P + k];
      for (int a = tid; a < A; a += kThreads) auto_s[a] = make_int4(0, 0, 0, 0);
      const int e0 = g_off[c], ne = g_off[c + 1] - e0;
      // this CTA's rows use the entries [lo, hi) of the channel (the second half
      // starts at the first slot of virtual warp 16)
      const int mid = g_base[(size_t)c * 2 * kWarps * kSlots + kWarps * kSlots];
      const int lo = rank ? mid : 0, hi = rank ? ne : mid;
      if (ent_in_smem) {
        for (int k = lo + tid; k < hi; k += kThreads) {
          enta_s[k - lo] = g_ent_a[e0 + k];
          entw_s[k - lo] = g_ent_w[e0 + k];
        }
        ent_a = enta_s;
        ent_w = entw_s;
        eoff = lo;
      } else {
        ent_a = g_ent_a + e0;
        ent_w = g_ent_w + e0;
        eoff = 0;
      }
      __syncthreads();
    }
    if (u + 1 < u1) load_raw(cn, tn, raw_next);

    // E holds this sample's fields already when they were unpacked while the
    // previous sample waited at its cluster barrier
    if (!have_next) {
      unpack(raw);
      __syncthreads();
    }
    have_next = false;

    // 2. grid (gather, fixed order) and 3a. row transforms; thread (local row
    //    `line`, n1) owns cells (64 rank + line, n1 + 8 n2).  A warp whose four
    //    rows hold no entries (outside the aperture of a padded grid) skips its
    //    transforms: the transform of a zero line is zero.
    int any = 0;
#pragma unroll
    for (int q = 0; q < kSlots; ++q) any |= cnt_s[warp * kSlots + q];
    {
      float2 v[P][16];
#pragma unroll
      for (int n2 = 0; n2 < 16; ++n2) {
        const int K = cnt_s[warp * kSlots + n2];
        const int b = base_s[warp * kSlots + n2] - eoff + lane;
        float2 gx = make_float2(0.f, 0.f), gy = make_float2(0.f, 0.f);
        for (int k = 0; k < K; k += 2) {  // K is even: two entries per step, added in order
          const int a0 = ent_a[b + 32 * k], a1 = ent_a[b + 32 * k + 32];
          const float w0 = ent_w[b + 32 * k], w1 = ent_w[b + 32 * k + 32];
          if constexpr (P == 2) {
            const float4 e0 = E4[a0], e1 = E4[a1];
            gx.x = fmaf(w1, e1.x, fmaf(w0, e0.x, gx.x));
            gx.y = fmaf(w1, e1.y, fmaf(w0, e0.y, gx.y));
            gy.x = fmaf(w1, e1.z, fmaf(w0, e0.z, gy.x));
            gy.y = fmaf(w1, e1.w, fmaf(w0, e0.w, gy.y));
          } else {
            const float2 e0 = E2[a0], e1 = E2[a1];
            gx.x = fmaf(w1, e1.x, fmaf(w0, e0.x, gx.x));
            gx.y = fmaf(w1, e1.y, fmaf(w0, e0.y, gx.y));
          }
        }
        v[0][n2] = gx;
        if constexpr (P == 2) v[1][n2] = gy;
      }
      // this sample's exchange slab written by this CTA
      float2* xw = xb + (size_t)(((u - u0) & 1) * 2 + rank) * kXSlab;
      const int m1w = line & 7, jw = line >> 3;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        float2* row = Rbuf + (size_t)(p * kRows + line) * kN;
        if (any) fft_line128(v[p], tw_s, row, line, n1);
#pragma unroll
        for (int s = 0; s < 16; ++s) {
          const int k = kidx(n1, s);
          if ((k >> 6) == (int)rank)
            row[cpos(line, k)] = v[p][s];
          else
            __stcg(xw + (((size_t)p * kRows + (k & 63)) * 8 + jw) * 8 + m1w, v[p][s]);
        }
      }
    }
    // rows of both CTAs complete, in shared memory and in the exchange buffer;
    // while the release of the exchange writes completes, unpack the next
    // sample of the same channel (every thread has finished reading E)
    __syncthreads();
    cluster_arrive();
    if (u + 1 < u1 && cn == c) {
      unpack(raw_next);
      have_next = true;
    }
    cluster_wait();

    // 3b. column transforms and 4. products; thread (column 64 rank + line, m1 = n1)
    {
      float2 v[P][16];
      // row n1 + 8 m2 is local row n1 + 8 (m2 & 7) of CTA m2 / 8
      const float2* xr = xb + (size_t)(((u - u0) & 1) * 2 + (rank ^ 1u)) * kXSlab;
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int m2 = 0; m2 < 16; ++m2) {
          const int j = m2 & 7, yl = n1 + 8 * j;
          if ((m2 >> 3) == (int)rank)
            v[p][m2] = Rbuf[(p * kRows + yl) * kN + cpos(yl, kglob)];
          else
            v[p][m2] = __ldcg(xr + (((size_t)p * kRows + line) * 8 + j) * 8 + n1);
        }
      // every thread of this CTA has read its rows; the row buffers become scratch
      __syncthreads();
#pragma unroll
      for (int p = 0; p < P; ++p) fft_line128(v[p], tw_s, Rbuf + (size_t)(p * kRows + line) * kN, line, n1);

      float a[16], b[16];
      if constexpr (P == 2) {
        tmem_ld16(tacc, a);
        tmem_ld16(tacc + 16u, b);
        tmem_wait_ld();
#pragma unroll
        for (int s = 0; s < 16; ++s) {
          const float2 X = v[0][s], Y = v[1][s];
          a[s] = fmaf(X.x, X.x, fmaf(X.y, X.y, a[s]));
          b[s] = fmaf(Y.x, Y.x, fmaf(Y.y, Y.y, b[s]));
        }
        tmem_st16(tacc, a);
        tmem_st16(tacc + 16u, b);
        tmem_ld16(tacc + 32u, a);
        tmem_ld16(tacc + 48u, b);
        tmem_wait_ld();
#pragma unroll
        for (int s = 0; s < 16; ++s) {
          const float2 X = v[0][s], Y = v[1][s];
          a[s] = fmaf(X.x, Y.x, fmaf(X.y, Y.y, a[s]));   // Re X conj(Y)
          b[s] = fmaf(X.y, Y.x, fmaf(-X.x, Y.y, b[s]));  // Im X conj(Y)
        }
        tmem_st16(tacc + 32u, a);
        tmem_st16(tacc + 48u, b);
      } else {
        tmem_ld16(tacc, a);
        tmem_wait_ld();
#pragma unroll
        for (int s = 0; s < 16; ++s) {
          const float2 X = v[0][s];
          a[s] = fmaf(X.x, X.x, fmaf(X.y, X.y, a[s]));
        }
        tmem_st16(tacc, a);
      }
      tmem_wait_st();
    }
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) raw[k] = raw_next[k];
    cu = cn;
    tu = tn;
    // the next unit's unpack and row pass reuse E and the row buffers
    __syncthreads();
  }
  flush(cur_c);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(*taddr_s, kTmemCols);
}

template <int P>
size_t smem_for(const Plan& p, int ent_in_smem) {
  return f128_layout<P>(p.A, p.gt.max_chan_entries, ent_in_smem).total;
}

template <int P>
cudaError_t config(Plan& p, int* clusters) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  p.ent_in_smem = smem_for<P>(p, 1) <= (size_t)optin ? 1 : 0;
  p.smem = smem_for<P>(p, p.ent_in_smem);
  p.threads = kThreads;
  if (p.smem > (size_t)optin) return cudaErrorInvalidConfiguration;
  e = allow_max_smem(fft128_image_kernel<P>);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * p.sm_count, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, fft128_image_kernel<P>, &cfg);
}

template <int P>
cudaError_t launch(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part, int* part_auto,
                   float2* xbuf, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * ws.ctas, 1, 1);  // ws.ctas counts clusters
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fft128_image_kernel<P>, d_volts, T, p.C, p.A, (long long)ws.W, ws.units,
                            ws.spans, (const float2*)p.d_coef, (const int*)p.gt.d_cnt, (const int*)p.gt.d_base,
                            (const int*)p.gt.d_chan_off, (const uint16_t*)p.gt.d_ent_a, (const float*)p.gt.d_ent_w,
                            p.gt.max_chan_entries, p.ent_in_smem, (const float2*)p.d_twiddle, part, part_auto,
                            xbuf);
}

}  // namespace

size_t fft128_smem_need(int A, int P) {
  return P == 2 ? f128_layout<2>(A, 0, 0).total : f128_layout<1>(A, 0, 0).total;
}
int fft128_max_ant() { return kMaxAnt; }

cudaError_t fft128_config(Plan& p, int* clusters) {
  return p.P == 2 ? config<2>(p, clusters) : config<1>(p, clusters);
}

size_t fft128_xbuf_elems(int clusters, int P) { return (size_t)clusters * 4 * P * kRows * kRows; }

cudaError_t launch_fft128_image_ws(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                                   int* part_auto, cudaStream_t s) {
  return p.P == 2 ? launch<2>(p, d_volts, T, ws, part, part_auto, p.d_xbuf, s)
                  : launch<1>(p, d_volts, T, ws, part, part_auto, p.d_xbuf, s);
}

}  // namespace epic
