// epic_fft.cu -- the FP32 imaging path: one fused kernel per block that unpacks,
// calibrates, grids, transforms and squares, accumulating images on chip.
//
// Per work unit (time sample t of channel c), following Eq. (5) and Sec. 3.2:
//   1. unpack the A x P bytes of (t, c) (4+4-bit complex, Sec. 3.2), multiply by
//      the calibration coefficient k (delay compensation and gain, Fig. 2) and
//      accumulate each antenna's self power (Fig. 2 "Accumulate
//      Autocorrelations") exactly, on the integer samples;
//   2. grid: every cell gathers w * e from the antennas whose kernel box covers
//      it (the convolution W * E' of Eq. (5)), atomics-free and in a fixed order;
//   3. transform: 2-D FFT with the exp(+2 pi i ...) kernel of Eq. (5) ("inverse
//      FT", Sec. 3.2), as radix-8 passes: rows in registers with a warp-local
//      exchange, one CTA-wide transpose through shared memory, columns likewise;
//   4. square and cross-multiply (XX, YY, XY; Sec. 2.1, Fig. 2 "Square and
//      Accumulate") into per-thread register accumulators that stay resident
//      for the CTA's whole span of samples.
// The grid of one (t, c) never leaves the SM.  A CTA owns a contiguous range of
// (c, t) units (channel-major) and writes one partial image per channel it
// touches; a separate kernel sums partials in CTA order and removes the
// autocorrelation term.
#include <algorithm>

#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int kMaxAnt = 2048;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }

// 4-point DFT with the exp(+2 pi i nk/4) kernel; natural order in and out.
__device__ __forceinline__ void dft4(float2& y0, float2& y1, float2& y2, float2& y3) {
  const float2 s02 = cadd(y0, y2), d02 = csub(y0, y2);
  const float2 s13 = cadd(y1, y3), d13 = mul_i(csub(y1, y3));
  y0 = cadd(s02, s13);
  y2 = csub(s02, s13);
  y1 = cadd(d02, d13);
  y3 = csub(d02, d13);
}

// 8-point DFT with the exp(+2 pi i nk/8) kernel: one radix-2 split into even
// and odd outputs, then two 4-point DFTs.  Natural order in and out.
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  const float h = 0.70710678118654752f;  // 1/sqrt(2)
  float2 a0 = cadd(x[0], x[4]), a1 = cadd(x[1], x[5]), a2 = cadd(x[2], x[6]), a3 = cadd(x[3], x[7]);
  float2 b0 = csub(x[0], x[4]);
  const float2 t1 = csub(x[1], x[5]);
  float2 b1 = make_float2(h * (t1.x - t1.y), h * (t1.x + t1.y));   // * exp(+i pi/4)
  float2 b2 = mul_i(csub(x[2], x[6]));                             // * exp(+i pi/2)
  const float2 t3 = csub(x[3], x[7]);
  float2 b3 = make_float2(-h * (t3.x + t3.y), h * (t3.x - t3.y));  // * exp(+3i pi/4)
  dft4(a0, a1, a2, a3);
  dft4(b0, b1, b2, b3);
  x[0] = a0; x[2] = a1; x[4] = a2; x[6] = a3;
  x[1] = b0; x[3] = b1; x[5] = b2; x[7] = b3;
}

// Thread geometry of an N-point line transform: R1 threads per line, 8 points
// per thread (element n1 + R1*n2 held by thread n1 as its n2-th value).
// swz is an XOR layout of the row buffer, scr a padded layout of the warp
// scratch (slot (k2, n1) of line r, written by thread n1 and read by thread k2);
// both were checked offline to be free of shared-memory bank conflicts for every
// access pattern below.  scr is additive so that each thread's eight stores and
// eight loads are one base address plus compile-time offsets.
template <int N> struct Geo;
template <> struct Geo<64> {
  static constexpr int R1 = 8, THREADS = 512, RPW = 4, SCR = 4 * 72;
  __device__ static int swz(int y) { return (9 * (y & 7)) & 15; }
  __device__ static int scr(int r, int k2, int n1) { return r * 72 + 9 * k2 + n1; }
  // output index held as value s by thread q after a line transform
  __host__ __device__ static constexpr int kidx(int q, int s) { return q + 8 * s; }
  // (kidx(n1, s) ^ sw) for the row buffer, written as two per-thread bases and
  // a compile-time offset: n1 < 8 and sw < 16 leave the bits of 16 (s >> 1) alone
  __device__ static int rowpos(int n1, int s, int sw) {
    const int t = n1 ^ sw;
    return ((s & 1) ? (t ^ 8) : t) + 16 * (s >> 1);
  }
};
template <> struct Geo<32> {
  static constexpr int R1 = 4, THREADS = 128, RPW = 8, SCR = 8 * 36;
  __device__ static int swz(int y) { return (5 * (y & 7)) & 15; }
  __device__ static int scr(int r, int k2, int n1) { return r * 36 + 4 * k2 + n1 + (k2 >> 1); }
  __host__ __device__ static constexpr int kidx(int q, int s) { return 2 * q + (s >> 2) + 8 * (s & 3); }
  __device__ static int rowpos(int n1, int s, int sw) { return kidx(n1, s) ^ sw; }
};

// One N-point transform of a line held by R1 threads (Cooley-Tukey N = R1 x 8):
// 8-point DFT over n2, twiddle exp(+2 pi i n1 k2 / N), exchange through warp
// scratch, then the R1-point DFT over n1.  On return thread q holds output
// Geo<N>::kidx(q, s) as v[s].
template <int N>
__device__ __forceinline__ void fft_line(float2 (&v)[8], const float2 (&tw)[8], float2* __restrict__ scr, int r,
                                         int n1) {
  using G = Geo<N>;
  dft8(v);
#pragma unroll
  for (int k2 = 1; k2 < 8; ++k2) v[k2] = cmul(v[k2], tw[k2]);
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) scr[G::scr(r, k2, n1)] = v[k2];
  __syncwarp();
  if constexpr (N == 64) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = scr[G::scr(r, n1, m)];
    dft8(v);
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int m = 0; m < 4; ++m) v[4 * h + m] = scr[G::scr(r, 2 * n1 + h, m)];
    dft4(v[0], v[1], v[2], v[3]);
    dft4(v[4], v[5], v[6], v[7]);
  }
  __syncwarp();
}

// Shared-memory layout of the imaging kernel, in bytes from the base.
struct FftSmem {
  size_t R, scr, wst, coef, E, E2, autos, ent_a, ent_w, total;
};

// The 64 x 64 two-polarisation kernel with one antenna per thread can unpack
// each next sample early, on the four warps whose gather is lightest (chosen at
// plan time from the gather tables), into a second field buffer (see
// fft_image_kernel and choose_unpack_warps).
template <int N, int P, bool Q, int KA>
constexpr bool kEarlyUnpack = N == 64 && P == 2 && !Q && KA == 1;

template <int N, int P>
__host__ __device__ inline FftSmem fft_smem_layout(int A, int max_entries, int ent_in_smem, bool two_e = false) {
  using G = Geo<N>;
  FftSmem L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) & ~(size_t)15;
    return at;
  };
  L.R = take(sizeof(float2) * P * N * N);
  L.scr = take(sizeof(float2) * (G::THREADS / 32) * G::SCR);
  L.wst = take(sizeof(int) * 2 * (G::THREADS / 32) * 8);
  L.coef = take(sizeof(float2) * A * P);
  L.E = take((P == 2 ? 16 : 8) * (size_t)(A + 1));
  L.E2 = two_e ? take((P == 2 ? 16 : 8) * (size_t)(A + 1)) : L.E;
  L.autos = take(sizeof(int4) * A);
  L.ent_a = take(ent_in_smem ? sizeof(uint16_t) * (size_t)max_entries : 0);
  L.ent_w = take(ent_in_smem ? sizeof(float) * (size_t)max_entries : 0);
  L.total = o;
  return L;
}

// Q (N = 64 only): a 128 x 128 grid run as four 64 x 64 problems, virtual
// channel 4 c + q per output-parity subset q = alpha + 2 beta: the gather tables
// fold the four quadrants with signed weights (layout kFft64Q), each gathered
// cell (y, x) is multiplied by exp(+2 pi i (alpha x + beta y) / 128), and the
// reduction interleaves the four 64 x 64 partial images (pixel (j, i) of subset
// q is pixel (2 j + beta, 2 i + alpha)).  `twiddle` then holds the 128-point
// table, `C` the real channel count.
// KA: antennas per thread whose bytes are prefetched (1 when the array fits the
// block, else enough for kMaxAnt), which keeps registers free for small arrays.
// At N = 32 (128-thread blocks) four blocks share an SM: 16 warps hide latency
// that the two blocks of an unbounded register allocation could not.
template <int N, int P, bool Q = false, int KA = (kMaxAnt + Geo<N>::THREADS - 1) / Geo<N>::THREADS>
__global__ void __launch_bounds__(Geo<N>::THREADS, N == 32 ? 4 : 1)
    fft_image_kernel(const uint8_t* __restrict__ volts, int T, int C, int A, long long W, long long units, int spans,
                     const float2* __restrict__ coef, const int* __restrict__ g_cnt, const int* __restrict__ g_base,
                     const int* __restrict__ g_off, const uint16_t* __restrict__ g_ent_a,
                     const float* __restrict__ g_ent_w, int max_entries, int ent_in_smem,
                     const float2* __restrict__ twiddle, float* __restrict__ part, int* __restrict__ part_auto,
                     unsigned unpack_warps) {
  using G = Geo<N>;
  constexpr int NT = G::THREADS, NN = N * N, R1 = G::R1, HALF = N / 2;
  constexpr int MAXK = KA;
  constexpr int NPL = (P == 2) ? 4 : 1;

  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int WARPS = NT / 32;
  const bool early = kEarlyUnpack<N, P, Q, KA> && unpack_warps != 0u;
  const FftSmem L = fft_smem_layout<N, P>(A, max_entries, ent_in_smem, early);
  float2* Rbuf = reinterpret_cast<float2*>(smem + L.R);
  float2* scr = reinterpret_cast<float2*>(smem + L.scr) + (threadIdx.x >> 5) * G::SCR;
  int* cnt_s = reinterpret_cast<int*>(smem + L.wst);    // [warps][8] trip counts
  int* base_s = cnt_s + WARPS * 8;                      // [warps][8] first entries
  float2* coef_s = reinterpret_cast<float2*>(smem + L.coef);
  float4* E4 = reinterpret_cast<float4*>(smem + L.E);
  float2* E2 = reinterpret_cast<float2*>(smem + L.E);
  float4* E4n = reinterpret_cast<float4*>(smem + L.E2);  // the next sample's fields (early unpack)
  int4* auto_s = reinterpret_cast<int4*>(smem + L.autos);
  uint16_t* enta_s = reinterpret_cast<uint16_t*>(smem + L.ent_a);
  float* entw_s = reinterpret_cast<float*>(smem + L.ent_w);

  const int tid = threadIdx.x;
  const int line = tid / R1, n1 = tid % R1, r = line % G::RPW;

  float2 tw[8];
  tw[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int k2 = 1; k2 < 8; ++k2) tw[k2] = twiddle[Q ? ((n1 * k2) & (N - 1)) * 2 : (n1 * k2) & (N - 1)];

  const long long u0 = (long long)blockIdx.x * W;
  const long long u1 = min(u0 + W, units);
  if (u0 >= u1) return;
  const int c_first = (int)(u0 / T);

  float acc[NPL][8];
#pragma unroll
  for (int pl = 0; pl < NPL; ++pl)
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[pl][s] = 0.f;

  // raw bytes of the thread's antennas, prefetched one unit ahead; unit u is
  // (channel cu, sample tu), stepped without 64-bit divisions
  unsigned raw[MAXK] = {}, raw_next[MAXK] = {};
  int cu = c_first, tu = (int)(u0 - (long long)c_first * T);
  auto load_raw = [&](int cv, int t, unsigned (&dst)[MAXK]) {
    const int c = cv >> (Q ? 2 : 0);
    const uint8_t* base = volts + ((size_t)t * C + c) * (size_t)A * P;
#pragma unroll
    for (int k = 0; k < MAXK; ++k) {
      const int a = tid + k * NT;
      if (a < A) {
        if constexpr (P == 2)
          dst[k] = __ldg(reinterpret_cast<const unsigned short*>(base) + a);
        else
          dst[k] = __ldg(base + a);
      }
    }
  };
  load_raw(cu, tu, raw);

  // early unpack: the four warps of unpack_warps, whose rows hold few
  // gather entries, unpack the next sample of the same channel into E4n after
  // their row transforms, while the other warps still gather; its raw bytes (up
  // to four antennas per unpack thread, A <= 512) are requested at the start of
  // the sample
  const int warp_id = tid >> 5;
  const bool uwarp = early && ((unpack_warps >> warp_id) & 1u);
  const int ut = __popc(unpack_warps & ((1u << warp_id) - 1u)) * 32 + (tid & 31);
  constexpr int kUT = 32 * 4;  // unpack threads (four warps)
  unsigned rawu[4] = {0u, 0u, 0u, 0u};
  bool have_e = false;  // E4 already holds this sample's fields

  int cur_c = -1;
  const uint16_t* ent_a = g_ent_a;
  const float* ent_w = g_ent_w;
  const int warp = tid >> 5, lane = tid & 31;

  auto flush = [&](int c) {
    const int slot = c - c_first;
    float* dst = part + (size_t)((long long)blockIdx.x * spans + slot) * 4 * NN;
    // thread (column k = line, q = n1) holds pixel rows kidx(q, s); shift so that
    // pixel N/2 is the zero frequency (reading R4)
    const int col = (line + HALF) & (N - 1);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int row = (G::kidx(n1, s) + HALF) & (N - 1);
#pragma unroll
      for (int pl = 0; pl < NPL; ++pl) dst[(size_t)pl * NN + row * N + col] = acc[pl][s];
    }
    int4* pa = reinterpret_cast<int4*>(part_auto) + (size_t)((long long)blockIdx.x * spans + slot) * A;
    for (int a = tid; a < A; a += NT) pa[a] = auto_s[a];
  };

  for (long long u = u0; u < u1; ++u) {
    const int c = cu;
    int cn = cu, tn = tu + 1;  // the next unit
    if (tn == T) {
      tn = 0;
      ++cn;
    }
    if (c != cur_c) {
      if (cur_c >= 0) {
        flush(cur_c);
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl)
#pragma unroll
          for (int s = 0; s < 8; ++s) acc[pl][s] = 0.f;
      }
      cur_c = c;
      if (tid < WARPS * 8) {
        cnt_s[tid] = g_cnt[(size_t)c * WARPS * 8 + tid];
        base_s[tid] = g_base[(size_t)c * WARPS * 8 + tid];
      }
      for (int k = tid; k < A * P; k += NT) coef_s[k] = coef[(size_t)(c >> (Q ? 2 : 0)) * A * P + k];
      for (int a = tid; a < A; a += NT) auto_s[a] = make_int4(0, 0, 0, 0);
      const int e0 = g_off[c], ne = g_off[c + 1] - e0;
      if (ent_in_smem) {
        for (int k = tid; k < ne; k += NT) {
          enta_s[k] = g_ent_a[e0 + k];
          entw_s[k] = g_ent_w[e0 + k];
        }
        ent_a = enta_s;
        ent_w = entw_s;
      } else {
        ent_a = g_ent_a + e0;
        ent_w = g_ent_w + e0;
      }
      __syncthreads();
    }
    if (u + 1 < u1) load_raw(cn, tn, raw_next);
    const bool early_next = early && u + 1 < u1 && cn == c;  // the next sample is unpacked early
    if (early_next && uwarp) {
      const uint8_t* bn = volts + ((size_t)tn * C + cn) * (size_t)A * P;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int a = ut + kUT * j;
        if (a < A) rawu[j] = __ldg(reinterpret_cast<const unsigned short*>(bn) + a);
      }
    }

    // 1. unpack, calibrate, exact integer self powers (unless unpacked early)
    if (!have_e) {
#pragma unroll
      for (int k = 0; k < MAXK; ++k) {
        const int a = tid + k * NT;
        if (a < A) {
          const int xr = nib_hi(raw[k] & 0xffu), xi = nib_lo(raw[k] & 0xffu);
          const float2 kx = coef_s[a * P];
          const float2 ex = make_float2(kx.x * xr - kx.y * xi, kx.x * xi + kx.y * xr);
          int4 au = auto_s[a];
          au.x += xr * xr + xi * xi;
          if constexpr (P == 2) {
            const int yr = nib_hi(raw[k] >> 8), yi = nib_lo(raw[k] >> 8);
            const float2 ky = coef_s[a * P + 1];
            const float2 ey = make_float2(ky.x * yr - ky.y * yi, ky.x * yi + ky.y * yr);
            E4[a] = make_float4(ex.x, ex.y, ey.x, ey.y);
            au.y += yr * yr + yi * yi;
            au.z += xr * yr + xi * yi;
            au.w += xi * yr - xr * yi;
          } else {
            E2[a] = ex;
          }
          auto_s[a] = au;
        }
      }
      __syncthreads();
    }

    // 2. grid (gather, fixed order) and 3a. row transforms; thread (row y, n1)
    {
      const int y = line;
      float2 v[P][8];
      // the warp's eight trip counts and first entries, read before the first slot
      // (measured faster except for the folded 128 x 128 grids, which read them per slot)
      int Ks[8], bs[8];
      if constexpr (!Q) {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
          Ks[n2] = cnt_s[warp * 8 + n2];
          bs[n2] = base_s[warp * 8 + n2];
        }
      }
#pragma unroll
      for (int n2 = 0; n2 < 8; ++n2) {
        // cell (y, n1 + R1 n2): lane-interleaved entries, warp-uniform trip count
        const int K = Q ? cnt_s[warp * 8 + n2] : Ks[n2];
        const int bse = Q ? base_s[warp * 8 + n2] : bs[n2];
        // a lane's entries 2j, 2j + 1 side by side (entry_pos): one 32-bit load of
        // both antennas, one 8-byte load of both weights
        const uint32_t* ea2 = reinterpret_cast<const uint32_t*>(ent_a) + (bse >> 1) + lane;
        const float2* ew2 = reinterpret_cast<const float2*>(ent_w) + (bse >> 1) + lane;
        float2 gx = make_float2(0.f, 0.f), gy = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int k = 0; k < K; k += 2) {  // K is even: two entries per step, added in order
          const uint32_t aa = ea2[16 * k];
          const float2 ww = ew2[16 * k];
          const int a0 = (int)(aa & 0xffffu), a1 = (int)(aa >> 16);
          const float w0 = ww.x, w1 = ww.y;
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
        if constexpr (Q) {
          // H_q = exp(+2 pi i (alpha x + beta y) / 128) x the folded gather
          const float2 w = __ldg(twiddle + (((cur_c & 1) * (n1 + R1 * n2) + ((cur_c >> 1) & 1) * y) & 127));
          gx = make_float2(gx.x * w.x - gx.y * w.y, gx.x * w.y + gx.y * w.x);
          gy = make_float2(gy.x * w.x - gy.y * w.y, gy.x * w.y + gy.y * w.x);
        }
        v[0][n2] = gx;
        if constexpr (P == 2) v[1][n2] = gy;
      }
      const int sw = G::swz(y);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        fft_line<N>(v[p], tw, scr, r, n1);
        float2* Rrow = Rbuf + (size_t)p * NN + y * N;
#pragma unroll
        for (int s = 0; s < 8; ++s) Rrow[G::rowpos(n1, s, sw)] = v[p][s];
      }
    }
    if (early_next && uwarp) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int a = ut + kUT * j;
        if (a < A) {
          const unsigned rb = rawu[j];
          const int xr = nib_hi(rb & 0xffu), xi = nib_lo(rb & 0xffu);
          const int yr = nib_hi(rb >> 8), yi = nib_lo(rb >> 8);
          const float2 kx = coef_s[a * P], ky = coef_s[a * P + 1];
          E4n[a] = make_float4(kx.x * xr - kx.y * xi, kx.x * xi + kx.y * xr, ky.x * yr - ky.y * yi,
                               ky.x * yi + ky.y * yr);
          int4 au = auto_s[a];
          au.x += xr * xr + xi * xi;
          au.y += yr * yr + yi * yi;
          au.z += xr * yr + xi * yi;
          au.w += xi * yr - xr * yi;
          auto_s[a] = au;
        }
      }
    }
    __syncthreads();

    // 3b. column transforms and 4. products; thread (column k, m1)
    {
      const int k = line;
      float2 v[P][8];
      // both polarisations' columns loaded before the first transform (its warp
      // syncs would otherwise hold the second one's loads back)
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int m2 = 0; m2 < 8; ++m2) {
          const int y = n1 + R1 * m2;
          v[p][m2] = Rbuf[(size_t)p * NN + y * N + (k ^ G::swz(y))];
        }
#pragma unroll
      for (int p = 0; p < P; ++p) fft_line<N>(v[p], tw, scr, r, n1);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float2 X = v[0][s];
        acc[0][s] = fmaf(X.x, X.x, fmaf(X.y, X.y, acc[0][s]));
        if constexpr (P == 2) {
          const float2 Y = v[1][s];
          acc[1][s] = fmaf(Y.x, Y.x, fmaf(Y.y, Y.y, acc[1][s]));
          acc[2][s] = fmaf(X.x, Y.x, fmaf(X.y, Y.y, acc[2][s]));
          acc[3][s] = fmaf(X.y, Y.x, fmaf(-X.x, Y.y, acc[3][s]));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < MAXK; ++k) raw[k] = raw_next[k];
    cu = cn;
    tu = tn;
    if (early_next) {  // the next sample's fields are in E4n (written before the row barrier)
      float4* t = E4;
      E4 = E4n;
      E4n = t;
    }
    have_e = early_next;
  }
  flush(cur_c);
}

template <int N, int P>
cudaError_t occupancy(int threads, size_t smem, int* per_sm) {
  cudaError_t e = allow_max_smem(fft_image_kernel<N, P>);
  if (e == cudaSuccess) e = allow_max_smem(fft_image_kernel<N, P, false, 1>);
  if (e == cudaSuccess && N == 64) e = allow_max_smem(fft_image_kernel<64, P, true>);
  if (e == cudaSuccess && N == 64) e = allow_max_smem(fft_image_kernel<64, P, true, 1>);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fft_image_kernel<N, P>, threads, smem);
}

// One imaging launch with the prefetch sized for the array.
template <int N, int P, bool Q>
cudaError_t launch_image(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, const float2* coef,
                         float* part, int* part_auto, cudaStream_t s) {
  if (p.A <= Geo<N>::THREADS)
    fft_image_kernel<N, P, Q, 1><<<ws.ctas, p.threads, p.smem, s>>>(
        d_volts, T, p.C, p.A, ws.W, ws.units, ws.spans, coef, p.gt.d_cnt, p.gt.d_base, p.gt.d_chan_off,
        p.gt.d_ent_a, p.gt.d_ent_w, p.gt.max_chan_entries, p.ent_in_smem, p.d_twiddle, part, part_auto,
        p.unpack_warps);
  else
    fft_image_kernel<N, P, Q><<<ws.ctas, p.threads, p.smem, s>>>(
        d_volts, T, p.C, p.A, ws.W, ws.units, ws.spans, coef, p.gt.d_cnt, p.gt.d_base, p.gt.d_chan_off,
        p.gt.d_ent_a, p.gt.d_ent_w, p.gt.max_chan_entries, p.ent_in_smem, p.d_twiddle, part, part_auto, 0u);
  return cudaGetLastError();
}

// Every N x N FP32 imaging launch not run on clusters: 32 x 32, 64 x 64, and
// 128 x 128 grids as four folded 64 x 64 problems.
cudaError_t launch_image_any(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, const float2* coef,
                             float* part, int* part_auto, cudaStream_t s) {
  if (p.N == 128)
    return p.P == 2 ? launch_image<64, 2, true>(p, d_volts, T, ws, coef, part, part_auto, s)
                    : launch_image<64, 1, true>(p, d_volts, T, ws, coef, part, part_auto, s);
  if (p.N == 64)
    return p.P == 2 ? launch_image<64, 2, false>(p, d_volts, T, ws, coef, part, part_auto, s)
                    : launch_image<64, 1, false>(p, d_volts, T, ws, coef, part, part_auto, s);
  return p.P == 2 ? launch_image<32, 2, false>(p, d_volts, T, ws, coef, part, part_auto, s)
                  : launch_image<32, 1, false>(p, d_volts, T, ws, coef, part, part_auto, s);
}

size_t smem_for(const Plan& p, int ent_in_smem) {
  const int me = p.gt.max_chan_entries;
  // the second field buffer of the early unpack
  const bool two_e = p.unpack_warps != 0u;
  if (p.N == 64 || p.vq == 4) return p.P == 2 ? fft_smem_layout<64, 2>(p.A, me, ent_in_smem, two_e).total
                                 : fft_smem_layout<64, 1>(p.A, me, ent_in_smem).total;
  return p.P == 2 ? fft_smem_layout<32, 2>(p.A, me, ent_in_smem).total
                  : fft_smem_layout<32, 1>(p.A, me, ent_in_smem).total;
}

bool ent_fits(const Plan& p) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return smem_for(p, 1) <= (size_t)optin;
}

// The gridding step alone, for the debug entry point: the same gather table,
// entry order and FP32 fused multiply-adds as the imaging kernel.
template <int P>
__global__ void debug_grid_kernel(const uint8_t* __restrict__ volts, int T, int C, int A, int N, int t, int c, int pol,
                                  const float2* __restrict__ coef, const int* __restrict__ csr_ptr,
                                  const int2* __restrict__ csr_ent, int nnz, float* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* E = reinterpret_cast<float2*>(smem);
  const uint8_t* base = volts + ((size_t)t * C + c) * (size_t)A * P;
  for (int a = threadIdx.x; a < A; a += blockDim.x) {
    const unsigned b = base[a * P + pol];
    const int re = nib_hi(b), im = nib_lo(b);
    const float2 k = coef[((size_t)c * A + a) * P + pol];
    E[a] = make_float2(k.x * re - k.y * im, k.x * im + k.y * re);
  }
  __syncthreads();
  const int* ptr = csr_ptr + (size_t)c * (N * N + 1);
  const int2* ent = csr_ent + (size_t)c * nnz;
  for (int cell = threadIdx.x; cell < N * N; cell += blockDim.x) {
    float2 g = make_float2(0.f, 0.f);
    for (int e = ptr[cell]; e < ptr[cell + 1]; ++e) {
      const int2 en = ent[e];
      const float w = __int_as_float(en.y);
      const float2 ev = E[en.x];
      g.x = fmaf(w, ev.x, g.x);
      g.y = fmaf(w, ev.y, g.y);
    }
    grid[2 * cell] = g.x;
    grid[2 * cell + 1] = g.y;
  }
}

// The transform step alone, for the debug entry point: the gridded field of one
// (t, c, pol) (the CSR order and FP32 fused multiply-adds of the gather), then
// the imaging kernel's own row pass and column pass (the same line transforms,
// twiddles and shared-memory layouts), written out with the pixel shift of
// reading R4: out[row m][column l][re, im].  One CTA of the imaging block size.
template <int N>
__global__ void __launch_bounds__(Geo<N>::THREADS)
    debug_transform_kernel(const uint8_t* __restrict__ volts, int T, int C, int A, int P, int t, int c, int pol,
                           const float2* __restrict__ coef, const int* __restrict__ csr_ptr,
                           const int2* __restrict__ csr_ent, int nnz, const float2* __restrict__ twiddle,
                           float* __restrict__ out) {
  using G = Geo<N>;
  constexpr int NT = G::THREADS, NN = N * N, R1 = G::R1, HALF = N / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* Rbuf = reinterpret_cast<float2*>(smem);  // [N][N], rows XOR-swizzled as in the imaging kernel
  float2* scr_all = Rbuf + NN;                     // [warps][SCR]
  float2* E = scr_all + (NT / 32) * G::SCR;        // [A] calibrated fields of polarisation pol
  const int tid = threadIdx.x, line = tid / R1, n1 = tid % R1, r = line % G::RPW;
  float2* scr = scr_all + (tid >> 5) * G::SCR;

  const uint8_t* base = volts + ((size_t)t * C + c) * (size_t)A * P;
  for (int a = tid; a < A; a += NT) {
    const unsigned b = base[a * P + pol];
    const int re = nib_hi(b), im = nib_lo(b);
    const float2 k = coef[((size_t)c * A + a) * P + pol];
    E[a] = make_float2(k.x * re - k.y * im, k.x * im + k.y * re);
  }
  __syncthreads();
  const int* ptr = csr_ptr + (size_t)c * (NN + 1);
  const int2* ent = csr_ent + (size_t)c * nnz;
  for (int cell = tid; cell < NN; cell += NT) {
    float2 g = make_float2(0.f, 0.f);
    for (int e = ptr[cell]; e < ptr[cell + 1]; ++e) {
      const int2 en = ent[e];
      const float w = __int_as_float(en.y);
      g.x = fmaf(w, E[en.x].x, g.x);
      g.y = fmaf(w, E[en.x].y, g.y);
    }
    const int y = cell / N, x = cell % N;
    Rbuf[y * N + (x ^ G::swz(y))] = g;
  }
  __syncthreads();

  float2 tw[8];
  tw[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int k2 = 1; k2 < 8; ++k2) tw[k2] = twiddle[(n1 * k2) & (N - 1)];
  {  // row pass: thread (row y, n1) holds cells (y, n1 + R1 n2)
    const int y = line, sw = G::swz(y);
    float2 v[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) v[n2] = Rbuf[y * N + ((n1 + R1 * n2) ^ sw)];
    fft_line<N>(v, tw, scr, r, n1);
#pragma unroll
    for (int s = 0; s < 8; ++s) Rbuf[y * N + G::rowpos(n1, s, sw)] = v[s];
  }
  __syncthreads();
  {  // column pass: thread (column k, n1) ends with rows kidx(n1, s) of column k
    const int k = line;
    float2 v[8];
#pragma unroll
    for (int m2 = 0; m2 < 8; ++m2) {
      const int y = n1 + R1 * m2;
      v[m2] = Rbuf[y * N + (k ^ G::swz(y))];
    }
    fft_line<N>(v, tw, scr, r, n1);
    const int col = (k + HALF) & (N - 1);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int row = (G::kidx(n1, s) + HALF) & (N - 1);
      out[2 * (row * N + col)] = v[s].x;
      out[2 * (row * N + col) + 1] = v[s].y;
    }
  }
}

}  // namespace

cudaError_t launch_debug_transform(Plan& p, const uint8_t* d_volts, int T, int t, int c, int pol, float* d_y,
                                   cudaStream_t s) {
  const int nnz = p.A * p.S * p.S;
  auto run = [&](auto kernel, int threads, int n) -> cudaError_t {
    const size_t scr = (size_t)(threads / 32) * (n == 64 ? Geo<64>::SCR : Geo<32>::SCR);
    const size_t smem = sizeof(float2) * ((size_t)n * n + scr + p.A);
    cudaError_t e = allow_max_smem(kernel);
    if (e != cudaSuccess) return e;
    kernel<<<1, threads, smem, s>>>(d_volts, T, p.C, p.A, p.P, t, c, pol, p.d_coef, p.d_csr_ptr, p.d_csr_ent, nnz,
                                    p.d_twiddle, d_y);
    return cudaGetLastError();
  };
  return p.N == 64 ? run(debug_transform_kernel<64>, Geo<64>::THREADS, 64)
                   : run(debug_transform_kernel<32>, Geo<32>::THREADS, 32);
}

// The early unpack's four warps (fft_image_kernel): per warp, the largest over
// channels of its padded gather steps (sum over its slots of the trip count);
// the four cheapest warps unpack each next sample if even the costliest of them
// gathers at most half as much as the costliest warp -- rows outside the
// aperture leave that much slack -- else none does (0).  Only for the kernel
// variant that has the early unpack (64 x 64, two polarisations, not folded,
// A <= 512).
unsigned choose_unpack_warps(const Plan& p) {
  if (!(p.N == 64 && p.vq != 4 && p.P == 2 && p.A <= Geo<64>::THREADS)) return 0u;
  constexpr int kW = Geo<64>::THREADS / 32;
  std::vector<int> cnt((size_t)p.C * kW * 8);
  if (cudaMemcpy(cnt.data(), p.gt.d_cnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return 0u;
  long long cost[kW] = {};
  for (int c = 0; c < p.C; ++c)
    for (int w = 0; w < kW; ++w) {
      long long k = 0;
      for (int s = 0; s < 8; ++s) k += cnt[((size_t)c * kW + w) * 8 + s];
      cost[w] = std::max(cost[w], k);
    }
  int order[kW];
  for (int w = 0; w < kW; ++w) order[w] = w;
  std::stable_sort(order, order + kW, [&](int a, int b) { return cost[a] < cost[b]; });
  const long long worst = cost[order[kW - 1]];
  if (2 * cost[order[3]] > worst) return 0u;
  unsigned mask = 0u;
  for (int i = 0; i < 4; ++i) mask |= 1u << order[i];
  return mask;
}

cudaError_t fft_image_config(Plan& p, int* ctas_per_sm) {
  p.unpack_warps = choose_unpack_warps(p);
  if (p.unpack_warps != 0u) {
    // the second field buffer must not push the gather tables out of shared memory
    const unsigned keep = p.unpack_warps;
    p.unpack_warps = 0u;
    const bool fits_without = ent_fits(p);
    p.unpack_warps = keep;
    if (fits_without && !ent_fits(p)) p.unpack_warps = 0u;
  }
  p.ent_in_smem = ent_fits(p) ? 1 : 0;
  p.smem = smem_for(p, p.ent_in_smem);
  const bool n64 = p.N == 64 || p.vq == 4;  // 128 x 128 grids folded into 64 x 64 problems
  p.threads = n64 ? Geo<64>::THREADS : Geo<32>::THREADS;
  if (n64) return p.P == 2 ? occupancy<64, 2>(p.threads, p.smem, ctas_per_sm)
                                 : occupancy<64, 1>(p.threads, p.smem, ctas_per_sm);
  return p.P == 2 ? occupancy<32, 2>(p.threads, p.smem, ctas_per_sm)
                  : occupancy<32, 1>(p.threads, p.smem, ctas_per_sm);
}

cudaError_t launch_fft_image(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, cudaStream_t s) {
  if (p.N == 128 && p.vq == 1) return launch_fft128_image_ws(p, d_volts, T, ws, p.d_part, p.d_part_auto, s);
  return launch_image_any(p, d_volts, T, ws, p.d_coef, p.d_part, p.d_part_auto, s);
}

cudaError_t launch_fft_image_ws(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                                int* part_auto, cudaStream_t s) {
  if (p.N == 128 && p.vq == 1) return launch_fft128_image_ws(p, d_volts, T, ws, part, part_auto, s);
  return launch_image_any(p, d_volts, T, ws, p.d_coef, part, part_auto, s);
}

cudaError_t launch_debug_grid(Plan& p, const uint8_t* d_volts, int T, int t, int c, int pol, float* d_grid,
                              cudaStream_t s) {
  const int nnz = p.A * p.S * p.S;
  const size_t smem = sizeof(float2) * p.A;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(p.P == 2 ? debug_grid_kernel<2> : debug_grid_kernel<1>);
    if (e != cudaSuccess) return e;
  }
  if (p.P == 2)
    debug_grid_kernel<2><<<1, 256, smem, s>>>(d_volts, T, p.C, p.A, p.N, t, c, pol, p.d_coef, p.d_csr_ptr,
                                              p.d_csr_ent, nnz, d_grid);
  else
    debug_grid_kernel<1><<<1, 256, smem, s>>>(d_volts, T, p.C, p.A, p.N, t, c, pol, p.d_coef, p.d_csr_ptr,
                                              p.d_csr_ent, nnz, d_grid);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Adjoint pass of the gain gradient (epic_grad), N = 64.
//
// For L = sum_pix (I_pp - M_pp)^2 with R = 2 (I - M), the gradient with respect
// to conj(g_ap) has a data term
//   sum_t conj(e~_ap(t)) D_ap(t),  D_ap(t) = sum_cells w_a(cell) H_p,t(cell),
//   H_p,t = F^H (R_pp . Y_p,t)   (the transform of Eq. (5) with the opposite sign)
// where e~ is the delay-compensated field without the gain and Y the image of
// sample t.  The gridded fields are recomputed per sample, not stored: each
// unit repeats the forward gather + FFT of fft_image_kernel, multiplies by R,
// runs the conjugate FFT (conj, the same +i line transforms, conj) through the
// same register layouts in reverse (columns, then rows), and degrids H over each
// antenna's kernel box.  Per-antenna sums stay in registers (thread a owns
// antenna a) and are written per channel span, like the partial images.
//
// N = 32 and N = 64 grids run directly; a 128 x 128 grid folded into four
// 64 x 64 problems (Q: virtual channel 4 c + q, output-parity subset q =
// alpha + 2 beta) runs the adjoint of the fold as well: the forward field is
// H_q = Tw . Fold_q(G) with Tw = exp(+2 pi i (alpha x + beta y) / 128) and
// Fold_q(G)[y][x] = sum_{u,s} (-1)^(alpha s + beta u) G[y + 64 u][x + 64 s], so
// the back-projected field at grid cell (y + 64 u, x + 64 s) is
// (-1)^(alpha s + beta u) conj(Tw[y][x]) H'_q[y][x], which the degrid reads; the
// residual of subset q is that of the output pixels (2 j + beta, 2 i + alpha).
// ---------------------------------------------------------------------------
namespace {

struct AdjSmem {
  size_t R, scr, wst, coef, dph, E, resid, box, wts, ent_a, ent_w, total;
};

template <int N, int P>
__host__ __device__ inline AdjSmem adj_smem_layout(int A, int S, int max_entries, int ent_in_smem) {
  using G = Geo<N>;
  AdjSmem L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) & ~(size_t)15;
    return at;
  };
  L.R = take(sizeof(float2) * P * N * N);
  L.scr = take(sizeof(float2) * (G::THREADS / 32) * G::SCR);
  L.wst = take(sizeof(int) * 2 * (G::THREADS / 32) * 8);
  L.coef = take(sizeof(float2) * A * P);
  L.dph = take(sizeof(float2) * A * P);
  L.E = take((P == 2 ? 16 : 8) * (size_t)(A + 1));
  L.resid = take(sizeof(float) * P * N * N);
  L.box = take(sizeof(int2) * A);
  L.wts = take(sizeof(float) * 2 * (size_t)A * S);
  L.ent_a = take(ent_in_smem ? sizeof(uint16_t) * (size_t)max_entries : 0);
  L.ent_w = take(ent_in_smem ? sizeof(float) * (size_t)max_entries : 0);
  L.total = o;
  return L;
}

template <int N, int P, bool Q>
__global__ void __launch_bounds__(Geo<N>::THREADS, 1)
    adjoint_kernel(const uint8_t* __restrict__ volts, int T, int C, int A, int S, long long W, long long units,
                   int spans, const float2* __restrict__ coef, const double2* __restrict__ dphase,
                   const int* __restrict__ g_cnt, const int* __restrict__ g_base, const int* __restrict__ g_off,
                   const uint16_t* __restrict__ g_ent_a, const float* __restrict__ g_ent_w, int max_entries,
                   int ent_in_smem, const float2* __restrict__ twiddle, const float* __restrict__ resid,
                   const int* __restrict__ box, const double* __restrict__ wx, const double* __restrict__ wy,
                   float2* __restrict__ gpart) {
  using G = Geo<N>;
  constexpr int NT = G::THREADS, NN = N * N, R1 = G::R1, HALF = N / 2, WARPS = NT / 32;
  constexpr int NG = Q ? 2 * N : N;  // side of the plan's grid (and residual)
  extern __shared__ __align__(16) unsigned char smem[];
  const AdjSmem L = adj_smem_layout<N, P>(A, S, max_entries, ent_in_smem);
  float2* Rbuf = reinterpret_cast<float2*>(smem + L.R);
  float2* scr = reinterpret_cast<float2*>(smem + L.scr) + (threadIdx.x >> 5) * G::SCR;
  int* cnt_s = reinterpret_cast<int*>(smem + L.wst);
  int* base_s = cnt_s + WARPS * 8;
  float2* coef_s = reinterpret_cast<float2*>(smem + L.coef);
  float2* dph_s = reinterpret_cast<float2*>(smem + L.dph);
  float4* E4 = reinterpret_cast<float4*>(smem + L.E);
  float2* E2 = reinterpret_cast<float2*>(smem + L.E);
  float* res_s = reinterpret_cast<float*>(smem + L.resid);
  int2* box_s = reinterpret_cast<int2*>(smem + L.box);
  float* wx_s = reinterpret_cast<float*>(smem + L.wts);
  float* wy_s = wx_s + (size_t)A * S;
  uint16_t* enta_s = reinterpret_cast<uint16_t*>(smem + L.ent_a);
  float* entw_s = reinterpret_cast<float*>(smem + L.ent_w);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int line = tid / R1, n1 = tid % R1, r = line % G::RPW;
  float2 tw[8];
  tw[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int k2 = 1; k2 < 8; ++k2) tw[k2] = twiddle[Q ? ((n1 * k2) & (N - 1)) * 2 : (n1 * k2) & (N - 1)];

  const long long u0 = (long long)blockIdx.x * W;
  const long long u1 = min(u0 + W, units);
  if (u0 >= u1) return;
  const int c_first = (int)(u0 / T);

  float2 gacc[P];  // thread a (< A): sum_t conj(e~) D of its antenna
#pragma unroll
  for (int p = 0; p < P; ++p) gacc[p] = make_float2(0.f, 0.f);
  const uint16_t* ent_a = g_ent_a;
  const float* ent_w = g_ent_w;
  int cur_c = -1;

  auto flush = [&](int c) {
    if (tid < A) {
      float2* dst = gpart + ((size_t)((long long)blockIdx.x * spans + (c - c_first)) * A + tid) * P;
#pragma unroll
      for (int p = 0; p < P; ++p) dst[p] = gacc[p];
    }
  };

  int cu = c_first, tu = (int)(u0 - (long long)c_first * T);  // unit u = (channel cu, sample tu)
  // the raw bytes of antenna tid, prefetched one unit ahead
  auto load_raw1 = [&](int cv, int ts) -> unsigned {
    if (tid >= A) return 0u;
    const uint8_t* base = volts + ((size_t)ts * C + (Q ? cv >> 2 : cv)) * (size_t)A * P;
    if constexpr (P == 2)
      return __ldg(reinterpret_cast<const unsigned short*>(base) + tid);
    else
      return __ldg(base + tid);
  };
  unsigned raw_pref = load_raw1(cu, tu);
  for (long long u = u0; u < u1; ++u) {
    const int c = cu;
    if (++tu == T) {
      tu = 0;
      ++cu;
    }
    const unsigned raw = raw_pref;
    if (u + 1 < u1) raw_pref = load_raw1(cu, tu);
    const int cr = Q ? c >> 2 : c;  // the plan's channel (c is a virtual channel when folded)
    if (c != cur_c) {
      if (cur_c >= 0) {
        flush(cur_c);
#pragma unroll
        for (int p = 0; p < P; ++p) gacc[p] = make_float2(0.f, 0.f);
      }
      cur_c = c;
      __syncthreads();  // the previous unit's degrid has finished with the tables
      if (tid < WARPS * 8) {
        cnt_s[tid] = g_cnt[(size_t)c * WARPS * 8 + tid];
        base_s[tid] = g_base[(size_t)c * WARPS * 8 + tid];
      }
      for (int k = tid; k < A * P; k += NT) {
        coef_s[k] = coef[(size_t)cr * A * P + k];
        const double2 d = dphase[(size_t)cr * A * P + k];
        dph_s[k] = make_float2((float)d.x, (float)d.y);
      }
      // the residual of the pixels this (virtual) channel images
      for (int k = tid; k < P * NN; k += NT) {
        const int p = k / NN, j = (k % NN) / N, i = k % N;
        const int al = Q ? (c & 1) : 0, be = Q ? ((c >> 1) & 1) : 0;
        res_s[k] = Q ? resid[((size_t)cr * 2 + p) * NG * NG + (size_t)(2 * j + be) * NG + 2 * i + al]
                     : resid[(size_t)c * 2 * NN + k];
      }
      for (int a = tid; a < A; a += NT) {
        box_s[a] = make_int2(box[((size_t)cr * A + a) * 2], box[((size_t)cr * A + a) * 2 + 1]);
        for (int k = 0; k < S; ++k) {
          wx_s[a * S + k] = (float)wx[((size_t)cr * A + a) * S + k];
          wy_s[a * S + k] = (float)wy[((size_t)cr * A + a) * S + k];
        }
      }
      const int e0 = g_off[c], ne = g_off[c + 1] - e0;
      if (ent_in_smem) {
        for (int k = tid; k < ne; k += NT) {
          enta_s[k] = g_ent_a[e0 + k];
          entw_s[k] = g_ent_w[e0 + k];
        }
        ent_a = enta_s;
        ent_w = entw_s;
      } else {
        ent_a = g_ent_a + e0;
        ent_w = g_ent_w + e0;
      }
      __syncthreads();
    }

    // 1. unpack and calibrate with the call's coefficients (thread a = tid)
    if (tid < A) {
      const int xr = nib_hi(raw & 0xffu), xi = nib_lo(raw & 0xffu);
      const float2 kx = coef_s[tid * P];
      const float2 ex = make_float2(kx.x * xr - kx.y * xi, kx.x * xi + kx.y * xr);
      if constexpr (P == 2) {
        const int yr = nib_hi(raw >> 8), yi = nib_lo(raw >> 8);
        const float2 ky = coef_s[tid * P + 1];
        E4[tid] = make_float4(ex.x, ex.y, ky.x * yr - ky.y * yi, ky.x * yi + ky.y * yr);
      } else {
        E2[tid] = ex;
      }
    }
    __syncthreads();

    // 2. forward: gather (same tables and order as the imaging kernel), row FFTs
    {
      const int y = line;
      float2 v[P][8];
      int Ks[8], bs[8];  // read before the first slot, as in the imaging kernel
      if constexpr (!Q) {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
          Ks[n2] = cnt_s[warp * 8 + n2];
          bs[n2] = base_s[warp * 8 + n2];
        }
      }
#pragma unroll
      for (int n2 = 0; n2 < 8; ++n2) {
        const int K = Q ? cnt_s[warp * 8 + n2] : Ks[n2];
        const int bse = Q ? base_s[warp * 8 + n2] : bs[n2];
        const uint32_t* ea2 = reinterpret_cast<const uint32_t*>(ent_a) + (bse >> 1) + lane;
        const float2* ew2 = reinterpret_cast<const float2*>(ent_w) + (bse >> 1) + lane;
        float2 gx = make_float2(0.f, 0.f), gy = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int k = 0; k < K; k += 2) {  // the imaging kernel's entry pairs, in the same order
          const uint32_t aa = ea2[16 * k];
          const float2 ww = ew2[16 * k];
          const int a0 = (int)(aa & 0xffffu), a1 = (int)(aa >> 16);
          const float w0 = ww.x, w1 = ww.y;
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
        if constexpr (Q) {
          // H_q = exp(+2 pi i (alpha x + beta y) / 128) x the folded gather, as in fft_image_kernel
          const float2 w = __ldg(twiddle + (((cur_c & 1) * (n1 + R1 * n2) + ((cur_c >> 1) & 1) * y) & 127));
          gx = make_float2(gx.x * w.x - gx.y * w.y, gx.x * w.y + gx.y * w.x);
          gy = make_float2(gy.x * w.x - gy.y * w.y, gy.x * w.y + gy.y * w.x);
        }
        v[0][n2] = gx;
        if constexpr (P == 2) v[1][n2] = gy;
      }
      const int sw = G::swz(y);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        fft_line<N>(v[p], tw, scr, r, n1);
        float2* Rrow = Rbuf + (size_t)p * NN + y * N;
#pragma unroll
        for (int s = 0; s < 8; ++s) Rrow[G::rowpos(n1, s, sw)] = v[p][s];
      }
    }
    __syncthreads();

    // 3. forward column FFTs -> Y; conj(R . Y); conjugate column FFTs; write back
    {
      const int k = line;
      const int col = (k + HALF) & (N - 1);
      // both polarisations' columns loaded before the first transform (its warp
      // syncs would otherwise hold the second one's loads back)
      float2 vp[P][8];
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int m2 = 0; m2 < 8; ++m2) {
          const int y = n1 + R1 * m2;
          vp[p][m2] = Rbuf[(size_t)p * NN + y * N + (k ^ G::swz(y))];
        }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        float2 (&v)[8] = vp[p];
        fft_line<N>(v, tw, scr, r, n1);
        // thread (k, q = n1) holds Y[j = n1 + 8 s][k]; pixel row (j + N/2) mod N
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int row = (G::kidx(n1, s) + HALF) & (N - 1);
          const float rr = res_s[(size_t)p * NN + row * N + col];
          v[s] = make_float2(rr * v[s].x, -rr * v[s].y);  // conj(R Y)
        }
        if constexpr (N != 64) {
          // at N = 32 a thread's outputs (rows kidx(n1, s)) are not the elements
          // n1 + R1 s the next transform takes: pass the column through shared
          // memory (its R1 threads are lanes of one warp, the only ones using it)
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const int y = G::kidx(n1, s);
            Rbuf[(size_t)p * NN + y * N + (k ^ G::swz(y))] = v[s];
          }
          __syncwarp();
#pragma unroll
          for (int m2 = 0; m2 < 8; ++m2) {
            const int y = n1 + R1 * m2;
            v[m2] = Rbuf[(size_t)p * NN + y * N + (k ^ G::swz(y))];
          }
          __syncwarp();
        }
        fft_line<N>(v, tw, scr, r, n1);  // at N = 64 element index n1 + 8 s: the input layout again
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int y = G::kidx(n1, s);
          Rbuf[(size_t)p * NN + y * N + (k ^ G::swz(y))] = v[s];
        }
      }
    }
    __syncthreads();

    // 4. conjugate row FFTs -> H = conj(result) on the thread's own cells (y, n1 + 8 s)
    {
      const int y = line;
      const int sw = G::swz(y);
      // element n1 + R1 n2 of the row (at N = 64 the same position as rowpos(n1, n2)),
      // both polarisations loaded first
      float2 vp[P][8];
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) vp[p][n2] = Rbuf[(size_t)p * NN + y * N + ((n1 + R1 * n2) ^ sw)];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        float2 (&v)[8] = vp[p];
        float2* Rrow = Rbuf + (size_t)p * NN + y * N;
        fft_line<N>(v, tw, scr, r, n1);
#pragma unroll
        for (int s = 0; s < 8; ++s) Rrow[G::rowpos(n1, s, sw)] = make_float2(v[s].x, -v[s].y);
      }
    }
    __syncthreads();

    // 5. degrid H over each antenna's box and accumulate conj(e~) D
    if (tid < A) {
      const int2 bx = box_s[tid];
      float2 D[P];
#pragma unroll
      for (int p = 0; p < P; ++p) D[p] = make_float2(0.f, 0.f);
      for (int dy = 0; dy < S; ++dy) {
        const int yg = bx.y + dy, y = yg & (N - 1);  // grid row, and its row of the folded field
        const float wyv = wy_s[tid * S + dy];
        const int sw = G::swz(y);
        for (int dx = 0; dx < S; ++dx) {
          const int xg = bx.x + dx, x = xg & (N - 1);
          float w = wyv * wx_s[tid * S + dx];
          float2 tc = make_float2(1.f, 0.f);
          if constexpr (Q) {
            // the fold's adjoint: sign (-1)^(alpha s + beta u), conj(Tw[y][x])
            const int al = cur_c & 1, be = (cur_c >> 1) & 1;
            if ((al & (xg >> 6)) ^ (be & (yg >> 6))) w = -w;
            const float2 tw128 = __ldg(twiddle + ((al * x + be * y) & 127));
            tc = make_float2(tw128.x, -tw128.y);
          }
          const int idx = y * N + (x ^ sw);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            float2 h = Rbuf[(size_t)p * NN + idx];
            if constexpr (Q) h = make_float2(h.x * tc.x - h.y * tc.y, h.x * tc.y + h.y * tc.x);
            D[p].x = fmaf(w, h.x, D[p].x);
            D[p].y = fmaf(w, h.y, D[p].y);
          }
        }
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const unsigned b = (raw >> (8 * p)) & 0xffu;
        const int re = nib_hi(b), im = nib_lo(b);
        const float2 d = dph_s[tid * P + p];
        const float er = d.x * re - d.y * im, ei = d.x * im + d.y * re;  // e~ = delay phase x E'
        gacc[p].x = fmaf(er, D[p].x, fmaf(ei, D[p].y, gacc[p].x));     // conj(e~) D
        gacc[p].y = fmaf(er, D[p].y, fmaf(-ei, D[p].x, gacc[p].y));
      }
    }
  }
  flush(cur_c);
}

}  // namespace

cudaError_t launch_fft_image_coef(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, const float2* coef,
                                  cudaStream_t s) {
  return launch_image_any(p, d_volts, T, ws, coef, p.d_part, p.d_part_auto, s);
}

namespace {
size_t adj_smem(const Plan& p, int ent) {
  const int me = p.gt.max_chan_entries;
  if (p.N == 32)
    return p.P == 2 ? adj_smem_layout<32, 2>(p.A, p.S, me, ent).total : adj_smem_layout<32, 1>(p.A, p.S, me, ent).total;
  return p.P == 2 ? adj_smem_layout<64, 2>(p.A, p.S, me, ent).total : adj_smem_layout<64, 1>(p.A, p.S, me, ent).total;
}

template <int N, int P, bool Q>
cudaError_t adjoint_launch(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, int ent, size_t smem,
                           cudaStream_t s) {
  auto fn = adjoint_kernel<N, P, Q>;
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  fn<<<ws.ctas, Geo<N>::THREADS, smem, s>>>(d_volts, T, p.C, p.A, p.S, ws.W, ws.units, ws.spans, p.d_gcoef,
                                            p.d_dphase, p.gt.d_cnt, p.gt.d_base, p.gt.d_chan_off, p.gt.d_ent_a,
                                            p.gt.d_ent_w, p.gt.max_chan_entries, ent, p.d_twiddle, p.d_resid,
                                            p.d_box, p.d_wx, p.d_wy, p.d_gpart);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_adjoint(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, cudaStream_t s) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int ent = adj_smem(p, 1) <= (size_t)optin ? 1 : 0;
  const size_t smem = adj_smem(p, ent);
  if (p.N == 32)
    return p.P == 2 ? adjoint_launch<32, 2, false>(p, d_volts, T, ws, ent, smem, s)
                    : adjoint_launch<32, 1, false>(p, d_volts, T, ws, ent, smem, s);
  if (p.N == 128)  // folded into four 64 x 64 problems
    return p.P == 2 ? adjoint_launch<64, 2, true>(p, d_volts, T, ws, ent, smem, s)
                    : adjoint_launch<64, 1, true>(p, d_volts, T, ws, ent, smem, s);
  return p.P == 2 ? adjoint_launch<64, 2, false>(p, d_volts, T, ws, ent, smem, s)
                  : adjoint_launch<64, 1, false>(p, d_volts, T, ws, ent, smem, s);
}

// Antennas an adjoint launch handles: one per thread.
int adjoint_max_ant(int N) { return N == 32 ? Geo<32>::THREADS : Geo<64>::THREADS; }

size_t adjoint_smem_need(const Plan& p) { return adj_smem(p, 0); }

}  // namespace epic
