// epic_reduce.cu -- block end of an imaging call (Fig. 2 "Remove
// Autocorrelations"): sum the per-CTA partial images of each channel in CTA
// order, subtract the autocorrelation term and write or accumulate the output.
//
// The autocorrelation term of pixel (l, m) is sum_a P_a |W_a(l,m)|^2 (reading
// R9), with P_a the antenna's self power accumulated over the block (exact
// integer sums times |k|^2, or k_X conj(k_Y) for XY, formed in FP64) and
// |W_a|^2 = |FT w_x|^2 (column) x |FT w_y|^2 (row) of its separable kernel.
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int kReduceThreads = 256;

// One block per (channel, `rows` rows).  With vq = 4 (the tensor path on
// 128 x 128 grids) the partials are the 64 x 64 sub-images of virtual channels
// 4 c + q, and pixel (j, i) of sub-image q lands on output pixel
// (2 j + beta, 2 i + alpha), alpha = q & 1, beta = q >> 1.  With dec = 2 (the
// tensor path on 32 x 32 grids) the partials are 64 x 64 and output pixel (j, i)
// is their pixel (2 j, 2 i).
template <int P>
__global__ void __launch_bounds__(kReduceThreads)
    reduce_kernel(int T, int C, int A, int N, int vq, int dec, long long W, int ctas, int spans, int subtract,
                  int accumulate,
                  int rows, const float* __restrict__ part, const int* __restrict__ part_auto,
                  const double2* __restrict__ coef64, const float* __restrict__ kx2, const float* __restrict__ ky2,
                  float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* Pw = reinterpret_cast<float4*>(smem);        // [A] self powers XX, YY, Re XY, Im XY
  float* kys = reinterpret_cast<float*>(Pw + A);       // [A][rows] |FT w_y|^2 of this block's rows
  const int cv = blockIdx.x;                           // (virtual) channel of the partials
  const int c = vq == 4 ? cv >> 2 : cv;                // output channel
  const int alpha = vq == 4 ? (cv & 1) : 0, beta = vq == 4 ? (cv >> 1) & 1 : 0;
  const int Ns = vq == 4 ? N / 2 : N * dec;            // side of a partial image
  const int L = vq == 4 ? Ns : N;                      // side of the pixel loop
  const int j0 = blockIdx.y * rows;
  const int NN = N * N, NNs = Ns * Ns;
  auto orow = [&](int j) { return vq == 4 ? 2 * j + beta : j; };
  auto ocol = [&](int i) { return vq == 4 ? 2 * i + alpha : i; };
  const long long b_lo = ((long long)cv * T) / W;
  const long long b_hi = min(((long long)(cv + 1) * T - 1) / W, (long long)ctas - 1);

  if (subtract) {
    for (int a = threadIdx.x; a < A; a += blockDim.x) {
      long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (long long b = b_lo; b <= b_hi; ++b) {
        const int slot = cv - (int)((b * W) / T);
        const int4 v = reinterpret_cast<const int4*>(part_auto)[(b * spans + slot) * A + a];
        s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
      }
      const double2 kx = coef64[((size_t)c * A + a) * P];
      float4 pw = make_float4((float)((kx.x * kx.x + kx.y * kx.y) * (double)s0), 0.f, 0.f, 0.f);
      if (P == 2) {
        const double2 ky = coef64[((size_t)c * A + a) * P + 1];
        const double mr = kx.x * ky.x + kx.y * ky.y, mi = kx.y * ky.x - kx.x * ky.y;  // k_X conj(k_Y)
        pw.y = (float)((ky.x * ky.x + ky.y * ky.y) * (double)s1);
        pw.z = (float)(mr * (double)s2 - mi * (double)s3);
        pw.w = (float)(mr * (double)s3 + mi * (double)s2);
      }
      Pw[a] = pw;
      for (int jj = 0; jj < rows; ++jj) kys[a * rows + jj] = ky2[((size_t)c * A + a) * N + orow(j0 + jj)];
    }
    __syncthreads();
  }

  for (int q = threadIdx.x; q < rows * L; q += blockDim.x) {
    const int jj = q / L, i = q % L, pix = dec * (j0 + jj) * Ns + dec * i;
    const int opix = orow(j0 + jj) * N + ocol(i);
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long b = b_lo; b <= b_hi; ++b) {
      const int slot = cv - (int)((b * W) / T);
      const float* src = part + (size_t)(b * spans + slot) * 4 * NNs + pix;
      s[0] += src[0];
      if (P == 2) {
        s[1] += src[NNs];
        s[2] += src[2 * NNs];
        s[3] += src[3 * NNs];
      }
    }
    if (subtract) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      const float* kxc = kx2 + (size_t)c * A * N + ocol(i);
      for (int a = 0; a < A; ++a) {
        const float w2 = kxc[(size_t)a * N] * kys[a * rows + jj];
        const float4 pw = Pw[a];
        a0 = fmaf(pw.x, w2, a0);
        if (P == 2) {
          a1 = fmaf(pw.y, w2, a1);
          a2 = fmaf(pw.z, w2, a2);
          a3 = fmaf(pw.w, w2, a3);
        }
      }
      s[0] -= a0; s[1] -= a1; s[2] -= a2; s[3] -= a3;
    }
    float* o = out + (size_t)c * 4 * NN + opix;
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) o[pl * NN] = accumulate ? o[pl * NN] + s[pl] : s[pl];
  }
}

// Post-processing of accumulated images, one thread per (channel, pixel):
// pseudo-Stokes planes from the coherencies of linear feeds (Sec. 4.3: linear
// combinations of the coherency products; YX = conj XY) and division by the
// kernel imprint (Sec. 3.2, last paragraph).
__global__ void postprocess_kernel(int C, int NN, int flags, float floor, const float* __restrict__ beam,
                                   const float* in, float* out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)C * NN) return;
  const size_t c = idx / NN, pix = idx % NN;
  float v[4];
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) v[pl] = in[(c * 4 + pl) * NN + pix];
  if (flags & EPIC_POST_STOKES) {
    const float xx = v[0], yy = v[1], xyr = v[2], xyi = v[3];
    v[0] = xx + yy;          // I
    v[1] = xx - yy;          // Q
    v[2] = 2.f * xyr;        // U = XY + YX
    v[3] = 2.f * xyi;        // V = -i (XY - YX)
  }
  if (flags & EPIC_POST_BEAM) {
    const float b = beam[c * NN + pix];
    const float scale = b >= floor ? 1.f / b : 0.f;
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) v[pl] *= scale;
  }
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) out[(c * 4 + pl) * NN + pix] = v[pl];
}

__global__ void zero_kernel(float* __restrict__ out, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    out[k] = 0.f;
}

__global__ void debug_unpack_kernel(const uint8_t* __restrict__ in, size_t n, int8_t* __restrict__ out) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const unsigned b = in[k];
    out[2 * k] = (int8_t)nib_hi(b);
    out[2 * k + 1] = (int8_t)nib_lo(b);
  }
}

}  // namespace

cudaError_t launch_reduce(Plan& p, int T, const WorkSplit& ws, float* d_out, int accumulate, cudaStream_t s) {
  const int L = p.vq == 4 ? p.N / 2 : p.N;  // side of the reduction's pixel loop
  int rows = 1;
  while (rows * L < kReduceThreads && rows < L) rows *= 2;
  const size_t smem = p.subtract ? (sizeof(float4) * p.A + sizeof(float) * (size_t)p.A * rows) : 16;
  auto fn = p.P == 2 ? reduce_kernel<2> : reduce_kernel<1>;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(fn);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(p.C * p.vq, L / rows);
  fn<<<grid, kReduceThreads, smem, s>>>(T, p.C, p.A, p.N, p.vq, p.dec, ws.W, ws.ctas, ws.spans, p.subtract, accumulate, rows,
                                        p.d_part, p.d_part_auto, p.d_coef64, p.d_kx2, p.d_ky2, d_out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_ws(const Plan& p, int T, const WorkSplit& ws, const float* part, const int* part_auto,
                             float* d_out, int accumulate, cudaStream_t s) {
  const int L = p.vq == 4 ? p.N / 2 : p.N;  // side of the reduction's pixel loop
  int rows = 1;
  while (rows * L < kReduceThreads && rows < L) rows *= 2;
  const size_t smem = p.subtract ? (sizeof(float4) * p.A + sizeof(float) * (size_t)p.A * rows) : 16;
  auto fn = p.P == 2 ? reduce_kernel<2> : reduce_kernel<1>;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(fn);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(p.C * p.vq, L / rows);
  fn<<<grid, kReduceThreads, smem, s>>>(T, p.C, p.A, p.N, p.vq, p.dec, ws.W, ws.ctas, ws.spans, p.subtract, accumulate, rows,
                                        part, part_auto, p.d_coef64, p.d_kx2, p.d_ky2, d_out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_coef(Plan& p, int T, const WorkSplit& ws, const double2* coef64, float* d_out,
                               cudaStream_t s) {
  const int L = p.vq == 4 ? p.N / 2 : p.N;  // side of the reduction's pixel loop
  int rows = 1;
  while (rows * L < kReduceThreads && rows < L) rows *= 2;
  const size_t smem = p.subtract ? (sizeof(float4) * p.A + sizeof(float) * (size_t)p.A * rows) : 16;
  auto fn = p.P == 2 ? reduce_kernel<2> : reduce_kernel<1>;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(fn);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(p.C * p.vq, L / rows);
  fn<<<grid, kReduceThreads, smem, s>>>(T, p.C, p.A, p.N, p.vq, p.dec, ws.W, ws.ctas, ws.spans, p.subtract, 0, rows, p.d_part,
                                        p.d_part_auto, coef64, p.d_kx2, p.d_ky2, d_out);
  return cudaGetLastError();
}

cudaError_t launch_postprocess(const Plan& p, const float* d_in, float* d_out, int flags, float floor,
                               cudaStream_t s) {
  const size_t n = (size_t)p.C * p.N * p.N;
  postprocess_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.C, p.N * p.N, flags, floor, p.d_beam, d_in,
                                                                   d_out);
  return cudaGetLastError();
}

cudaError_t launch_zero(float* d_out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  zero_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(d_out, n);
  return cudaGetLastError();
}

cudaError_t launch_debug_unpack(const uint8_t* d_in, size_t n, int8_t* d_out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  debug_unpack_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(d_in, n, d_out);
  return cudaGetLastError();
}

}  // namespace epic
