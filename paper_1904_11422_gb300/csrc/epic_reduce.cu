// epic_reduce.cu -- block end of an imaging call (Fig. 2 "Remove
// Autocorrelations"): sum the per-CTA partial images of each channel in CTA
// order, subtract the autocorrelation term and write or accumulate the output.
//
// The autocorrelation term of pixel (l, m) is sum_a P_a |W_a(l,m)|^2 (reading
// R9), with P_a the antenna's self power accumulated over the block (exact
// integer sums times |k|^2, or k_X conj(k_Y) for XY, formed in FP64) and
// |W_a|^2 = |FT w_x|^2 (column) x |FT w_y|^2 (row) of its separable kernel.
#include "epic_internal.cuh"
#include "epic_reduce.cuh"

namespace epic {

namespace {

constexpr int kReduceThreads = 256;
constexpr int kReducePixels = 1;     // pixels of one row per thread (more warps beat more reuse here)
constexpr size_t kReduceSmemCap = 64 * 1024;

// One block per (virtual channel, `rows` rows); the arithmetic is reduce_rows
// (epic_reduce.cuh), which the persistent batch kernel runs too.
template <int P>
__global__ void __launch_bounds__(kReduceThreads)
    reduce_kernel(int T, int C, int A, int N, int vq, int dec, long long W, int ctas, int spans, int subtract,
                  int accumulate,
                  int rows, const float* __restrict__ part, const int* __restrict__ part_auto,
                  const double2* __restrict__ coef64, const float* __restrict__ kx2, const float* __restrict__ ky2,
                  float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ReduceArgs r{T, C, A, N, vq, dec, ctas, spans, subtract, accumulate, W, part, part_auto, coef64,
                     kx2, ky2, out};
  reduce_rows<P, kReducePixels>(r, blockIdx.x, blockIdx.y * rows, rows, threadIdx.x, blockDim.x, smem);
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
  const int rows = reduce_rows_per_piece(L, kReduceThreads * kReducePixels, p.A, kReduceSmemCap);
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
  const int rows = reduce_rows_per_piece(L, kReduceThreads * kReducePixels, p.A, kReduceSmemCap);
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
  const int rows = reduce_rows_per_piece(L, kReduceThreads * kReducePixels, p.A, kReduceSmemCap);
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
