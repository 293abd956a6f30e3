// epic_plan.cu -- plan-time terms, generated on the GPU in FP64 (Sec. 3.2).
//
// Per (channel c, antenna a):
//   lambda_c = c0 / nu_c;  u = x_a / (lambda_c d) + N/2;  v likewise     (Sec. 3.2,
//   grid spacing of a fraction of each channel's wavelength);
//   box origin i0 = floor(u + 1/2) - (S-1)/2, j0 likewise;
//   Gaussian illumination kernel sampled at cell centres and normalised to sum 1,
//   stored as its two 1-D factors w_x[S], w_y[S] (a Gaussian separates exactly);
//   |FT w_x|^2 on every output column and |FT w_y|^2 on every output row, the
//   factors of |W_a(l,m)|^2 used to remove the autocorrelation term (Fig. 2);
//   calibration coefficient k = g exp(-2 pi i nu tau) per polarisation (Sec. 3.2
//   delay compensation, Fig. 2 gain multiplication).
// Then the gridder's gather table: for every cell, the antennas whose box covers
// it, in antenna order, with weight w_x * w_y (FP64 product rounded to FP32).
#include <cmath>

#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr double kC0 = 299792458.0;

// Cell coordinate of a position; every operation rounded on its own (no fused
// multiply-add) so that the host-side validation reproduces it bit for bit.
__device__ __forceinline__ double cell_coord(double pos_m, double freq_hz, double cell_lambda, int N) {
  const double lambda = __ddiv_rn(kC0, freq_hz);
  return __dadd_rn(__ddiv_rn(pos_m, __dmul_rn(lambda, cell_lambda)), 0.5 * (double)N);
}

__global__ void plan_terms_kernel(int A, int P, int C, int N, int S, double cell_lambda, double sigma,
                                  const double* __restrict__ ant_xy, const double* __restrict__ freq,
                                  const double* __restrict__ gains, const double* __restrict__ delays,
                                  int* __restrict__ box, double* __restrict__ wx, double* __restrict__ wy,
                                  float2* __restrict__ coef, double2* __restrict__ coef64,
                                  double2* __restrict__ dphase,
                                  float* __restrict__ kx2, float* __restrict__ ky2, int* __restrict__ status) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)C * A) return;
  const int c = (int)(idx / A), a = (int)(idx % A);
  const double nu = freq[c];
  const double u = cell_coord(ant_xy[2 * a + 0], nu, cell_lambda, N);
  const double v = cell_coord(ant_xy[2 * a + 1], nu, cell_lambda, N);
  const int i0 = (int)floor(__dadd_rn(u, 0.5)) - (S - 1) / 2;
  const int j0 = (int)floor(__dadd_rn(v, 0.5)) - (S - 1) / 2;
  if (i0 < 0 || j0 < 0 || i0 + S > N || j0 + S > N) atomicExch(status, kDevOffGrid);
  box[2 * idx + 0] = i0;
  box[2 * idx + 1] = j0;

  // 1-D Gaussian factors, each normalised to sum 1 (their product then sums to 1)
  double fx[16], fy[16];
  double sx = 0.0, sy = 0.0;
  for (int k = 0; k < S; ++k) {
    if (S == 1) {
      fx[k] = 1.0;
      fy[k] = 1.0;
    } else {
      const double dx = (double)(i0 + k) - u, dy = (double)(j0 + k) - v;
      fx[k] = exp(-(dx * dx) / (2.0 * sigma * sigma));
      fy[k] = exp(-(dy * dy) / (2.0 * sigma * sigma));
    }
    sx += fx[k];
    sy += fy[k];
  }
  for (int k = 0; k < S; ++k) {
    fx[k] /= sx;
    fy[k] /= sy;
    wx[idx * S + k] = fx[k];
    wy[idx * S + k] = fy[k];
  }

  // |sum_k w[k] exp(+2 pi i f k / N)|^2 for f = i - N/2 (the box origin only
  // contributes a unit-modulus phase)
  for (int i = 0; i < N; ++i) {
    const int f = i - N / 2;
    double xr = 0.0, xi = 0.0, yr = 0.0, yi = 0.0;
    for (int k = 0; k < S; ++k) {
      const int m = (((f * k) % N) + N) % N;
      double sn, cs;
      sincospi(2.0 * (double)m / (double)N, &sn, &cs);
      xr += fx[k] * cs;
      xi += fx[k] * sn;
      yr += fy[k] * cs;
      yi += fy[k] * sn;
    }
    kx2[idx * N + i] = (float)(xr * xr + xi * xi);
    ky2[idx * N + i] = (float)(yr * yr + yi * yi);
  }

  // k = g * exp(-2 pi i nu tau)
  for (int p = 0; p < P; ++p) {
    double gr = 1.0, gi = 0.0, tau = 0.0;
    if (gains) {
      gr = gains[2 * (idx * P + p)];
      gi = gains[2 * (idx * P + p) + 1];
    }
    if (delays) tau = delays[a * P + p];
    double sn, cs;
    sincospi(-2.0 * nu * tau, &sn, &cs);
    const double kr = gr * cs - gi * sn, ki = gr * sn + gi * cs;
    coef64[idx * P + p] = make_double2(kr, ki);
    coef[idx * P + p] = make_float2((float)kr, (float)ki);
    dphase[idx * P + p] = make_double2(cs, sn);
  }
}

__global__ void twiddle_kernel(int N, float2* __restrict__ tw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  double sn, cs;
  sincospi(2.0 * (double)m / (double)N, &sn, &cs);
  tw[m] = make_float2((float)cs, (float)sn);
}

// One CTA per channel.  Pass 1 counts, per cell, the antennas whose box covers
// it; a block scan turns counts into row pointers; pass 2 writes the entries in
// antenna order, so the table (and every sum over it) is deterministic.
constexpr int kCsrThreads = 1024;

__global__ void __launch_bounds__(kCsrThreads) build_csr_kernel(int A, int N, int S, const int* __restrict__ box,
                                                                const double* __restrict__ wx,
                                                                const double* __restrict__ wy,
                                                                int* __restrict__ csr_ptr, int2* __restrict__ csr_ent) {
  extern __shared__ int sh[];
  int* bx = sh;                 // [A][2]
  int* tsum = sh + 2 * A;       // [kCsrThreads]
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  const int NN = N * N;
  const int* cbox = box + (size_t)c * A * 2;
  for (int k = tid; k < 2 * A; k += blockDim.x) bx[k] = cbox[k];
  __syncthreads();

  // contiguous chunk of cells per thread
  const int per = (NN + blockDim.x - 1) / blockDim.x;
  const int cell0 = min(tid * per, NN), cell1 = min(cell0 + per, NN);
  int local = 0;
  for (int cell = cell0; cell < cell1; ++cell) {
    const int y = cell / N, x = cell % N;
    for (int a = 0; a < A; ++a) {
      const int dx = x - bx[2 * a], dy = y - bx[2 * a + 1];
      local += (dx >= 0 && dx < S && dy >= 0 && dy < S);
    }
  }
  tsum[tid] = local;
  __syncthreads();
  // inclusive Hillis-Steele scan of the per-thread totals
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const int add = (tid >= off) ? tsum[tid - off] : 0;
    __syncthreads();
    tsum[tid] += add;
    __syncthreads();
  }
  int run = tsum[tid] - local;  // exclusive prefix of this thread's chunk
  int* ptr = csr_ptr + (size_t)c * (NN + 1);
  int2* ent = csr_ent + (size_t)c * A * S * S;
  const double* cwx = wx + (size_t)c * A * S;
  const double* cwy = wy + (size_t)c * A * S;
  for (int cell = cell0; cell < cell1; ++cell) {
    ptr[cell] = run;
    const int y = cell / N, x = cell % N;
    for (int a = 0; a < A; ++a) {
      const int dx = x - bx[2 * a], dy = y - bx[2 * a + 1];
      if (dx >= 0 && dx < S && dy >= 0 && dy < S) {
        const float w = (float)(cwx[a * S + dx] * cwy[a * S + dy]);
        ent[run] = make_int2(a, __float_as_int(w));
        ++run;
      }
    }
  }
  if (tid == blockDim.x - 1) ptr[NN] = tsum[tid];
}

// Image of the illumination kernels (Sec. 3.2, last paragraph: "the imprint of
// the image of the gridding illumination kernels"): B_c(l,m) = (1/A) sum_a
// |W_a(l,m)|^2, each factor the product of the antenna's 1-D power spectra;
// 1 at the zero frequency since every kernel sums to 1.
__global__ void beam_kernel(int A, int N, const float* __restrict__ kx2, const float* __restrict__ ky2,
                            float* __restrict__ beam) {
  const int c = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= N * N) return;
  const int j = pix / N, i = pix % N;
  double s = 0.0;
  for (int a = 0; a < A; ++a)
    s += (double)kx2[((size_t)c * A + a) * N + i] * (double)ky2[((size_t)c * A + a) * N + j];
  beam[(size_t)c * N * N + pix] = (float)(s / A);
}

}  // namespace

cudaError_t launch_beam(Plan& p, cudaStream_t s) {
  dim3 grid((p.N * p.N + 255) / 256, p.C);
  beam_kernel<<<grid, 256, 0, s>>>(p.A, p.N, p.d_kx2, p.d_ky2, p.d_beam);
  return cudaGetLastError();
}

cudaError_t launch_plan_terms(Plan& p, cudaStream_t s) {
  const long long n = (long long)p.C * p.A;
  const int threads = 128;
  const long long blocks = (n + threads - 1) / threads;
  plan_terms_kernel<<<(unsigned)blocks, threads, 0, s>>>(p.A, p.P, p.C, p.N, p.S, p.cell_lambda, p.sigma,
                                                          p.d_ant_xy, p.d_freq, p.d_gains, p.d_delays, p.d_box,
                                                          p.d_wx, p.d_wy, p.d_coef, p.d_coef64, p.d_dphase, p.d_kx2, p.d_ky2,
                                                          p.d_status);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(Plan& p, cudaStream_t s) {
  twiddle_kernel<<<(p.N + 127) / 128, 128, 0, s>>>(p.N, p.d_twiddle);
  return cudaGetLastError();
}

cudaError_t launch_build_csr(Plan& p, cudaStream_t s) {
  const size_t smem = sizeof(int) * (2 * (size_t)p.A + kCsrThreads);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(build_csr_kernel);
    if (e != cudaSuccess) return e;
  }
  build_csr_kernel<<<p.C, kCsrThreads, smem, s>>>(p.A, p.N, p.S, p.d_box, p.d_wx, p.d_wy, p.d_csr_ptr, p.d_csr_ent);
  return cudaGetLastError();
}

}  // namespace epic
