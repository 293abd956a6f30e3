// epic_grad.cu -- gradient of an image-plane calibration loss with respect to
// the per-antenna complex gains (the gain multiplication of Fig. 2, which the
// EPICal block the paper plans would solve for; Sec. 6).
//
//   L = sum_c sum_{pp in XX, YY} sum_pix (I_pp - M_pp)^2,   R = 2 (I - M),
//   dL/d conj(g_ap) = sum_t conj(e~_ap) D_ap(t)  -  [autos removed] g_ap P~_ap S_ap,
//   S_ap = sum_pix R_pp(pix) |W_a(pix)|^2,   P~_ap = sum_t |E'_ap|^2,
// and the returned gradient is dL/dRe g + i dL/dIm g = 2 dL/d conj(g).  The data
// term comes from the adjoint kernel (epic_fft.cu); this file holds the
// coefficient, residual/loss and final reduction kernels and the entry point.
#include "epic_internal.cuh"

namespace epic {

namespace {

// k = g * exp(-2 pi i nu tau) of the call, FP32 and FP64
__global__ void grad_coef_kernel(int n, const float* __restrict__ gains, const double2* __restrict__ dphase,
                                 float2* __restrict__ coef, double2* __restrict__ coef64) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double gr = gains[2 * k], gi = gains[2 * k + 1];
  const double2 d = dphase[k];
  const double kr = gr * d.x - gi * d.y, ki = gr * d.y + gi * d.x;
  coef64[k] = make_double2(kr, ki);
  coef[k] = make_float2((float)kr, (float)ki);
}

// R = 2 (I - M) for XX (and YY), and the channel's share of the loss (FP64,
// fixed-order block reduction).  One block per channel.
constexpr int kResThreads = 256;
__global__ void __launch_bounds__(kResThreads)
    residual_kernel(int NN, int P, const float* __restrict__ image, const float* __restrict__ model,
                    float* __restrict__ resid, double* __restrict__ loss_part) {
  __shared__ double red[kResThreads];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int p = 0; p < P; ++p)
    for (int k = threadIdx.x; k < NN; k += blockDim.x) {
      const float d = image[((size_t)c * 4 + p) * NN + k] - model[((size_t)c * 2 + p) * NN + k];
      resid[((size_t)c * 2 + p) * NN + k] = 2.f * d;
      acc += (double)d * (double)d;
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[c] = red[0];
}

__global__ void loss_sum_kernel(int C, const double* __restrict__ loss_part, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int c = 0; c < C; ++c) s += loss_part[c];
    *loss = (float)s;
  }
}

// Final gradient per (c, a, p): CTA sums of the data term in CTA order (FP64),
// minus the autocorrelation term, times 2.  Block (c, group of 8 antennas), one
// warp per antenna; the channel's residual planes are staged in shared memory
// (row stride N + 1, so the lanes' rows fall in different banks).  For
// S = sum_pix R |W_a|^2 = sum_j |FT w_y(j)|^2 sum_i R[j][i] |FT w_x(i)|^2 the lanes
// take rows j = lane, lane + 32, ... (each row sum in FP32 in column order), and
// the warp adds |FT w_y(j)| x row in FP64.
constexpr int kGradAntPerBlock = 8;
__global__ void __launch_bounds__(32 * kGradAntPerBlock)
    grad_reduce_kernel(int T, int A, int P, int N, int vq, long long W, int ctas, int spans, int subtract,
                       const float2* __restrict__ gpart, const int* __restrict__ part_auto,
                       const float* __restrict__ resid, const float* __restrict__ kx2,
                       const float* __restrict__ ky2, const float* __restrict__ gains,
                       float* __restrict__ grad) {
  extern __shared__ float Rs[];  // [P][N][N + 1]
  const int c = blockIdx.x, NN = N * N, ld = N + 1;
  if (subtract)
    for (int k = threadIdx.x; k < P * NN; k += blockDim.x) {
      const int p = k / NN, j = (k % NN) / N, i = k % N;
      Rs[(p * N + j) * ld + i] = resid[((size_t)c * 2 + p) * NN + j * N + i];
    }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.y * kGradAntPerBlock + warp;
  if (a >= A) return;
  // data term: the CTA sums of every (virtual) channel of c, in order; self
  // powers from the first (each virtual channel of a folded grid holds them all)
  double dr[2] = {0.0, 0.0}, di[2] = {0.0, 0.0};
  long long pw[2] = {0, 0};
  for (int q = 0; q < vq; ++q) {
    const int cv = c * vq + q;
    const long long b_lo = ((long long)cv * T) / W;
    const long long b_hi = min(((long long)(cv + 1) * T - 1) / W, (long long)ctas - 1);
    for (long long b = b_lo; b <= b_hi; ++b) {
      const int slot = cv - (int)((b * W) / T);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        if (p >= P) break;
        const float2 v = gpart[((size_t)(b * spans + slot) * A + a) * P + p];
        dr[p] += v.x;
        di[p] += v.y;
      }
      if (q == 0) {
        const int4 qa = reinterpret_cast<const int4*>(part_auto)[(b * spans + slot) * A + a];
        pw[0] += qa.x;
        pw[1] += qa.y;
      }
    }
  }
  const float* kx = kx2 + ((size_t)c * A + a) * N;
  const float* ky = ky2 + ((size_t)c * A + a) * N;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    if (p >= P) break;
    double S = 0.0;
    if (subtract) {
      for (int j = lane; j < N; j += 32) {
        const float* Rj = Rs + (p * N + j) * ld;
        float row = 0.f;
        for (int i = 0; i < N; ++i) row = fmaf(Rj[i], __ldg(kx + i), row);
        S += (double)__ldg(ky + j) * (double)row;
      }
      for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(0xffffffffu, S, off);
    }
    if (lane == 0) {
      double ar = 0.0, ai = 0.0;
      if (subtract) {
        const double gr = gains[2 * (((size_t)c * A + a) * P + p)], gi = gains[2 * (((size_t)c * A + a) * P + p) + 1];
        ar = gr * (double)pw[p] * S;
        ai = gi * (double)pw[p] * S;
      }
      float* o = grad + 2 * (((size_t)c * A + a) * P + p);
      o[0] = (float)(2.0 * (dr[p] - ar));
      o[1] = (float)(2.0 * (di[p] - ai));
    }
  }
}

}  // namespace

cudaError_t launch_grad_coef(Plan& p, const float* d_gains, cudaStream_t s) {
  const int n = p.C * p.A * p.P;
  grad_coef_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, d_gains, p.d_dphase, p.d_gcoef, p.d_gcoef64);
  return cudaGetLastError();
}

cudaError_t launch_residual(Plan& p, const float* d_model, float* d_loss, cudaStream_t s) {
  residual_kernel<<<p.C, kResThreads, 0, s>>>(p.N * p.N, p.P, p.d_gimage, d_model, p.d_resid, p.d_loss_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  loss_sum_kernel<<<1, 32, 0, s>>>(p.C, p.d_loss_part, d_loss);
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(Plan& p, int T, const WorkSplit& ws, const float* d_gains, float* d_grad,
                               cudaStream_t s) {
  const size_t smem = p.subtract ? sizeof(float) * (size_t)p.P * p.N * (p.N + 1) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(grad_reduce_kernel);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(p.C, (p.A + kGradAntPerBlock - 1) / kGradAntPerBlock);
  grad_reduce_kernel<<<grid, 32 * kGradAntPerBlock, smem, s>>>(T, p.A, p.P, p.N, p.vq, ws.W, ws.ctas, ws.spans,
                                                               p.subtract, p.d_gpart, p.d_part_auto, p.d_resid,
                                                               p.d_kx2, p.d_ky2, d_gains, d_grad);
  return cudaGetLastError();
}

}  // namespace epic
