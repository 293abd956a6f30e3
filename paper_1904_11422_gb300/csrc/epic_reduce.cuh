// epic_reduce.cuh -- the block end of an imaging call (Fig. 2 "Remove
// Autocorrelations") for one (virtual) channel and a range of its rows, as a
// device function: run by the reduction kernel (one CTA per piece) and by the
// persistent batch kernel of the tensor-core path (one claimed item per piece),
// with the same arithmetic in the same order, so both give the same bits.
//
// Sums the per-CTA partial images of the channel in CTA order, subtracts the
// autocorrelation term sum_a P_a |W_a(l,m)|^2 (reading R9: P_a the antenna's self
// power over the block -- exact integer sums times |k|^2, or k_X conj(k_Y) for
// XY, formed in FP64 -- and |W_a|^2 = |FT w_x|^2 (column) x |FT w_y|^2 (row) of
// its separable kernel) and writes or accumulates the output pixels.
#pragma once

#include "epic_internal.cuh"

namespace epic {

// Rows [j0, j0 + rows) of virtual channel cv, by threads tid of nthreads (all of
// which call it); smem holds A float4 + A x rows floats.  With vq = 4 (128 x 128
// grids folded into four 64 x 64 problems) the partials are the sub-images of
// virtual channels 4 c + q, and pixel (j, i) of sub-image q lands on output pixel
// (2 j + beta, 2 i + alpha), alpha = q & 1, beta = q >> 1.  With dec = 2 (the
// tensor path on 32 x 32 grids) the partials are 64 x 64 and output pixel (j, i)
// is their pixel (2 j, 2 i).  Partials are read from L2 (they may have been
// written by other CTAs of the same launch).
template <int P, int kReducePix>
__device__ __forceinline__ void reduce_rows(const ReduceArgs& r, int cv, int j0, int rows, int tid, int nthreads,
                                            unsigned char* smem) {
  float4* Pw = reinterpret_cast<float4*>(smem);      // [A] self powers XX, YY, Re XY, Im XY
  float* kys = reinterpret_cast<float*>(Pw + r.A);   // [A][rows] |FT w_y|^2 of the rows
  const int A = r.A, N = r.N, vq = r.vq, dec = r.dec;
  const int c = vq == 4 ? cv >> 2 : cv;               // output channel
  const int alpha = vq == 4 ? (cv & 1) : 0, beta = vq == 4 ? (cv >> 1) & 1 : 0;
  const int Ns = vq == 4 ? N / 2 : N * dec;           // side of a partial image
  const int L = vq == 4 ? Ns : N;                     // side of the pixel loop
  const int NN = N * N, NNs = Ns * Ns;
  auto orow = [&](int j) { return vq == 4 ? 2 * j + beta : j; };
  auto ocol = [&](int i) { return vq == 4 ? 2 * i + alpha : i; };
  const long long W = r.W, T = r.T;
  const long long b_lo = ((long long)cv * T) / W;
  const long long b_hi = min(((long long)(cv + 1) * T - 1) / W, (long long)r.ctas - 1);
  // CTA b's first channel floor(b W / T) (its partials' slot 0), stepped over b
  // from b_lo with additions only: b W = q T + rem
  const long long q_lo = (b_lo * W) / T, rem_lo = b_lo * W - q_lo * T, wq = W / T, wr = W - wq * T;
  auto next_b = [&](long long& q, long long& rem) {
    rem += wr;
    q += wq;
    if (rem >= T) {
      rem -= T;
      ++q;
    }
  };

  if (r.subtract) {
    for (int a = tid; a < A; a += nthreads) {
      long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      long long q = q_lo, rem = rem_lo;
      for (long long b = b_lo; b <= b_hi; ++b, next_b(q, rem)) {
        const int slot = cv - (int)q;
        const int4 v = __ldcg(reinterpret_cast<const int4*>(r.part_auto) + (b * r.spans + slot) * A + a);
        s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
      }
      const double2 kx = r.coef64[((size_t)c * A + a) * P];
      float4 pw = make_float4((float)((kx.x * kx.x + kx.y * kx.y) * (double)s0), 0.f, 0.f, 0.f);
      if (P == 2) {
        const double2 ky = r.coef64[((size_t)c * A + a) * P + 1];
        const double mr = kx.x * ky.x + kx.y * ky.y, mi = kx.y * ky.x - kx.x * ky.y;  // k_X conj(k_Y)
        pw.y = (float)((ky.x * ky.x + ky.y * ky.y) * (double)s1);
        pw.z = (float)(mr * (double)s2 - mi * (double)s3);
        pw.w = (float)(mr * (double)s3 + mi * (double)s2);
      }
      Pw[a] = pw;
      for (int jj = 0; jj < rows; ++jj) kys[a * rows + jj] = r.ky2[((size_t)c * A + a) * N + orow(j0 + jj)];
    }
    __syncthreads();
  }

  // each thread takes kReducePix consecutive pixels of one row (L is a multiple),
  // which share the per-antenna loads of P_a and |FT w_y|^2; every pixel's sums
  // run over CTAs, then antennas, in order, whatever kReducePix is
  for (int q0 = tid * kReducePix; q0 < rows * L; q0 += nthreads * kReducePix) {
    const int jj = q0 / L, i0 = q0 % L;
    float s[kReducePix][4];
#pragma unroll
    for (int e = 0; e < kReducePix; ++e) {
      const int pix = dec * (j0 + jj) * Ns + dec * (i0 + e);
      s[e][0] = s[e][1] = s[e][2] = s[e][3] = 0.f;
      long long q = q_lo, rem = rem_lo;
      for (long long b = b_lo; b <= b_hi; ++b, next_b(q, rem)) {
        const int slot = cv - (int)q;
        const float* src = r.part + (size_t)(b * r.spans + slot) * 4 * NNs + pix;
        s[e][0] += __ldcg(src);
        if (P == 2) {
          s[e][1] += __ldcg(src + NNs);
          s[e][2] += __ldcg(src + 2 * NNs);
          s[e][3] += __ldcg(src + 3 * NNs);
        }
      }
    }
    if (r.subtract) {
      float acc[kReducePix][4];
#pragma unroll
      for (int e = 0; e < kReducePix; ++e) acc[e][0] = acc[e][1] = acc[e][2] = acc[e][3] = 0.f;
      const float* kxc = r.kx2 + (size_t)c * A * N;
      for (int a = 0; a < A; ++a) {
        const float ky = kys[a * rows + jj];
        const float4 pw = Pw[a];
#pragma unroll
        for (int e = 0; e < kReducePix; ++e) {
          const float w2 = kxc[(size_t)a * N + ocol(i0 + e)] * ky;
          acc[e][0] = fmaf(pw.x, w2, acc[e][0]);
          if (P == 2) {
            acc[e][1] = fmaf(pw.y, w2, acc[e][1]);
            acc[e][2] = fmaf(pw.z, w2, acc[e][2]);
            acc[e][3] = fmaf(pw.w, w2, acc[e][3]);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < kReducePix; ++e)
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) s[e][pl] -= acc[e][pl];
    }
#pragma unroll
    for (int e = 0; e < kReducePix; ++e) {
      float* o = r.out + (size_t)c * 4 * NN + orow(j0 + jj) * N + ocol(i0 + e);
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) o[pl * NN] = r.accumulate ? o[pl * NN] + s[e][pl] : s[e][pl];
    }
  }
}

// Rows of the pixel loop per reduction piece: pieces of at least `min_pixels`
// pixels (whole rows; the loop side L is N, or N/2 for folded grids), fewer when
// the staging of A antennas (A float4 + A x rows floats) would exceed smem_cap.
__host__ __device__ inline int reduce_rows_per_piece(int L, int min_pixels, int A, size_t smem_cap) {
  int rows = 1;
  while (rows * L < min_pixels && rows < L) rows *= 2;
  while (rows > 1 && (size_t)A * (16 + 4 * (size_t)rows) > smem_cap) rows /= 2;
  return rows;
}

}  // namespace epic
