/*
 * epic_oracle.c -- plain, slow, FP64 CPU oracle for E-field direct imaging
 * (MOFF / EPIC, Kent et al., "A Real-Time, All-Sky, High Time Resolution,
 * Direct Imager for the Long Wavelength Array").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Every function follows the paper's definition literally, in FP64, with no
 * blocking, fusion or reordering beyond what the definition states:
 *
 *   Eq. (5)  I(l,m) = < | FT{ W * E' }(l,m) |^2 >   coplanar gridded MOFF
 *   Eq. (2)  V_ab   = E_a (x) E_b^*                  FX visibilities
 *   Sec. 3.2 unpack 4+4-bit -> complex, delay calibration, gridding onto a
 *            lambda/2 grid with a user-defined illumination kernel, inverse
 *            spatial FT, square / cross-multiply, accumulate, remove autos.
 *
 * Readings of points the paper leaves open:
 *   R1 sample byte: real part in the high nibble, imaginary part in the low
 *      nibble, both 4-bit two's complement in [-8, 7].
 *   R3 transform: exp(+2 pi i (...)) as printed in Eq. (5), unnormalised.
 *   R4 pixel (i, j) <-> l = (i - N/2)/(N d), m = (j - N/2)/(N d); output rows
 *      are m, columns are l; array centre at grid cell N/2.
 *   R5 cell size d = cell_lambda wavelengths of each channel.
 *   R6 kernel: Gaussian exp(-r^2 / 2 sigma^2) sampled at cell centres over an
 *      S x S box whose origin is floor(u + 1/2) - (S-1)/2, normalised to sum 1.
 *   R7 the grid is a torus (no padding): boxes must lie inside [0, N).
 *   R8 calibration coefficient k = g * exp(-2 pi i nu tau).
 *   R9 the removed autocorrelation term is sum_a P_a |W_a(l,m)|^2 with P_a the
 *      antenna's accumulated self-power and W_a the FT of its placed kernel.
 *
 * Floating point decides no integer anywhere in this file except the grid
 * box origin floor(u + 1/2), which is taken in FP64 like the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define EO_C0 299792458.0 /* speed of light, m/s */
#define EO_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Planted-mistake switch.  Used only by tests that show the pins catch a    */
/* plausible error; 0 (the default) is the oracle as specified.              */
/* ------------------------------------------------------------------------ */
static int eo_mutation = 0;
void eo_set_mutation(int m) { eo_mutation = m; }
int eo_get_mutation(void) { return eo_mutation; }
enum {
  EO_MUT_NONE = 0,
  EO_MUT_DFT_SIGN = 1,     /* exp(-2 pi i ...) instead of exp(+2 pi i ...)   */
  EO_MUT_NO_SHIFT = 2,     /* output pixel index = raw frequency index       */
  EO_MUT_TRANSPOSE = 3,    /* output rows are l instead of m                 */
  EO_MUT_DELAY_SIGN = 4,   /* exp(+2 pi i nu tau)                            */
  EO_MUT_NO_NORM = 5,      /* kernel weights not normalised                  */
  EO_MUT_XY_CONJ = 6,      /* XY formed as Y_y conj(Y_x)                     */
  EO_MUT_DROP_LAST_T = 7,  /* last time sample not accumulated               */
  EO_MUT_AUTO_HALF = 8,    /* autocorrelation term subtracted at half weight */
  EO_MUT_NIBBLE_SWAP = 9   /* real part taken from the low nibble            */
};

typedef struct {
  int n_ant, n_pol, n_chan, grid_n, support;
  double cell_lambda;   /* grid cell in wavelengths of each channel (R5) */
  double sigma_cells;   /* Gaussian sigma in cells (R6)                  */
  const double* ant_xy; /* [n_ant][2] metres from the array centre       */
  const double* freq;   /* [n_chan] Hz                                   */
  const double* gains;  /* [n_chan][n_ant][n_pol][2] or NULL (= 1)       */
  const double* delays; /* [n_ant][n_pol] seconds or NULL (= 0)          */
} eo_array;

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: channelised data arrive as 4+4-bit complex integers and are     */
/* promoted to complex floating point.  Reading R1.                          */
/* ------------------------------------------------------------------------ */
static int eo_nibble_to_int(int nib) { return nib >= 8 ? nib - 16 : nib; }

void eo_unpack(const uint8_t* in, int64_t n, int32_t* re, int32_t* im) {
  for (int64_t k = 0; k < n; ++k) {
    int hi = (in[k] >> 4) & 15, lo = in[k] & 15;
    if (eo_mutation == EO_MUT_NIBBLE_SWAP) { int s = hi; hi = lo; lo = s; }
    re[k] = eo_nibble_to_int(hi);
    im[k] = eo_nibble_to_int(lo);
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2 / Eq. (4)-(5): antenna a of channel c on the aperture grid.      */
/* u, v: continuous cell coordinates of the antenna, array centre at N/2     */
/* (readings R4, R5).  The S x S box of the illumination kernel W starts at  */
/* (i0, j0); w[jj*S + ii] is the weight of cell (j0 + jj, i0 + ii).          */
/* Returns 0, or -1 when the box leaves the grid (reading R7).               */
/* ------------------------------------------------------------------------ */
int eo_antenna_kernel(const eo_array* d, int c, int a, double* u, double* v,
                      int* i0, int* j0, double* w) {
  const int N = d->grid_n, S = d->support;
  const double lambda = EO_C0 / d->freq[c];
  const double uu = d->ant_xy[2 * a + 0] / (lambda * d->cell_lambda) + 0.5 * N;
  const double vv = d->ant_xy[2 * a + 1] / (lambda * d->cell_lambda) + 0.5 * N;
  const int ii0 = (int)floor(uu + 0.5) - (S - 1) / 2;
  const int jj0 = (int)floor(vv + 0.5) - (S - 1) / 2;
  if (u) *u = uu;
  if (v) *v = vv;
  if (i0) *i0 = ii0;
  if (j0) *j0 = jj0;
  if (w) {
    double sum = 0.0;
    for (int jj = 0; jj < S; ++jj)
      for (int ii = 0; ii < S; ++ii) {
        double val = 1.0;
        if (S > 1) {
          const double dx = (ii0 + ii) - uu, dy = (jj0 + jj) - vv;
          val = exp(-(dx * dx + dy * dy) / (2.0 * d->sigma_cells * d->sigma_cells));
        }
        w[jj * S + ii] = val;
        sum += val;
      }
    if (eo_mutation != EO_MUT_NO_NORM)
      for (int k = 0; k < S * S; ++k) w[k] /= sum;
  }
  if (ii0 < 0 || jj0 < 0 || ii0 + S > N || jj0 + S > N) return -1;
  return 0;
}

/* Sec. 3.2 delay calibration and the gain multiply of Fig. 2: reading R8.  */
void eo_coef(const eo_array* d, int c, int a, int p, double* kr, double* ki) {
  double gr = 1.0, gi = 0.0, tau = 0.0;
  if (d->gains) {
    const int64_t o = (((int64_t)c * d->n_ant + a) * d->n_pol + p) * 2;
    gr = d->gains[o];
    gi = d->gains[o + 1];
  }
  if (d->delays) tau = d->delays[a * d->n_pol + p];
  double ph = -EO_TWO_PI * d->freq[c] * tau;
  if (eo_mutation == EO_MUT_DELAY_SIGN) ph = -ph;
  const double cr = cos(ph), ci = sin(ph);
  *kr = gr * cr - gi * ci;
  *ki = gr * ci + gi * cr;
}

/* Calibrated field e = k * (re + i im) of sample (t, c, a, p) of a
 * [T][C][A][P] byte cube. */
static void eo_field(const eo_array* d, const uint8_t* volts, int t, int c, int a, int p,
                     double kr, double ki, double* er, double* ei) {
  const int64_t idx = (((int64_t)t * d->n_chan + c) * d->n_ant + a) * d->n_pol + p;
  int32_t re, im;
  eo_unpack(volts + idx, 1, &re, &im);
  *er = kr * re - ki * im;
  *ei = kr * im + ki * re;
}

/* ------------------------------------------------------------------------ */
/* Eq. (5), inner bracket: G = W * E', the calibrated point fields of all    */
/* antennas convolved with their illumination kernels on the N x N grid.     */
/* g is [N][N][2] (row y, column x, re/im).                                  */
/* ------------------------------------------------------------------------ */
int eo_grid(const eo_array* d, const uint8_t* volts, int t, int c, int p, double* g) {
  const int N = d->grid_n, S = d->support;
  double* w = (double*)malloc(sizeof(double) * S * S);
  memset(g, 0, sizeof(double) * 2 * N * N);
  int rc = 0;
  for (int a = 0; a < d->n_ant; ++a) {
    int i0, j0;
    if (eo_antenna_kernel(d, c, a, NULL, NULL, &i0, &j0, w) != 0) { rc = -1; break; }
    double kr, ki, er, ei;
    eo_coef(d, c, a, p, &kr, &ki);
    eo_field(d, volts, t, c, a, p, kr, ki, &er, &ei);
    for (int jj = 0; jj < S; ++jj)
      for (int ii = 0; ii < S; ++ii) {
        const int64_t o = 2 * ((int64_t)(j0 + jj) * N + (i0 + ii));
        g[o] += w[jj * S + ii] * er;
        g[o + 1] += w[jj * S + ii] * ei;
      }
  }
  free(w);
  return rc;
}

/* exp(+2 pi i m / N) for m = 0..N-1: the phase of every term of Eq. (5) on
 * the grid, with the integer product reduced mod N before the cosine. */
static void eo_phase_table(int N, double* cs, double* sn) {
  const double sgn = (eo_mutation == EO_MUT_DFT_SIGN) ? -1.0 : 1.0;
  for (int m = 0; m < N; ++m) {
    cs[m] = cos(EO_TWO_PI * m / N);
    sn[m] = sgn * sin(EO_TWO_PI * m / N);
  }
}

/* Frequency index of output pixel i (reading R4: pixel i <-> i - N/2). */
static int eo_pix_freq(int N, int i) {
  return (eo_mutation == EO_MUT_NO_SHIFT) ? i : i - N / 2;
}

/* ------------------------------------------------------------------------ */
/* Eq. (5), the spatial FT written out directly (O(N^3), no FFT):           */
/*   Y[j][i] = sum_y sum_x G[y][x] exp(+2 pi i ((i-N/2) x + (j-N/2) y) / N)  */
/* taken as the x sum for every row, then the y sum for every column.        */
/* ------------------------------------------------------------------------ */
void eo_dft2(int N, const double* g, double* y) {
  double* cs = (double*)malloc(sizeof(double) * N);
  double* sn = (double*)malloc(sizeof(double) * N);
  double* z = (double*)malloc(sizeof(double) * 2 * N * N);
  eo_phase_table(N, cs, sn);
  for (int r = 0; r < N; ++r)
    for (int i = 0; i < N; ++i) {
      const int f = eo_pix_freq(N, i);
      double sr = 0.0, si = 0.0;
      for (int x = 0; x < N; ++x) {
        const int m = (int)((((int64_t)f * x) % N + N) % N);
        const double gr = g[2 * (r * N + x)], gi = g[2 * (r * N + x) + 1];
        sr += gr * cs[m] - gi * sn[m];
        si += gr * sn[m] + gi * cs[m];
      }
      z[2 * (r * N + i)] = sr;
      z[2 * (r * N + i) + 1] = si;
    }
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      const int f = eo_pix_freq(N, j);
      double sr = 0.0, si = 0.0;
      for (int r = 0; r < N; ++r) {
        const int m = (int)((((int64_t)f * r) % N + N) % N);
        const double zr = z[2 * (r * N + i)], zi = z[2 * (r * N + i) + 1];
        sr += zr * cs[m] - zi * sn[m];
        si += zr * sn[m] + zi * cs[m];
      }
      const int o = (eo_mutation == EO_MUT_TRANSPOSE) ? (i * N + j) : (j * N + i);
      y[2 * o] = sr;
      y[2 * o + 1] = si;
    }
  free(cs);
  free(sn);
  free(z);
}

/* ------------------------------------------------------------------------ */
/* The same transform through a textbook iterative radix-2 FFT (bit-reversal */
/* permutation, then log2 N butterfly passes), used by the timing mode.     */
/* N must be a power of two.  The (-1)^(x+y) factor on the input moves the   */
/* zero frequency to pixel N/2, as reading R4 asks.                          */
/* ------------------------------------------------------------------------ */
static void eo_fft1(int N, double* re, double* im, const double* cs, const double* sn) {
  for (int i = 1, j = 0; i < N; ++i) {
    int bit = N >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double tr = re[i]; re[i] = re[j]; re[j] = tr;
      double ti = im[i]; im[i] = im[j]; im[j] = ti;
    }
  }
  for (int len = 2; len <= N; len <<= 1) {
    const int step = N / len;
    for (int s = 0; s < N; s += len)
      for (int k = 0; k < len / 2; ++k) {
        const double wr = cs[k * step], wi = sn[k * step];
        const int p = s + k, q = s + k + len / 2;
        const double xr = re[q] * wr - im[q] * wi, xi = re[q] * wi + im[q] * wr;
        re[q] = re[p] - xr; im[q] = im[p] - xi;
        re[p] += xr; im[p] += xi;
      }
  }
}

void eo_fft2(int N, const double* g, double* y) {
  double* cs = (double*)malloc(sizeof(double) * N);
  double* sn = (double*)malloc(sizeof(double) * N);
  double* br = (double*)malloc(sizeof(double) * N);
  double* bi = (double*)malloc(sizeof(double) * N);
  double* z = (double*)malloc(sizeof(double) * 2 * N * N);
  eo_phase_table(N, cs, sn);
  for (int r = 0; r < N; ++r) {
    for (int x = 0; x < N; ++x) {
      const double s = ((x + r) & 1) ? -1.0 : 1.0;
      br[x] = s * g[2 * (r * N + x)];
      bi[x] = s * g[2 * (r * N + x) + 1];
    }
    eo_fft1(N, br, bi, cs, sn);
    for (int i = 0; i < N; ++i) { z[2 * (r * N + i)] = br[i]; z[2 * (r * N + i) + 1] = bi[i]; }
  }
  for (int i = 0; i < N; ++i) {
    for (int r = 0; r < N; ++r) { br[r] = z[2 * (r * N + i)]; bi[r] = z[2 * (r * N + i) + 1]; }
    eo_fft1(N, br, bi, cs, sn);
    for (int j = 0; j < N; ++j) { y[2 * (j * N + i)] = br[j]; y[2 * (j * N + i) + 1] = bi[j]; }
  }
  free(cs); free(sn); free(br); free(bi); free(z);
}

/* ------------------------------------------------------------------------ */
/* |W_a(l,m)|^2 of antenna a in channel c on every output pixel: the FT of   */
/* its placed S x S kernel, written out as the direct sum over the box.     */
/* out is [N][N].                                                            */
/* ------------------------------------------------------------------------ */
static void eo_kernel_ft(const eo_array* d, int c, int a, double* wre, double* wim) {
  const int N = d->grid_n, S = d->support;
  double* w = (double*)malloc(sizeof(double) * S * S);
  double* cs = (double*)malloc(sizeof(double) * N);
  double* sn = (double*)malloc(sizeof(double) * N);
  int i0, j0;
  eo_antenna_kernel(d, c, a, NULL, NULL, &i0, &j0, w);
  eo_phase_table(N, cs, sn);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      const int fi = eo_pix_freq(N, i), fj = eo_pix_freq(N, j);
      double sr = 0.0, si = 0.0;
      for (int jj = 0; jj < S; ++jj)
        for (int ii = 0; ii < S; ++ii) {
          const int64_t ph = (int64_t)fi * (i0 + ii) + (int64_t)fj * (j0 + jj);
          const int m = (int)((ph % N + N) % N);
          sr += w[jj * S + ii] * cs[m];
          si += w[jj * S + ii] * sn[m];
        }
      const int o = (eo_mutation == EO_MUT_TRANSPOSE) ? (i * N + j) : (j * N + i);
      wre[o] = sr;
      wim[o] = si;
    }
  free(w); free(cs); free(sn);
}

void eo_kernel_power(const eo_array* d, int c, int a, double* out) {
  const int N = d->grid_n;
  double* wr = (double*)malloc(sizeof(double) * N * N);
  double* wi = (double*)malloc(sizeof(double) * N * N);
  eo_kernel_ft(d, c, a, wr, wi);
  for (int k = 0; k < N * N; ++k) out[k] = wr[k] * wr[k] + wi[k] * wi[k];
  free(wr); free(wi);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1 and Sec. 3.2: the accumulated EPIC image of channels             */
/* [c_lo, c_hi) over the T samples of a [T][C][A][P] byte cube.              */
/*   out   [c_hi-c_lo][4][N][N]: XX, YY, Re XY, Im XY; planes 1-3 are zero   */
/*         for one polarisation.  Per pixel: XX = sum_t |Y_X|^2,             */
/*         YY = sum_t |Y_Y|^2, XY = sum_t Y_X conj(Y_Y).                     */
/*   autos [c_hi-c_lo][A][3][2] or NULL: P_a for XX, YY, XY (reading R9).    */
/* subtract != 0 removes sum_a P_a |W_a|^2 from every plane (Sec. 3.2, last  */
/* paragraph; reading R9).  use_fft != 0 takes eo_fft2 instead of eo_dft2.   */
/* Channels are independent; they are shared among n_threads OpenMP threads, */
/* each channel summed in time order, so the result does not depend on the   */
/* thread count.  Returns 0, or -1 when an antenna box leaves the grid.      */
/* ------------------------------------------------------------------------ */
int eo_image(const eo_array* d, const uint8_t* volts, int T, int c_lo, int c_hi,
             int subtract, int use_fft, int n_threads, double* out, double* autos) {
  const int N = d->grid_n, A = d->n_ant, P = d->n_pol;
  const int NN = N * N;
  int rc = 0;
  const int n_c = c_hi - c_lo;
  for (int c = c_lo; c < c_hi; ++c)
    for (int a = 0; a < A; ++a)
      if (eo_antenna_kernel(d, c, a, NULL, NULL, NULL, NULL, NULL) != 0) return -1;
  const int T_used = (eo_mutation == EO_MUT_DROP_LAST_T && T > 0) ? T - 1 : T;
#ifdef _OPENMP
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int cc = 0; cc < n_c; ++cc) {
    const int c = c_lo + cc;
    double* img = out + (int64_t)cc * 4 * NN;
    double* g = (double*)malloc(sizeof(double) * 2 * NN);
    double* y[2];
    y[0] = (double*)malloc(sizeof(double) * 2 * NN);
    y[1] = (double*)malloc(sizeof(double) * 2 * NN);
    double* pw = (double*)calloc((size_t)A * 6, sizeof(double));
    double* kc = (double*)malloc(sizeof(double) * A * P * 2);
    memset(img, 0, sizeof(double) * 4 * NN);
    for (int a = 0; a < A; ++a)
      for (int p = 0; p < P; ++p) eo_coef(d, c, a, p, &kc[2 * (a * P + p)], &kc[2 * (a * P + p) + 1]);
    for (int t = 0; t < T_used; ++t) {
      for (int p = 0; p < P; ++p) {
        eo_grid(d, volts, t, c, p, g);
        if (use_fft) eo_fft2(N, g, y[p]); else eo_dft2(N, g, y[p]);
      }
      for (int k = 0; k < NN; ++k) {
        const double xr = y[0][2 * k], xi = y[0][2 * k + 1];
        img[k] += xr * xr + xi * xi;
        if (P == 2) {
          const double yr = y[1][2 * k], yi = y[1][2 * k + 1];
          img[NN + k] += yr * yr + yi * yi;
          if (eo_mutation == EO_MUT_XY_CONJ) {
            img[2 * NN + k] += yr * xr + yi * xi;
            img[3 * NN + k] += yi * xr - yr * xi;
          } else {
            img[2 * NN + k] += xr * yr + xi * yi;
            img[3 * NN + k] += xi * yr - xr * yi;
          }
        }
      }
      /* Fig. 2 "Accumulate Autocorrelations": per-antenna self power. */
      for (int a = 0; a < A; ++a) {
        double er[2] = {0, 0}, ei[2] = {0, 0};
        for (int p = 0; p < P; ++p)
          eo_field(d, volts, t, c, a, p, kc[2 * (a * P + p)], kc[2 * (a * P + p) + 1], &er[p], &ei[p]);
        pw[6 * a + 0] += er[0] * er[0] + ei[0] * ei[0];
        if (P == 2) {
          pw[6 * a + 2] += er[1] * er[1] + ei[1] * ei[1];
          pw[6 * a + 4] += er[0] * er[1] + ei[0] * ei[1];
          pw[6 * a + 5] += ei[0] * er[1] - er[0] * ei[1];
        }
      }
    }
    if (autos) memcpy(autos + (int64_t)cc * A * 6, pw, sizeof(double) * A * 6);
    if (subtract) {
      /* Fig. 2 "Remove Autocorrelations" (reading R9). */
      double* wp = (double*)malloc(sizeof(double) * NN);
      const double f = (eo_mutation == EO_MUT_AUTO_HALF) ? 0.5 : 1.0;
      for (int a = 0; a < A; ++a) {
        eo_kernel_power(d, c, a, wp);
        for (int k = 0; k < NN; ++k) {
          img[k] -= f * pw[6 * a + 0] * wp[k];
          if (P == 2) {
            img[NN + k] -= f * pw[6 * a + 2] * wp[k];
            img[2 * NN + k] -= f * pw[6 * a + 4] * wp[k];
            img[3 * NN + k] -= f * pw[6 * a + 5] * wp[k];
          }
        }
      }
      free(wp);
    }
    free(g); free(y[0]); free(y[1]); free(pw); free(kc);
  }
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Eq. (2): FX visibilities of channel c, V[pq][a][b] = sum_t e_ap conj(e_bq)*/
/* for pq in {XX, YY, XY}; v is [3][A][A][2] (YY, XY zero for one pol).      */
/* ------------------------------------------------------------------------ */
void eo_visibilities(const eo_array* d, const uint8_t* volts, int T, int c, double* v) {
  const int A = d->n_ant, P = d->n_pol;
  double* er = (double*)malloc(sizeof(double) * A * P);
  double* ei = (double*)malloc(sizeof(double) * A * P);
  memset(v, 0, sizeof(double) * 3 * A * A * 2);
  const int T_used = (eo_mutation == EO_MUT_DROP_LAST_T && T > 0) ? T - 1 : T;
  for (int t = 0; t < T_used; ++t) {
    for (int a = 0; a < A; ++a)
      for (int p = 0; p < P; ++p) {
        double kr, ki;
        eo_coef(d, c, a, p, &kr, &ki);
        eo_field(d, volts, t, c, a, p, kr, ki, &er[a * P + p], &ei[a * P + p]);
      }
    for (int pq = 0; pq < (P == 2 ? 3 : 1); ++pq) {
      const int p = (pq == 1) ? 1 : 0, q = (pq == 0) ? 0 : 1;
      for (int a = 0; a < A; ++a)
        for (int b = 0; b < A; ++b) {
          const double ar = er[a * P + p], ai = ei[a * P + p];
          const double br = er[b * P + q], bi = ei[b * P + q];
          double* o = v + 2 * (((int64_t)pq * A + a) * A + b);
          o[0] += ar * br + ai * bi;
          o[1] += ai * br - ar * bi;
        }
    }
  }
  free(er); free(ei);
}

/* ------------------------------------------------------------------------ */
/* Brute-force FX image of channel c from Eq. (2) and the convolution        */
/* theorem: I_pq(pix) = sum_{a,b} V_ab,pq W_a(pix) conj(W_b(pix)), with      */
/* W_a the FT of antenna a's placed kernel.  include_autos = 0 drops a == b. */
/* out is [4][N][N] in the same plane order as eo_image.  O(A^2 N^2).        */
/* ------------------------------------------------------------------------ */
int eo_fx_brute(const eo_array* d, const uint8_t* volts, int T, int c, int include_autos, double* out) {
  const int N = d->grid_n, A = d->n_ant, P = d->n_pol, NN = N * N;
  for (int a = 0; a < A; ++a)
    if (eo_antenna_kernel(d, c, a, NULL, NULL, NULL, NULL, NULL) != 0) return -1;
  double* v = (double*)malloc(sizeof(double) * 3 * A * A * 2);
  double* wr = (double*)malloc(sizeof(double) * (int64_t)A * NN);
  double* wi = (double*)malloc(sizeof(double) * (int64_t)A * NN);
  eo_visibilities(d, volts, T, c, v);
  for (int a = 0; a < A; ++a) eo_kernel_ft(d, c, a, wr + (int64_t)a * NN, wi + (int64_t)a * NN);
  memset(out, 0, sizeof(double) * 4 * NN);
  for (int pq = 0; pq < (P == 2 ? 3 : 1); ++pq)
    for (int k = 0; k < NN; ++k) {
      double sr = 0.0, si = 0.0;
      for (int a = 0; a < A; ++a)
        for (int b = 0; b < A; ++b) {
          if (!include_autos && a == b) continue;
          const double* vv = v + 2 * (((int64_t)pq * A + a) * A + b);
          /* V * W_a * conj(W_b) */
          const double ar = wr[(int64_t)a * NN + k], ai = wi[(int64_t)a * NN + k];
          const double br = wr[(int64_t)b * NN + k], bi = -wi[(int64_t)b * NN + k];
          const double mr = ar * br - ai * bi, mi = ar * bi + ai * br;
          sr += vv[0] * mr - vv[1] * mi;
          si += vv[0] * mi + vv[1] * mr;
        }
      if (pq < 2) {
        out[pq * NN + k] = sr;  /* XX, YY are real */
      } else {
        out[2 * NN + k] = sr;
        out[3 * NN + k] = si;
      }
    }
  free(v); free(wr); free(wi);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gridded FX image of channel c: every visibility V_ab is gridded at its    */
/* baseline with the cross-correlation of the two antennas' kernels,         */
/* (W_a star W_b)[d] = sum_x W_a[x + d] W_b[x] on the N x N torus (reading   */
/* R7), and the visibility grid is transformed once with eo_dft2.            */
/* include_autos = 0 drops a == b.  out is [4][N][N].  O(A^2 S^4 + N^3).     */
/* ------------------------------------------------------------------------ */
int eo_fx_gridded(const eo_array* d, const uint8_t* volts, int T, int c, int include_autos, double* out) {
  const int N = d->grid_n, A = d->n_ant, P = d->n_pol, S = d->support, NN = N * N;
  double* w = (double*)malloc(sizeof(double) * (int64_t)A * S * S);
  int* i0 = (int*)malloc(sizeof(int) * A);
  int* j0 = (int*)malloc(sizeof(int) * A);
  for (int a = 0; a < A; ++a)
    if (eo_antenna_kernel(d, c, a, NULL, NULL, &i0[a], &j0[a], w + (int64_t)a * S * S) != 0) {
      free(w); free(i0); free(j0);
      return -1;
    }
  double* v = (double*)malloc(sizeof(double) * 3 * A * A * 2);
  double* vg = (double*)malloc(sizeof(double) * 2 * NN);
  double* y = (double*)malloc(sizeof(double) * 2 * NN);
  eo_visibilities(d, volts, T, c, v);
  memset(out, 0, sizeof(double) * 4 * NN);
  for (int pq = 0; pq < (P == 2 ? 3 : 1); ++pq) {
    memset(vg, 0, sizeof(double) * 2 * NN);
    for (int a = 0; a < A; ++a)
      for (int b = 0; b < A; ++b) {
        if (!include_autos && a == b) continue;
        const double* vv = v + 2 * (((int64_t)pq * A + a) * A + b);
        for (int ja = 0; ja < S; ++ja)
          for (int ia = 0; ia < S; ++ia)
            for (int jb = 0; jb < S; ++jb)
              for (int ib = 0; ib < S; ++ib) {
                /* lag d = (cell of a) - (cell of b), mod N */
                const int dx = (((i0[a] + ia) - (i0[b] + ib)) % N + N) % N;
                const int dy = (((j0[a] + ja) - (j0[b] + jb)) % N + N) % N;
                const double ww = w[(int64_t)a * S * S + ja * S + ia] * w[(int64_t)b * S * S + jb * S + ib];
                vg[2 * (dy * N + dx)] += ww * vv[0];
                vg[2 * (dy * N + dx) + 1] += ww * vv[1];
              }
      }
    eo_dft2(N, vg, y);
    for (int k = 0; k < NN; ++k) {
      if (pq < 2) {
        out[pq * NN + k] = y[2 * k];
      } else {
        out[2 * NN + k] = y[2 * k];
        out[3 * NN + k] = y[2 * k + 1];
      }
    }
  }
  free(w); free(i0); free(j0); free(v); free(vg); free(y);
  return 0;
}

int eo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gradient of the image-plane calibration loss with respect to the complex  */
/* gains (the gain multiplication of Fig. 2, solved for by the EPICal block  */
/* the paper plans in Sec. 6):                                               */
/*   L = sum_c sum_{pp in XX, YY} sum_pix (I_pp - M_pp)^2,                   */
/* with I the autocorrelation-removed image.  From the FX form (Eq. (2)),    */
/*   I_pp = sum_{a != b} g_ap conj(g_bp) V~_ab W_a conj(W_b),                */
/* V~_ab = sum_t e~_a conj(e~_b) the visibilities without gains (e~ carries  */
/* the delay phase only), W_a the FT of antenna a's placed kernel.  Hence    */
/*   dL/d conj(g_cp) = sum_pix R_pp sum_{a != c} g_ap V~_ac W_a conj(W_c),   */
/* R = 2 (I - M), and the gradient in the convention dL/dRe g + i dL/dIm g   */
/* is twice that.  model is [C][2][N][N] (XX, YY); grad [C][A][P][2]; loss a */
/* scalar.  O(A^2 N^2) per channel and polarisation: small cases only.       */
/* ------------------------------------------------------------------------ */
int eo_grad_fx(const eo_array* d, const uint8_t* volts, int T, const double* model, double* grad, double* loss) {
  const int N = d->grid_n, A = d->n_ant, P = d->n_pol, C = d->n_chan, NN = N * N;
  if (A > 1024) return -2;
  eo_array dn = *d;
  dn.gains = NULL;  /* visibilities without gains: delay phase only */
  double* v = (double*)malloc(sizeof(double) * 3 * A * A * 2);
  double* wr = (double*)malloc(sizeof(double) * (int64_t)A * NN);
  double* wi = (double*)malloc(sizeof(double) * (int64_t)A * NN);
  double* img = (double*)malloc(sizeof(double) * NN);
  double total = 0.0;
  memset(grad, 0, sizeof(double) * (size_t)C * A * P * 2);
  for (int c = 0; c < C; ++c) {
    for (int a = 0; a < A; ++a)
      if (eo_antenna_kernel(d, c, a, NULL, NULL, NULL, NULL, NULL) != 0) {
        free(v); free(wr); free(wi); free(img);
        return -1;
      }
    eo_visibilities(&dn, volts, T, c, v);
    for (int a = 0; a < A; ++a) eo_kernel_ft(d, c, a, wr + (int64_t)a * NN, wi + (int64_t)a * NN);
    for (int p = 0; p < P; ++p) {
      const int pq = p;  /* XX for p = 0, YY for p = 1 */
      double gr[1024], gi[1024];
      for (int a = 0; a < A && a < 1024; ++a) {
        gr[a] = 1.0; gi[a] = 0.0;
        if (d->gains) {
          gr[a] = d->gains[2 * (((int64_t)c * A + a) * P + p)];
          gi[a] = d->gains[2 * (((int64_t)c * A + a) * P + p) + 1];
        }
      }
      /* I_pp over the pixels */
      for (int k = 0; k < NN; ++k) {
        double s = 0.0;
        for (int a = 0; a < A; ++a)
          for (int b = 0; b < A; ++b) {
            if (a == b) continue;
            const double* vv = v + 2 * (((int64_t)pq * A + a) * A + b);
            /* g_a conj(g_b) */
            const double qr = gr[a] * gr[b] + gi[a] * gi[b], qi = gi[a] * gr[b] - gr[a] * gi[b];
            /* W_a conj(W_b) */
            const double ar = wr[(int64_t)a * NN + k], ai = wi[(int64_t)a * NN + k];
            const double br = wr[(int64_t)b * NN + k], bi = -wi[(int64_t)b * NN + k];
            const double mr = ar * br - ai * bi, mi = ar * bi + ai * br;
            const double tr = qr * vv[0] - qi * vv[1], ti = qr * vv[1] + qi * vv[0];
            s += tr * mr - ti * mi;  /* real part; the imaginary parts cancel over (a, b), (b, a) */
          }
        img[k] = s;
      }
      const double* M = model + ((int64_t)c * 2 + pq) * NN;
      for (int k = 0; k < NN; ++k) total += (img[k] - M[k]) * (img[k] - M[k]);
      /* gradient */
      for (int cc = 0; cc < A; ++cc) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < NN; ++k) {
          const double R = 2.0 * (img[k] - M[k]);
          double ur = 0.0, ui = 0.0;  /* sum_{a != cc} g_a V~_{a cc} W_a */
          for (int a = 0; a < A; ++a) {
            if (a == cc) continue;
            const double* vv = v + 2 * (((int64_t)pq * A + a) * A + cc);
            const double tr = gr[a] * vv[0] - gi[a] * vv[1], ti = gr[a] * vv[1] + gi[a] * vv[0];
            const double ar = wr[(int64_t)a * NN + k], ai = wi[(int64_t)a * NN + k];
            ur += tr * ar - ti * ai;
            ui += tr * ai + ti * ar;
          }
          /* times conj(W_cc) */
          const double cr = wr[(int64_t)cc * NN + k], ci = -wi[(int64_t)cc * NN + k];
          sr += R * (ur * cr - ui * ci);
          si += R * (ur * ci + ui * cr);
        }
        double* o = grad + 2 * (((int64_t)c * A + cc) * P + p);
        o[0] = 2.0 * sr;
        o[1] = 2.0 * si;
      }
    }
  }
  *loss = total;
  free(v); free(wr); free(wi); free(img);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Post-processing (Sec. 3.2 last paragraph; Sec. 4.3).                      */
/* eo_beam: image of the illumination kernels of channel c, the mean over    */
/* antennas of |W_a(l,m)|^2 ([N][N]).                                        */
/* eo_stokes: pseudo-Stokes planes of linear feeds from [4][N][N] XX, YY,    */
/* Re XY, Im XY: I = XX + YY, Q = XX - YY, U = XY + YX, V = -i (XY - YX),    */
/* with YX = conj(XY).                                                       */
/* ------------------------------------------------------------------------ */
void eo_beam(const eo_array* d, int c, double* beam) {
  const int NN = d->grid_n * d->grid_n;
  double* wp = (double*)malloc(sizeof(double) * NN);
  memset(beam, 0, sizeof(double) * NN);
  for (int a = 0; a < d->n_ant; ++a) {
    eo_kernel_power(d, c, a, wp);
    for (int k = 0; k < NN; ++k) beam[k] += wp[k];
  }
  for (int k = 0; k < NN; ++k) beam[k] /= d->n_ant;
  free(wp);
}

void eo_stokes(int NN, const double* in, double* out) {
  for (int k = 0; k < NN; ++k) {
    const double xx = in[k], yy = in[NN + k], xyr = in[2 * NN + k], xyi = in[3 * NN + k];
    /* YX = conj(XY): XY + YX = 2 Re XY; -i (XY - YX) = -i (2 i Im XY) = 2 Im XY */
    out[k] = xx + yy;
    out[NN + k] = xx - yy;
    out[2 * NN + k] = 2.0 * xyr;
    out[3 * NN + k] = 2.0 * xyi;
  }
}
