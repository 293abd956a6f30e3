// epic_dft.cu -- the tensor-core imaging path: the 2-D transform of Eq. (5) as
// two dense real GEMMs on tcgen05, fused with unpack, gridding, squaring and
// accumulation in one kernel per imaging call.
//
// With F[k][x] = exp(+2 pi i (k - N/2) x / N) (the pixel shift of reading R4
// folded into the rows), one (t, c) image set is Y_g = F G_g F^T for the two
// polarisation grids g.  Each complex product is one real GEMM with the 2N x 2N
// matrix Fre = [[Fr, -Fi], [Fi, Fr]] (rows interleaved re/im by eights) as the A operand:
//   stage 1 (along x): D1[(k,c)][(g,y)] = sum_(c',x) Fre[(k,c)][(c',x)] G[(g,y)][(c',x)]
//   stage 2 (along y): D2[(j,c)][(g,k)] = sum_(c',y) Fre[(j,c)][(c',y)] Z[(g,k)][(c',y)]
// where Z[(g,k)][(c,y)] = D1[(k,c)][(g,y)] is moved from tensor memory to shared
// memory (each thread holds 32 consecutive y of one row, so the transposition
// costs only 16-byte stores).  At N = 64 both stages are M = N = K = 128 GEMMs:
// Fre lives in tensor memory for the whole launch (A operand), the gridded
// fields and Z are K-major 128-byte-swizzled shared-memory B operands, and the
// FP32 accumulators are in tensor memory.  The operands are split into a high
// and a low 16-bit part (BF16 or FP16) and three products hi.hi + lo.hi + hi.lo
// are accumulated (the "x3" transforms), or only the high parts are used.
//
// The transform is always the 64-point one: a 128 x 128 grid runs as four 64 x 64
// problems of parity-folded fields (see Q128 below), a 32 x 32 grid as the 64 x 64
// transform of the zero-padded grid whose even output pixels are kept (done by
// the gather tables and the reduction; the kernel is the same).
//
// The samples of a CTA are software-pipelined: the stage-2 products of sample t
// run while sample t+1 is gridded, the stage-1 products of t+1 run while sample t
// is squared and accumulated, and sample t+2's fields are unpacked while stage 1
// of t+1 runs.
//
// One elected thread issues the MMAs and commits them to mbarriers; every wait
// on them is bounded (about one second) and reports EPIC_ERR_TIMEOUT through the
// plan's status word instead of hanging.
#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>

#include "epic_internal.cuh"
#include "epic_ptx.cuh"
#include "epic_reduce.cuh"

namespace epic {

namespace {

using namespace ptx;

constexpr int kN = 64;               // grid side of this kernel
constexpr int kThreads = 512;        // 16 warps
constexpr int kSlab = 128 * 128;     // one 128-row x 64-element 16-bit operand slab, bytes
constexpr unsigned long long kWaitNs = 1000000000ull;  // bounded waits: one second
// FP16 operands: power-of-two scales keep every 16-bit value below 2^15
// (FP16 overflows at 65 504) and the DFT matrix's low parts out of the
// subnormal range; the scales are exact and undone in FP32 (see dft_scale_kernel).
constexpr int kFp16MatExp = 12;      // the FP16 DFT matrix holds 2^12 F
constexpr int kFp16TopExp = 15;      // gridded fields and stage-1 results scaled below 2^15

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// Waits until the counter at p reaches `expected` (acquire at GPU scope, so the
// writes that preceded each increment are visible); false after limit_ns.
__device__ __forceinline__ bool wait_count_bounded(const int* p, int expected, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= expected) return true;
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(256);
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}


// Shared-memory matrix descriptor, K-major operand with the 128-byte swizzle:
// 8-row x 128-byte atoms (1024 B) stacked along M/N (stride 1024 B).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;             // leading-dimension offset (unused by this layout)
  d |= (uint64_t)(1024u >> 4) << 32;   // stride between 8-row groups
  d |= (uint64_t)1u << 46;             // descriptor version for tcgen05
  d |= (uint64_t)2u << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B K-major, M = N = 128.
template <bool kBf16>
__host__ __device__ constexpr uint32_t idesc_m128n128() {
  return (1u << 4) | ((kBf16 ? 1u : 0u) << 7) | ((kBf16 ? 1u : 0u) << 10) | ((128u >> 3) << 17) |
         ((128u >> 4) << 24);
}

// Byte offset of element (row r, k in [0,64)) inside a 128-row swizzled slab.
__host__ __device__ __forceinline__ uint32_t slab_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

// 16-bit operand type of a transform and its hi/lo split.
template <int XF> struct Prec;
template <> struct Prec<EPIC_XFORM_DFT_BF16X3> {
  using T = __nv_bfloat16;
  static constexpr bool kBf16 = true, kSplit = true;
};
template <> struct Prec<EPIC_XFORM_DFT_FP16X3> {
  using T = __half;
  static constexpr bool kBf16 = false, kSplit = true;
};
template <> struct Prec<EPIC_XFORM_DFT_BF16> {
  using T = __nv_bfloat16;
  static constexpr bool kBf16 = true, kSplit = false;
};
template <> struct Prec<EPIC_XFORM_DFT_FP16> {
  using T = __half;
  static constexpr bool kBf16 = false, kSplit = false;
};

template <bool kBf16>
__device__ __forceinline__ unsigned short to16(float v) {
  if constexpr (kBf16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  else return __half_as_ushort(__float2half_rn(v));
}
template <bool kBf16>
__device__ __forceinline__ float from16(unsigned short h) {
  if constexpr (kBf16) return __bfloat162float(__ushort_as_bfloat16(h));
  else return __half2float(__ushort_as_half(h));
}


// MMA with the A operand read from tensor memory (K-major rows in TMEM lanes,
// two 16-bit K elements per 32-bit column) and B from shared memory.
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Two floats to a packed pair of 16-bit values (low half = first) and back.
template <bool kBf16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (kBf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}
template <bool kBf16>
__device__ __forceinline__ float2 unpack2(uint32_t u) {
  if constexpr (kBf16) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
  else return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

// TMEM columns (512 allocated): the DFT matrix as A operand (hi, lo), the
// stage-1 accumulator D1 and two stage-2 accumulators D2 (double-buffered so the
// squaring of one sample overlaps the stage-2 products of the next).
constexpr uint32_t kColFhi = 0, kColFlo = 64, kColD1 = 128, kColD2 = 256;

// Shared memory (offsets from a 1024-byte aligned base).
struct DftSmem {
  static constexpr uint32_t B1 = 0;          // gridded fields, rows (g, y), K = (c', x): hi re, hi im, lo re, lo im
  static constexpr uint32_t B2 = 4 * kSlab;  // stage-1 result, rows (g, k), K = (c', y): same four slabs
  static constexpr uint32_t E = 8 * kSlab;   // [A] float4 calibrated fields, then coefficients, self powers, entries
};

// Q128: a 128 x 128 grid, transformed as four 64 x 64 problems.  With the
// output pixel (row 2 j + beta, column 2 k + alpha), one radix-2 step along each
// axis gives Y_128[2j+beta][2k+alpha] = (F_64 H_q F_64^T)[j][k] for
//   H_q[y][x] = exp(+2 pi i (alpha x + beta y) / 128)
//               sum_{u,s in {0,1}} (-1)^(alpha s + beta u) G[y + 64 u][x + 64 s],
// q = alpha + 2 beta.  The kernel runs virtual channels 4 c + q: the gather
// tables of virtual channel 4 c + q fold the four quadrants with signed weights
// (layout kLayoutPairQ), the twiddle is applied to each gathered cell, and the
// rest of the path is the 64 x 64 transform; the reduction interleaves the four
// sub-images.
// kBatch = false: one call of one plan, CTA b imaging span b of job0 (Q128 as
// the plan's grid says).  kBatch = true: a persistent launch whose CTAs claim
// the items of queue (spans of several plans' calls, 32 x 32, 64 x 64 and
// 128 x 128 grids alike; Q128 is then read from each job) until none is left.
// A_lay and max_entries size the shared-memory layout: the most antennas, and
// the most gather entries held in shared memory, of any job.
template <int XF, bool Q128, bool kBatch>
__global__ void __launch_bounds__(kThreads, 1)
    dft_image_kernel(const __grid_constant__ DftJob job0, const __grid_constant__ DftQueue queue, int A_lay,
                     int max_entries,
                     const uint32_t* __restrict__ fmat, const float2* __restrict__ twiddle,
                     unsigned long long test_wait_ns) {
  using Pr = Prec<XF>;
  constexpr bool kBf = Pr::kBf16;
  constexpr int NN = kN * kN;
  constexpr uint32_t kIdesc = idesc_m128n128<kBf>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char* sm = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(sm);
  float4* E4 = reinterpret_cast<float4*>(sm + DftSmem::E);
  float2* coef_s = reinterpret_cast<float2*>(E4 + A_lay);       // [A][2]
  int4* auto_s = reinterpret_cast<int4*>(coef_s + 2 * A_lay);    // [A]
  float2* tw_s = reinterpret_cast<float2*>(auto_s + A_lay);      // [128] exp(+2 pi i m / 128) (Q128)
  int* cnt_s = reinterpret_cast<int*>(tw_s + 128);           // [16 warps][8] trip counts
  int* base_s = cnt_s + 16 * 8;                              // [16 warps][8] first entries
  // stage 1, stage 2, and a barrier nothing ever arrives at (the failure test)
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(base_s + 16 * 8);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  float* entw_s = reinterpret_cast<float*>(abort_flag + 3);  // [max_entries]
  uint16_t* enta_s = reinterpret_cast<uint16_t*>(entw_s + max_entries);  // [max_entries]
  // batch: the current item's job, copied from the work list (its fields are read
  // in the per-sample code, where shared memory beats L1 under this much shared use)
  DftJob* job_s = reinterpret_cast<DftJob*>(
      (reinterpret_cast<uintptr_t>(enta_s + max_entries) + 15) & ~static_cast<uintptr_t>(15));
  int* claim_s = reinterpret_cast<int*>(abort_flag + 1);                  // batch: claimed item, wait result

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (!kBatch && (long long)blockIdx.x * job0.W >= job0.units) return;
  const uint32_t bar1 = smem_u32(&bars[0]), bar2 = smem_u32(&bars[1]), bar_never = smem_u32(&bars[2]);
  if (Q128 || (kBatch && twiddle))
    for (int m = tid; m < 128; m += kThreads) tw_s[m] = twiddle[m];

  // ---- set-up: TMEM, mbarriers, the DFT matrix into TMEM ----
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
    tc_fence_before();
  }
  if (tid == 0) {
    mbar_init(bar1, 1);
    mbar_init(bar2, 1);
    mbar_init(bar_never, 1);
    fence_mbar_init();
    *abort_flag = 0;
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int lg = warp & 3, cq = warp >> 2;  // TMEM lane group, column quarter
  const uint32_t lane_base = (uint32_t)(32 * lg) << 16;
  if (warp < 4) {
    // row m = 32 lg + lane of the real DFT matrix, hi then lo, 64 packed columns each
    const uint32_t* src = fmat + (size_t)(32 * lg + lane) * 64;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t r[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = src[(size_t)h * 128 * 64 + 16 * q + j];
        tmem_st16(tmem + lane_base + (h ? kColFlo : kColFhi) + 16 * q, r);
      }
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // the job and span being imaged (set per item; read through a pointer, so that
  // the job's fields stay in parameter or global memory rather than registers)
  const DftJob* jp = &job0;
  long long b_item = blockIdx.x, u0 = 0, u1 = 0;
  int c_first = 0;
  bool q128 = Q128;

  uint32_t ph1 = 0, ph2 = 0;
  uint32_t n_commit1 = 0, n_commit2 = 0;  // MMA groups committed to each barrier (every thread counts)
  bool first_wait = true;
  int d2buf = 0, have_prev = 0, prev_buf = 0;
  int pair[4] = {0, 0, 0, 0};                            // gridder: four cell pairs (y, 2r..2r+1), index y*32 + r
  // TMEM lane m = 32 lg + lane holds output row k = 8 (m >> 4) + (m & 7), part
  // c = (m >> 3) & 1 (real, imaginary) of D1 and D2 (see dft_matrix_kernel)
  const int ej = 16 * lg + 8 * (lane >> 4) + (lane & 7), ec = (lane >> 3) & 1;  // epilogue lanes (j, c) of D2
  const int ck = ej, cc = ec;                                                   // conversion lanes (k, c) of D1
  const int cg = cq >> 1, cy0 = 32 * (cq & 1);           // conversion columns (g, y0 .. y0+31)

  float acc[4][8];
#pragma unroll
  for (int pl = 0; pl < 4; ++pl)
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[pl][s] = 0.f;
  // FP16 transforms: the channel's power-of-two scales of the gridded fields and
  // of the stage-1 result, and the factor that undoes both (and the DFT
  // matrix's) on the squares
  float sc_g = 1.f, sc_z = 1.f, sc_out = 1.f;

  // Bounded wait for the next phase of a barrier; on time-out the plan's status
  // word and the CTA's abort flag are set (read by every thread after the next
  // CTA barrier).  With test_wait_ns, the CTA's first wait is instead made on a
  // barrier that nothing arrives at, limited to test_wait_ns: a time-out that
  // is certain to happen, for testing this path.
  auto wait_or_abort = [&](uint32_t bar, uint32_t& ph) -> bool {
    bool ok;
    if (test_wait_ns && first_wait) ok = mbar_wait_bounded(bar_never, 0, test_wait_ns);
    else ok = mbar_wait_bounded(bar, ph);
    first_wait = false;
    if (!ok) {
      atomicExch(jp->status, kDevTimeout);
      *abort_flag = 1;
    }
    ph ^= 1;
    tc_fence_after();
    return ok;
  };

  // squaring and accumulation of one stage-2 result (TMEM lanes (j, c), columns
  // (g, k)); partner lanes (lane ^ 8: same j, other c) exchange the other component
  // (tensor memory is read only by warps all of whose threads saw the products
  // complete; after a time-out the warp squares zeros instead)
  auto epilogue = [&](int buf, bool ok) {
    float X[16], Y[16];
    const uint32_t d2 = tmem + lane_base + kColD2 + 128 * buf;
    if (__all_sync(0xffffffffu, ok)) {
      tmem_ld16(d2 + 16 * cq, X);
      tmem_ld16(d2 + 64 + 16 * cq, Y);
      tmem_wait_ld();
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) X[k] = Y[k] = 0.f;
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float sx = ec ? X[s] : X[8 + s], sy = ec ? Y[s] : Y[8 + s];
      const float rx = __shfl_xor_sync(0xffffffffu, sx, 8), ry = __shfl_xor_sync(0xffffffffu, sy, 8);
      const float xr = ec ? rx : X[s], xi = ec ? X[8 + s] : rx;
      const float yr = ec ? ry : Y[s], yi = ec ? Y[8 + s] : ry;
      acc[0][s] = fmaf(xr, xr, fmaf(xi, xi, acc[0][s]));
      acc[1][s] = fmaf(yr, yr, fmaf(yi, yi, acc[1][s]));
      acc[2][s] = fmaf(xr, yr, fmaf(xi, yi, acc[2][s]));
      acc[3][s] = fmaf(xi, yr, fmaf(-xr, yi, acc[3][s]));
    }
  };

  auto flush = [&](int c) {
    const int slot = c - c_first;
    float* dst = jp->part + (size_t)(b_item * jp->spans + slot) * 4 * NN;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int k = 16 * cq + 8 * ec + s;
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) dst[(size_t)pl * NN + ej * kN + k] = kBf ? acc[pl][s] : acc[pl][s] * sc_out;
    }
    int4* pa = reinterpret_cast<int4*>(jp->part_auto) + (size_t)(b_item * jp->spans + slot) * jp->A;
    for (int a = tid; a < jp->A; a += kThreads) pa[a] = auto_s[a];
  };

  // the two bytes of each of the thread's antennas (a = ta + 512 k < A <= 1024),
  // prefetched one sample ahead so that the unpack never waits for HBM; packed
  // as antenna ta in the low and antenna ta + 512 in the high half.  ta is the
  // thread index shifted by half a block, so that arrays of up to 256 antennas
  // are unpacked by warps 8-15 and warp 0, which issues the products, is spared
  // the unpack of the next sample
  const int ta = (tid + kThreads / 2) & (kThreads - 1);
  auto load_raw = [&](int c, int t) -> unsigned {
    const int cr = q128 ? c >> 2 : c;
    const unsigned short* base =
        reinterpret_cast<const unsigned short*>(jp->volts + ((size_t)t * jp->C + cr) * (size_t)jp->A * 2);
    unsigned r = ta < jp->A ? (unsigned)__ldg(base + ta) : 0u;
    if (ta + kThreads < jp->A) r |= (unsigned)__ldg(base + ta + kThreads) << 16;
    return r;
  };
  unsigned raw = 0, raw_next = 0;
  const uint16_t* ent_a = enta_s;
  const float* ent_w = entw_s;

  // 1. unpack, calibrate, exact integer self powers of one sample's bytes
  auto unpack = [&](unsigned rw) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = ta + h * kThreads;
      const unsigned rb = h ? rw >> 16 : rw & 0xffffu;
      if (a < jp->A) {
        const int xr = nib_hi(rb & 0xffu), xi = nib_lo(rb & 0xffu);
        const int yr = nib_hi(rb >> 8), yi = nib_lo(rb >> 8);
        const float2 kx = coef_s[2 * a], ky = coef_s[2 * a + 1];
        E4[a] = make_float4(kx.x * xr - kx.y * xi, kx.x * xi + kx.y * xr, ky.x * yr - ky.y * yi,
                            ky.x * yi + ky.y * yr);
        int4 au = auto_s[a];
        au.x += xr * xr + xi * xi;
        au.y += yr * yr + yi * yi;
        au.z += xr * yr + xi * yi;
        au.w += xi * yr - xr * yi;
        auto_s[a] = au;
      }
    }
  };
  bool have_next = false;  // E already holds this sample (unpacked while stage 1 ran)
  int cur_c = -1;
  for (int it = 0;; ++it) {
    // ---- the next item: this CTA's span, or the next unclaimed one of the queue
    if constexpr (!kBatch) {
      if (it > 0) break;
    } else {
      __syncthreads();  // every thread has read the previous claim and the abort flag is settled
      if (*abort_flag) break;
      if (tid == 0) *claim_s = atomicAdd(queue.head, 1);
      __syncthreads();
      const int item = *claim_s;
      if (item >= queue.n_items) break;
      if (item >= queue.n_image_items) {
        // ---- a reduction item: rows of one virtual channel of one job, once
        // every imaging item that wrote a partial image of it has signalled
        int k = 0;
        while (k + 1 < queue.n_jobs && item >= queue.jobs[k + 1].red_first) ++k;
        const DftJob& rj = queue.jobs[k];
        const int L = rj.red.vq == 4 ? rj.red.N / 2 : rj.red.N;
        const int piece = item - rj.red_first, per_cv = L / rj.red_rows;
        const int cv = piece / per_cv, j0 = (piece % per_cv) * rj.red_rows;
        if (tid == 0) {
          const long long b_lo = ((long long)cv * rj.red.T) / rj.red.W;
          const long long b_hi = min(((long long)(cv + 1) * rj.red.T - 1) / rj.red.W, (long long)rj.red.ctas - 1);
          const bool ok = wait_count_bounded(rj.done + cv, (int)(b_hi - b_lo + 1) + queue.test_extra,
                                             queue.wait_ns ? queue.wait_ns : kWaitNs);
          if (!ok) atomicExch(rj.status, kDevTimeout);
          claim_s[1] = ok ? 1 : 0;
        }
        __syncthreads();
        if (claim_s[1]) reduce_rows<2, kBatchReducePix>(rj.red, cv, j0, rj.red_rows, tid, kThreads, sm);
        continue;
      }
      int k = 0;
      while (k + 1 < queue.n_jobs && item >= queue.jobs[k + 1].first_item) ++k;
      {
        const int* src = reinterpret_cast<const int*>(&queue.jobs[k]);
        int* dst = reinterpret_cast<int*>(job_s);
        for (int i = tid; i < (int)(sizeof(DftJob) / sizeof(int)); i += kThreads) dst[i] = src[i];
      }
      __syncthreads();
      jp = job_s;
      b_item = item - jp->first_item;
      q128 = jp->q128 != 0;
    }
    u0 = b_item * jp->W;
    u1 = min(u0 + jp->W, jp->units);
    if (u0 >= u1) continue;
    c_first = (int)(u0 / jp->T);
    // unit u = (channel cu, sample tu), stepped without 64-bit divisions
    int cu = c_first, tu = (int)(u0 - (long long)c_first * jp->T);
    raw = load_raw(cu, tu);
    have_next = false;
    cur_c = -1;
  for (long long u = u0; u < u1; ++u) {
    const int c = cu;
    int cn = cu, tn = tu + 1;  // the next unit
    if (tn == jp->T) {
      tn = 0;
      ++cn;
    }
    if (c != cur_c) {
      if (have_prev) {  // the last sample of the previous channel still owes its squares
        const bool ok2 = wait_or_abort(bar2, ph2);
        epilogue(prev_buf, ok2);
        have_prev = 0;
      }
      const int flushed = cur_c;
      if (cur_c >= 0) {
        flush(cur_c);
#pragma unroll
        for (int pl = 0; pl < 4; ++pl)
#pragma unroll
          for (int s = 0; s < 8; ++s) acc[pl][s] = 0.f;
        if constexpr (kBatch) __threadfence();  // the partial image is visible GPU-wide before the signal
      }
      cur_c = c;
      tc_fence_before();
      __syncthreads();
      if (kBatch && flushed >= 0 && tid == 0) atomicAdd(jp->done + flushed, 1);
      const int cr = q128 ? c >> 2 : c;
      if constexpr (!kBf) {
        const float4 sc = jp->dscale[c];
        sc_g = sc.x;
        sc_z = sc.y;
        sc_out = sc.z;
      }
      // (FP16: the fields' scale rides on the coefficients, exactly: a power of two)
      for (int k = tid; k < 2 * jp->A; k += kThreads) {
        float2 v = jp->coef[(size_t)cr * jp->A * 2 + k];
        if constexpr (!kBf) v = make_float2(v.x * sc_g, v.y * sc_g);
        coef_s[k] = v;
      }
      for (int a = tid; a < jp->A; a += kThreads) auto_s[a] = make_int4(0, 0, 0, 0);
      if (tid < 16 * 8) {
        cnt_s[tid] = jp->cnt[(size_t)c * 16 * 8 + tid];
        base_s[tid] = jp->base[(size_t)c * 16 * 8 + tid];
      }
      const int e0 = jp->off[c], ne = jp->off[c + 1] - e0;
      if (jp->ent_in_smem) {
        for (int k = tid; k < ne; k += kThreads) {
          enta_s[k] = jp->ent_a[e0 + k];
          entw_s[k] = jp->ent_w[e0 + k];
        }
        ent_a = enta_s;
        ent_w = entw_s;
      } else {
        ent_a = jp->ent_a + e0;
        ent_w = jp->ent_w + e0;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) pair[j] = jp->task[((size_t)c * kThreads + tid) * 4 + j];
      __syncthreads();
    }

    if (u + 1 < u1) raw_next = load_raw(cn, tn);

    if (!have_next) {
      unpack(raw);
      __syncthreads();
    }
    have_next = false;

    // 2. grid the thread's four cell pairs (y, 2r..2r+1) of both polarisations
    //    into rows (g, y) of the stage-1 B operand, split into 16-bit hi/lo parts
    //    (the previous sample's stage-1 products, which read this buffer,
    //    completed before its conversion)
    {
      float gre[2][8], gim[2][8];
      // the entry tables in shared memory or in L2: one inlined copy each, so
      // that each reads its tables with loads of the right address space
      // (unrolled by two when the tables are in shared memory; from L2 the
      // unrolled loop was slower: 11.66 -> 13.49 ms on 1 024 antennas at 128^2)
      auto gather = [&](const uint16_t* EA, const float* EW, auto in_smem) {
      // the warp's eight trip counts and first entries, read before the first slot
      int Ks[8], bs[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        Ks[s] = cnt_s[warp * 8 + s];
        bs[s] = base_s[warp * 8 + s];
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        // slot s = cell (s & 1) of pair s >> 1: lane-interleaved entries, warp-uniform trip count
        const int K = Ks[s];
        const int b = bs[s] + lane;
        float xr = 0.f, xi = 0.f, yr = 0.f, yi = 0.f;
        auto entry = [&](int k) {
          const float w = EW[b + 32 * k];
          const float4 ev = E4[EA[b + 32 * k]];
          xr = fmaf(w, ev.x, xr);
          xi = fmaf(w, ev.y, xi);
          yr = fmaf(w, ev.z, yr);
          yi = fmaf(w, ev.w, yi);
        };
        if constexpr (decltype(in_smem)::value) {
#pragma unroll 2
          for (int k = 0; k < K; ++k) entry(k);
        } else {
          for (int k = 0; k < K; ++k) entry(k);
        }
        gre[0][s] = xr; gim[0][s] = xi; gre[1][s] = yr; gim[1][s] = yi;
      }
      };
      if (jp->ent_in_smem)
        gather(enta_s, entw_s, std::true_type{});
      else
        gather(ent_a, ent_w, std::false_type{});
      if (q128) {
        // H_q = exp(+2 pi i (alpha x + beta y) / 128) x the folded gather
        const int alpha = cur_c & 1, beta = (cur_c >> 1) & 1;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int y = pair[s >> 1] >> 5, x = 2 * (pair[s >> 1] & 31) + (s & 1);
          const float2 w = tw_s[(alpha * x + beta * y) & 127];
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const float re = gre[g][s], im = gim[g][s];
            gre[g][s] = re * w.x - im * w.y;
            gim[g][s] = re * w.y + im * w.x;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int y = pair[j] >> 5, x = 2 * (pair[j] & 31);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const uint32_t off = slab_off(g * kN + y, x);
#pragma unroll
          for (int comp = 0; comp < 2; ++comp) {
            const float* v = comp ? gim[g] : gre[g];
            const uint32_t hi = pack2<kBf>(v[2 * j], v[2 * j + 1]);
            *reinterpret_cast<uint32_t*>(sm + DftSmem::B1 + comp * kSlab + off) = hi;
            if constexpr (Pr::kSplit) {
              const float2 back = unpack2<kBf>(hi);
              *reinterpret_cast<uint32_t*>(sm + DftSmem::B1 + (2 + comp) * kSlab + off) =
                  pack2<kBf>(v[2 * j] - back.x, v[2 * j + 1] - back.y);
            }
          }
        }
      }
    }
    fence_proxy_async();
    __syncthreads();

    // 3. stage 1: D1 = Fre . G^T, lanes (k, c), columns (g, y)
    if (tid == 0) {
      tc_fence_after();
      const uint32_t gHi = sbase + DftSmem::B1, gLo = gHi + 2 * kSlab;
      uint32_t accum = 0;
#pragma unroll
      for (int pr = 0; pr < (Pr::kSplit ? 3 : 1); ++pr) {
        const uint32_t fcol = (pr == 1) ? kColFlo : kColFhi;
        const uint32_t b = (pr == 2) ? gLo : gHi;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          mma_f16_ts(tmem + kColD1, tmem + fcol + 8 * kk, sdesc_sw128(b + (kk >> 2) * kSlab + (kk & 3) * 32),
                     kIdesc, accum);
          accum = 1;
        }
      }
      mma_commit(bar1);
    }
    ++n_commit1;

    // 4. while stage 1 runs: squares of the previous sample, and the next
    //    sample's fields if it is of the same channel (every thread has
    //    finished the gather that read E)
    if (have_prev) {
      const bool ok2 = wait_or_abort(bar2, ph2);
      epilogue(prev_buf, ok2);
    }
    if (u + 1 < u1 && cn == c) {
      unpack(raw_next);
      have_next = true;
    }

    // 5. Z = D1 -> stage-2 B operand rows (g, k), K = (c, y), split hi/lo (the
    //    previous sample's stage-2 products, which read this buffer, are
    //    complete), and 6. stage 2: D2[buf] = Fre . Z^T, lanes (j, c), columns
    //    (g, k), which runs while the next sample is unpacked and gridded.  The
    //    conversion is done in two halves along K (a thread's first 16 y values
    //    are the K steps 0, 2, 4, 6, its last 16 the steps 1, 3, 5, 7).
    const bool ok1 = wait_or_abort(bar1, ph1);
    uint32_t accum2 = 0;
    const uint32_t d1 = tmem + lane_base + kColD1 + 32 * cq;
    const int zrow = cg * kN + ck;
    // both halves of the thread's stage-1 row read at once (one wait)
    float vz[2][16];
    if (__all_sync(0xffffffffu, ok1)) {
      tmem_ld16(d1, vz[0]);
      tmem_ld16(d1 + 16, vz[1]);
      tmem_wait_ld();
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) vz[0][k] = vz[1][k] = 0.f;
    }
    auto convert_z = [&](int half, bool sync) {
      float (&v)[16] = vz[half];
      if constexpr (!kBf) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] *= sc_z;
      }
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          hi[h] = pack2<kBf>(v[8 * qq + 2 * h], v[8 * qq + 2 * h + 1]);
          if constexpr (Pr::kSplit) {
            const float2 back = unpack2<kBf>(hi[h]);
            lo[h] = pack2<kBf>(v[8 * qq + 2 * h] - back.x, v[8 * qq + 2 * h + 1] - back.y);
          }
        }
        const uint32_t off = slab_off(zrow, cy0 + 16 * half + 8 * qq);
        *reinterpret_cast<uint4*>(sm + DftSmem::B2 + cc * kSlab + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if constexpr (Pr::kSplit)
          *reinterpret_cast<uint4*>(sm + DftSmem::B2 + (2 + cc) * kSlab + off) =
              make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      if (sync) {
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
      }
    };
    auto issue_stage2 = [&](int half) {
      if (tid == 0) {
        tc_fence_after();
        const uint32_t zHi = sbase + DftSmem::B2, zLo = zHi + 2 * kSlab;
#pragma unroll
        for (int pr = 0; pr < (Pr::kSplit ? 3 : 1); ++pr) {
          const uint32_t fcol = (pr == 1) ? kColFlo : kColFhi;
          const uint32_t b = (pr == 2) ? zLo : zHi;
#pragma unroll
          for (int kq = 0; kq < 4; ++kq) {
            const int kk = 2 * kq + half;
            mma_f16_ts(tmem + kColD2 + 128 * d2buf, tmem + fcol + 8 * kk,
                       sdesc_sw128(b + (kk >> 2) * kSlab + (kk & 3) * 32), kIdesc, accum2);
            accum2 = 1;
          }
        }
        if (half == 1) mma_commit(bar2);
      }
      if (half == 1) ++n_commit2;
    };
    // both halves converted before one CTA barrier (a barrier between them, to start
    // the first half's products early, measured slower), then all of stage 2
    convert_z(0, false);
    convert_z(1, true);
    if (*abort_flag) break;  // no wait lies between here and the commit below
    issue_stage2(0);
    issue_stage2(1);
    have_prev = 1;
    prev_buf = d2buf;
    d2buf ^= 1;
    raw = raw_next;
    cu = cn;
    tu = tn;
  }
  // ---- end of the item: the last sample's squares, then its channel's partial
  if (*abort_flag) break;  // read after the loop's last CTA barrier: every thread agrees
  if (have_prev) {
    const bool ok2 = wait_or_abort(bar2, ph2);
    epilogue(prev_buf, ok2);
    have_prev = 0;
  }
  if (cur_c >= 0) flush(cur_c);
  if constexpr (kBatch) {
    __threadfence();
    __syncthreads();
    if (tid == 0 && cur_c >= 0) atomicAdd(jp->done + cur_c, 1);
  }
#pragma unroll
  for (int pl = 0; pl < 4; ++pl)
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[pl][s] = 0.f;
  }
  // after a timed-out wait the MMAs may still be running: one more bounded wait
  // for the last group committed to each barrier before the tensor memory they
  // write is released.  Each barrier is at most one phase behind: a group is
  // committed only after the wait for the barrier's previous group succeeded
  // (after a time-out the loop issues at most the current sample's stage 1,
  // whose barrier's previous wait did succeed, and leaves before stage 2)
  if (*abort_flag) {
    if (n_commit1) mbar_wait_bounded(bar1, (n_commit1 - 1) & 1);
    if (n_commit2) mbar_wait_bounded(bar2, (n_commit2 - 1) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- plan-time tables ----------------------------------------------------------
// The real 2N x 2N DFT matrix [[Fr, -Fi], [Fi, Fr]] with rows
// m = 16 (k / 8) + 8 c + k % 8 (c = 0 real, 1 imaginary output part: eight
// output rows k in a row, so that the eight threads of a 16-byte store phase of
// the stage-1 conversion write eight consecutive rows of one slab, free of
// bank conflicts) and columns K = c' N + x, split into 16-bit hi
// and lo parts in FP64, stored row-major as packed pairs (element K in the low
// half of word K/2 when K is even): [2 (hi, lo)][128 rows][64 words].  The FP16
// matrix is scaled by 2^kFp16MatExp, so that its low parts (up to 2^-12 of an
// entry) stay clear of FP16's subnormal range.
template <bool kBf16>
__global__ void dft_matrix_kernel(uint16_t* __restrict__ out) {
  const int m = blockIdx.x;          // 0..127
  const int kk = threadIdx.x;        // 0..127
  const int k = 8 * (m >> 4) + (m & 7), c = (m >> 3) & 1, cp = kk >> 6, x = kk & 63;
  const int f = k - kN / 2;
  const int ph = (((f * x) % kN) + kN) % kN;
  double sn, cs;
  sincospi(2.0 * (double)ph / (double)kN, &sn, &cs);
  // output re = Fr Gr - Fi Gi ; output im = Fi Gr + Fr Gi
  const double v = ldexp((c == 0) ? (cp == 0 ? cs : -sn) : (cp == 0 ? sn : cs), kBf16 ? 0 : kFp16MatExp);
  uint16_t hi, lo;
  if (kBf16) {
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(h)));
  } else {
    const __half h = __double2half(v);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__double2half(v - (double)__half2float(h)));
  }
  out[(size_t)m * 128 + kk] = hi;
  out[(size_t)128 * 128 + (size_t)m * 128 + kk] = lo;
}

// Power-of-two scales of the FP16 transforms, per virtual channel: bounds on
// the 64 x 64 field each virtual channel transforms (the grid itself, its four
// quadrants folded for a 128 x 128 grid, or a zero-padded 32 x 32 grid).  With
// cb(y, x) = 8 sqrt(2) sum_{a covering the field cell} |w_a| max_p |k_a,p| >=
// |G(y, x)| (a 4+4-bit sample has modulus at most 8 sqrt(2)),
//   bound_G = max_(y,x) cb,   bound_Z = max_y sum_x cb >= |stage-1 result|
// (every DFT matrix entry has modulus 1).  The fields are scaled by
// s_g = 2^(15 - e(bound_G)) and the stage-1 result (which carries s_g and the
// matrix's 2^12) by s_z = 2^(15 - e(2^12 s_g bound_Z)), where 2^e(b) is the
// next power of two above b, so that every 16-bit operand stays below 2^15;
// the squares of the stage-2 result carry (2^24 s_g s_z)^2, undone in FP32 by
// s_out.  All three are exact powers of two.
__global__ void dft_scale_kernel(int A, int P, int N, int S, int vq, const int* __restrict__ csr_ptr,
                                 const int2* __restrict__ csr_ent, const double2* __restrict__ coef64,
                                 float4* __restrict__ out) {
  __shared__ double row_sum[kN], row_max[kN];
  const int c = blockIdx.x, fy = threadIdx.x;  // one thread per field row
  const int NN = N * N;
  const int* ptr = csr_ptr + (size_t)c * (NN + 1);
  const int2* ent = csr_ent + (size_t)c * A * S * S;
  const double2* k = coef64 + (size_t)c * A * P;
  if (fy < kN) {
    double rs = 0.0, rm = 0.0;
    for (int fx = 0; fx < kN; ++fx) {
      double cb = 0.0;
      const int reps = (N == 128) ? 4 : 1;
      for (int r = 0; r < reps; ++r) {
        const int y = fy + kN * (r >> 1), x = fx + kN * (r & 1);
        if (y >= N || x >= N) continue;  // a 32 x 32 grid padded to 64 x 64
        for (int e = ptr[y * N + x]; e < ptr[y * N + x + 1]; ++e) {
          const int2 en = ent[e];
          double km = 0.0;
          for (int p = 0; p < P; ++p) km = fmax(km, hypot(k[(size_t)en.x * P + p].x, k[(size_t)en.x * P + p].y));
          cb += fabs((double)__int_as_float(en.y)) * km;
        }
      }
      cb *= 8.0 * 1.4142135623730951;
      rs += cb;
      rm = fmax(rm, cb);
    }
    row_sum[fy] = rs;
    row_max[fy] = rm;
  }
  __syncthreads();
  if (fy == 0) {
    double bg = 0.0, bz = 0.0;
    for (int y = 0; y < kN; ++y) {
      bg = fmax(bg, row_max[y]);
      bz = fmax(bz, row_sum[y]);
    }
    // 2^e above b: frexp gives b = m 2^e with m in [0.5, 1); a zero bound needs no scale
    int eg = 0, ez = 0;
    if (bg > 0.0) frexp(bg, &eg);
    const int sg = max(-100, min(100, kFp16TopExp - eg));
    if (bz > 0.0) frexp(ldexp(bz, kFp16MatExp + sg), &ez);
    int sz = max(-100, min(100, kFp16TopExp - ez));
    // the squares' factor 2^(-2 (2 * 12 + sg + sz)) must stay a normal FP32
    const int tot = max(-60, min(60, 2 * kFp16MatExp + sg + sz));
    sz = tot - 2 * kFp16MatExp - sg;
    const float4 v = make_float4(ldexpf(1.f, sg), ldexpf(1.f, sz), ldexpf(1.f, -2 * tot), 0.f);
    for (int q = 0; q < vq; ++q) out[(size_t)c * vq + q] = v;
  }
}

size_t dft_smem_bytes(int A, int max_entries) {
  size_t b = 8 * (size_t)kSlab;            // the two B operands (gridded fields, stage-1 result)
  b += 16 * (size_t)A + 16 * (size_t)A + 16 * (size_t)A;  // E, coefficients, self powers
  b += 128 * sizeof(float2);                // twiddles of the 128 x 128 split
  b += 2 * 16 * 8 * sizeof(int);            // gather trip counts and bases
  b += 40;                                  // three mbarriers, TMEM address, abort flag
  b += 6 * (size_t)max_entries;             // gather entries (weight, antenna)
  b += sizeof(DftJob) + 16;                 // a batch item's job
  return b + 1024;                          // alignment slack
}

// The job of one call of plan p over T samples with split ws.
DftJob job_of(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part, int* part_auto) {
  DftJob j{};
  j.volts = d_volts;
  j.coef = p.d_coef;
  j.cnt = p.gt.d_cnt;
  j.base = p.gt.d_base;
  j.off = p.gt.d_chan_off;
  j.task = p.gt.d_task;
  j.ent_a = p.gt.d_ent_a;
  j.ent_w = p.gt.d_ent_w;
  j.dscale = reinterpret_cast<const float4*>(p.d_dscale);
  j.part = part;
  j.part_auto = part_auto;
  j.status = p.d_status;
  j.W = ws.W;
  j.units = ws.units;
  j.T = T;
  j.C = p.C;
  j.A = p.A;
  j.spans = ws.spans;
  j.q128 = p.N == 128 ? 1 : 0;
  j.ent_in_smem = p.ent_in_smem;
  j.first_item = 0;
  j.n_items = ws.ctas;
  return j;
}

template <int XF>
cudaError_t dft_launch(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                       int* part_auto, cudaStream_t s, unsigned long long test_wait_ns) {
  const DftJob job = job_of(p, d_volts, T, ws, part, part_auto);
  const DftQueue none{nullptr, 0, 0, 0, nullptr, 0, 0};
  auto kern = p.N == 128 ? dft_image_kernel<XF, true, false> : dft_image_kernel<XF, false, false>;
  kern<<<ws.ctas, kThreads, p.smem, s>>>(job, none, p.A, p.ent_in_smem ? p.gt.max_chan_entries : 0,
                                         reinterpret_cast<const uint32_t*>(p.d_fmat), p.d_twiddle, test_wait_ns);
  return cudaGetLastError();
}

template <int XF>
cudaError_t dft_batch_launch(const DftQueue& q, int A_lay, int max_entries, const uint32_t* fmat,
                             const float2* twiddle, int ctas, size_t smem, cudaStream_t s) {
  const DftJob none{};
  dft_image_kernel<XF, false, true><<<ctas, kThreads, smem, s>>>(none, q, A_lay, max_entries, fmat, twiddle, 0ull);
  return cudaGetLastError();
}

template <int XF>
cudaError_t dft_attr() {
  cudaError_t e = allow_max_smem(dft_image_kernel<XF, false, false>);
  if (e == cudaSuccess) e = allow_max_smem(dft_image_kernel<XF, true, false>);
  if (e == cudaSuccess) e = allow_max_smem(dft_image_kernel<XF, false, true>);
  return e;
}

}  // namespace

// Shared memory the tensor kernel needs for a plan whose largest channel has
// max_entries padded gather entries.
size_t dft_smem_need(int A, int max_entries) { return dft_smem_bytes(A, max_entries); }

cudaError_t launch_dft_tables(Plan& p, cudaStream_t s) {
  if (p.xform == EPIC_XFORM_DFT_BF16X3 || p.xform == EPIC_XFORM_DFT_BF16) {
    dft_matrix_kernel<true><<<128, 128, 0, s>>>(p.d_fmat);
  } else {
    dft_matrix_kernel<false><<<128, 128, 0, s>>>(p.d_fmat);
    dft_scale_kernel<<<p.C, kN, 0, s>>>(p.A, p.P, p.N, p.S, p.vq, p.d_csr_ptr, p.d_csr_ent, p.d_coef64,
                                        reinterpret_cast<float4*>(p.d_dscale));
  }
  return cudaGetLastError();
}

cudaError_t dft_image_config(Plan& p, int* ctas_per_sm) {
  int dev = 0, optin = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e0 != cudaSuccess) return e0;
  p.threads = kThreads;
  // gather entries in shared memory when they fit, else read through L1/L2
  p.ent_in_smem = dft_smem_bytes(p.A, p.gt.max_chan_entries) <= (size_t)optin ? 1 : 0;
  p.smem = dft_smem_bytes(p.A, p.ent_in_smem ? p.gt.max_chan_entries : 0);
  if (p.smem > (size_t)optin) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  switch (p.xform) {
    case EPIC_XFORM_DFT_BF16X3: e = dft_attr<EPIC_XFORM_DFT_BF16X3>(); break;
    case EPIC_XFORM_DFT_FP16X3: e = dft_attr<EPIC_XFORM_DFT_FP16X3>(); break;
    case EPIC_XFORM_DFT_BF16: e = dft_attr<EPIC_XFORM_DFT_BF16>(); break;
    default: e = dft_attr<EPIC_XFORM_DFT_FP16>(); break;
  }
  if (e != cudaSuccess) return e;
  *ctas_per_sm = 1;  // the kernel holds all 512 TMEM columns
  return cudaSuccess;
}

size_t dft_batch_smem(int A_lay, int max_entries) { return dft_smem_bytes(A_lay, max_entries); }

cudaError_t launch_dft_batch(int xform, const DftQueue& q, int A_lay, int max_entries, const uint16_t* fmat,
                             const float2* twiddle, int ctas, cudaStream_t s) {
  const size_t smem = dft_smem_bytes(A_lay, max_entries);
  const uint32_t* f = reinterpret_cast<const uint32_t*>(fmat);
  switch (xform) {
    case EPIC_XFORM_DFT_BF16X3: return dft_batch_launch<EPIC_XFORM_DFT_BF16X3>(q, A_lay, max_entries, f, twiddle, ctas, smem, s);
    case EPIC_XFORM_DFT_FP16X3: return dft_batch_launch<EPIC_XFORM_DFT_FP16X3>(q, A_lay, max_entries, f, twiddle, ctas, smem, s);
    case EPIC_XFORM_DFT_BF16: return dft_batch_launch<EPIC_XFORM_DFT_BF16>(q, A_lay, max_entries, f, twiddle, ctas, smem, s);
    default: return dft_batch_launch<EPIC_XFORM_DFT_FP16>(q, A_lay, max_entries, f, twiddle, ctas, smem, s);
  }
}

DftJob dft_job(const Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part, int* part_auto) {
  return job_of(p, d_volts, T, ws, part, part_auto);
}

cudaError_t launch_dft_image(Plan& p, const uint8_t* d_volts, int T, const WorkSplit& ws, float* part,
                             int* part_auto, cudaStream_t s, unsigned long long test_wait_ns) {
  const unsigned long long tw = test_wait_ns;
  switch (p.xform) {
    case EPIC_XFORM_DFT_BF16X3: return dft_launch<EPIC_XFORM_DFT_BF16X3>(p, d_volts, T, ws, part, part_auto, s, tw);
    case EPIC_XFORM_DFT_FP16X3: return dft_launch<EPIC_XFORM_DFT_FP16X3>(p, d_volts, T, ws, part, part_auto, s, tw);
    case EPIC_XFORM_DFT_BF16: return dft_launch<EPIC_XFORM_DFT_BF16>(p, d_volts, T, ws, part, part_auto, s, tw);
    default: return dft_launch<EPIC_XFORM_DFT_FP16>(p, d_volts, T, ws, part, part_auto, s, tw);
  }
}

}  // namespace epic
