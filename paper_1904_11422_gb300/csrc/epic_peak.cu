// epic_peak.cu -- a measurement of the FP32 FMA rate this GPU sustains, the
// denominator of the FP32 imaging kernels' roofline (those kernels are bound
// by plain FP32 arithmetic, not by memory).  Every thread runs kChains
// independent chains of dependent FMAs, enough to cover the FMA latency at full
// occupancy; two CTAs of 1024 threads per SM fill every warp slot.
#include "epic_internal.cuh"

namespace {

constexpr int kChains = 8, kUnroll = 16, kThreads = 1024;

__global__ void __launch_bounds__(kThreads, 2)
    fma_chain_kernel(const float* __restrict__ seed, float* __restrict__ sink, long long iters) {
  const float a = seed[0], b = seed[1];
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = seed[2] + (float)(j + (threadIdx.x & 7));
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kUnroll; ++k)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  // never true for the seeds below; keeps the chains live
  if (s == seed[3]) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" epic_status epic_debug_fma_rate(long long iterations, double* tflops, void* stream) {
  if (!tflops || iterations < 1 || iterations > (1LL << 32)) return EPIC_ERR_INVALID_ARG;
  *tflops = 0.0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e == cudaErrorNoDevice ? EPIC_ERR_NO_DEVICE : EPIC_ERR_CUDA;
  const int ctas = 2 * sms;
  float* d = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&d), sizeof(float) * (4 + (size_t)ctas * kThreads)) != cudaSuccess) {
    (void)cudaGetLastError();
    return EPIC_ERR_OOM;
  }
  // x -> 0.999999 x + 1e-6 stays near 1: no overflow, no subnormals
  const float seed[4] = {0.999999f, 1e-6f, 1.0f, -12345.0f};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMemcpyAsync(d, seed, sizeof(seed), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_chain_kernel<<<ctas, kThreads, 0, s>>>(d, d + 4, iterations / 8 + 1);  // warm-up: clocks up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_chain_kernel<<<ctas, kThreads, 0, s>>>(d, d + 4, iterations);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return EPIC_ERR_CUDA;
  const double flops = 2.0 * kChains * kUnroll * (double)iterations * ctas * kThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return EPIC_OK;
}
