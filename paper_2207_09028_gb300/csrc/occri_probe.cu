// occri_probe.cu -- measured arithmetic peaks of the current GPU (no counterpart in the
// paper): the denominators of the roofline fractions of ALU-bound stages. Each kernel runs
// eight independent FMA chains per thread on every SM and is timed with CUDA events.
#include <cuda_runtime.h>

#include "occri_internal.h"

namespace occri {
namespace probe {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_f64(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * threadIdx.x + i;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_f32(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * threadIdx.x + i;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed FP32 pairs: one fma.rn.f32x2 is two FMAs
__global__ void __launch_bounds__(256) fma_f32x2(float* out, int iters, float a, float b) {
  unsigned long long x[kChains];
  unsigned long long av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    const float lo = 1e-3f * threadIdx.x + i, hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[i]) : "f"(lo), "f"(hi));
  }
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(av), "l"(bv));
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[i]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace probe
}  // namespace occri

extern "C" int occri_measure_fma_peak(int kind, double* tflops) {
  using namespace occri::probe;
  if (!tflops || kind < 0 || kind > 2) return OCCRI_EINVAL;
  *tflops = 0.0;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return OCCRI_ECUDA;
  }
  const int blocks = nsm * 8, threads = 256;
  const int iters = kind == 0 ? 1 << 12 : 1 << 16;
  void* out = nullptr;
  if (occri::device_malloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return OCCRI_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = OCCRI_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = OCCRI_ECUDA;
  float best = 0.f;
  for (int rep = 0; rep < 4 && st == OCCRI_OK; ++rep) {   // first run warms up
    cudaEventRecord(e0, 0);
    if (kind == 0) fma_f64<<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
    else if (kind == 1) fma_f32<<<blocks, threads>>>((float*)out, iters, 0.999f, 1e-4f);
    else fma_f32x2<<<blocks, threads>>>((float*)out, iters, 0.999f, 1e-4f);
    cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = OCCRI_ECUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (st == OCCRI_OK) {
    const double fmas = (double)blocks * threads * iters * kChains * (kind == 2 ? 2 : 1);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  } else {
    cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
