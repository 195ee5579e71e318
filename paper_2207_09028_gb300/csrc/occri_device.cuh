// occri_device.cuh -- small device helpers shared by the kernels.
#pragma once

#include "occri_internal.h"

namespace occri {
namespace dev {

template <typename T> __device__ __forceinline__ cplx_t<T> mk(T x, T y) { return {x, y}; }

template <typename T>
__device__ __forceinline__ cplx_t<T> cmul(cplx_t<T> a, cplx_t<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// conj(a) * b
template <typename T>
__device__ __forceinline__ cplx_t<T> cmulc(cplx_t<T> a, cplx_t<T> b) {
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double expm1_t(double x) { return expm1(x); }
__device__ __forceinline__ float expm1_t(float x) { return expm1f(x); }

// e^{sgn 2 pi i num / den} for integers, num reduced to [-den/2, den/2) first.
template <typename T>
__device__ __forceinline__ cplx_t<T> cis_frac(long long num, long long den, int sgn) {
  long long r = num % den;
  if (r < 0) r += den;
  if (2 * r >= den) r -= den;
  T s, c;
  sincospi_t(T(2) * T(r) / T(den), &s, &c);
  return {c, T(sgn) * s};
}

// Same for small arguments (|num|, den < 2^24): 32-bit integer reduction only.
template <typename T>
__device__ __forceinline__ cplx_t<T> cis_frac_i(int num, int den, int sgn) {
  int r = num % den;
  if (r < 0) r += den;
  if (2 * r >= den) r -= den;
  T s, c;
  sincospi_t(T(2 * r) / T(den), &s, &c);
  return {c, T(sgn) * s};
}

// T0 packing: three signed 10-bit lattice coordinates in one int.
__host__ __device__ __forceinline__ int pack_t0(int a, int b, int c) {
  return (a & 1023) | ((b & 1023) << 10) | ((c & 1023) << 20);
}
__device__ __forceinline__ void unpack_t0(int v, int* a, int* b, int* c) {
  const unsigned u = (unsigned)v;
  *a = (int)(u << 22) >> 22;
  *b = (int)(u << 12) >> 22;
  *c = (int)(u << 2) >> 22;
}

}  // namespace dev
}  // namespace occri
