// occri_pairs.cuh -- kernel-fused FFT round trips of pair densities (steps c, d).
//
// For output k-point k, a block of k' and every occupied pair (i, j), the field
//   rho(r) = conj(psi_{jk'}(r)) psi_{ik}(r) e^{-iq.r},   q = k - k'      (Eq. aodf)
// is transformed, multiplied by v(|G+q|)/N_g (Eqs. VGao, recipcoul) and
// transformed back; the potential W = e^{iq.r} u accumulates into
//   Y_{ik}(r) += psi_{jk'}(r) W(r)                                       (Eq. occrikinterm).
//
// A cubic N^3 field does not fit on one SM, so a round trip takes three passes
// over a scratch field stored as S[f][m3][n1][m2] (third axis outermost):
//   A: plane n1 -- form rho, FFT along n3 then n2, write column-major per m3;
//   B: plane m3 -- FFT along n1, kernel multiply, inverse along m1, inverse along m2;
//   C: plane n1 -- inverse along m3, multiply by e^{iq.r} psi_{jk'} and accumulate Y.
// Each pass moves whole contiguous planes (coalesced) and keeps one 1-D
// transform per thread in registers (fft_reg.cuh); the planes sit in shared
// memory with an odd pitch so that row and column accesses are conflict-free.
#pragma once

#include "fft_reg.cuh"
#include "occri_device.cuh"
#include "occri_internal.h"

namespace occri {
namespace pairs {

using dev::mk;
using dev::cmul;
using dev::cmulc;
using dev::cis_frac;
using dev::exp_t;
using dev::expm1_t;

constexpr int pitch(int n) { return (n % 2 == 0) ? n + 1 : n; }
constexpr int threads_for(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : 128); }

// Integer reduction of x = m + Q/D into [-N/2, N/2): returns X = x*D (exact),
// and whether it is an exact tie at -N/2.
__device__ __forceinline__ long long reduce_axis(int m, int Q, int D, int N, bool* tie) {
  const long long P = (long long)N * D;
  long long X = (long long)m * D + Q;
  // floor((2X + P) / (2P))
  long long num = 2 * X + P, den = 2 * P;
  long long fl = num / den;
  if ((num % den != 0) && ((num < 0) != (den < 0))) --fl;
  X -= P * fl;
  *tie = (2 * X == -P);
  return X;
}

struct AxisVal {
  double xa, xb;   // reduced coordinate and its second alias (== xa unless tied)
  bool zero;
};

__device__ __forceinline__ AxisVal axis_val(int m, int Q, int D, int N) {
  bool tie;
  long long X = reduce_axis(m, Q, D, N, &tie);
  AxisVal a;
  a.xa = double(X) / double(D);
  a.xb = tie ? double(X + (long long)N * D) / double(D) : a.xa;
  a.zero = (X == 0);
  return a;
}

// f(|G+q|)/(4 pi) of Eq. recipcoul for |G+q|^2 = g2 > 0.
template <typename T>
__device__ __forceinline__ T kernel_f(T g2, int kind, T inv4w2) {
  const T base = T(1) / g2;
  if (kind == OCCRI_COULOMB) return base;
  const T y = g2 * inv4w2;
  if (kind == OCCRI_ERFC) return -base * expm1_t(-y);
  return base * exp_t(-y);
}

// (d f/d omega)/(4 pi) = -/+ e^{-x^2/(4 omega^2)} / (2 omega^3) (erfc / erf).
template <typename T>
__device__ __forceinline__ T kernel_df(T g2, int kind, T inv4w2, T omega) {
  if (kind == OCCRI_COULOMB) return T(0);
  const T e = exp_t(-g2 * inv4w2) * T(0.5) / (omega * omega * omega);
  return kind == OCCRI_ERFC ? -e : e;
}

// field f of the wave -> (k' offset, i, j)
struct FieldIdx { int kpl, i, j; };
__device__ __forceinline__ FieldIdx field_idx(int f, int nocc) {
  FieldIdx r;
  r.j = f % nocc;
  r.i = (f / nocc) % nocc;
  r.kpl = f / (nocc * nocc);
  return r;
}

// ------------------------------------------------------------------ async plane staging
// cp.async copies global -> shared without staging through registers, so a whole
// plane is in flight per CTA. Element size 8 B (FP32 complex) or 16 B (FP64 complex).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING));
}

// Copy a contiguous N x N plane into shared memory with row pitch P.
template <typename T, int N, int P>
__device__ __forceinline__ void stage_plane(cplx_t<T>* dst, const cplx_t<T>* src) {
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int r = e / N, c = e - (e / N) * N;
    cp_async<sizeof(cplx_t<T>)>(dst + r * P + c, src + e);
  }
}

// ------------------------------------------------------------------ kernel values per bin
// Axis tables: reduced coordinate x (first alias), flags bit0 = tie, bit1 = x == 0.
// For axis 1 also g11 x^2 split hi/lo, so that |G+q|^2 costs a few FMAs per bin:
//   g2(m1) = a1(m1) + x1(m1) * beta + gamma,  beta = 2 (g12 x2 + g13 x3),
//   gamma = g22 x2^2 + 2 g23 x2 x3 + g33 x3^2 (per column, FP64 split hi/lo).
template <typename T>
struct Axis1 {
  T x, ah, al;
  int flags;
};

__device__ __forceinline__ int axis_flags(const AxisVal& a) {
  return (a.xa != a.xb ? 1 : 0) | (a.zero ? 2 : 0);
}

// Rare bins (an exact tie on some axis, or G+q = 0): full tie-averaged evaluation.
template <typename T, bool DERIV>
__device__ __noinline__ T slow_bin(const PairParams& p, int m1, int m2, int m3, const int* Q) {
  const AxisVal a = axis_val(m1, Q[0], p.D[0], p.N1);
  const AxisVal b = axis_val(m2, Q[1], p.D[1], p.N1);
  const AxisVal c = axis_val(m3, Q[2], p.D[2], p.N1);
  if (a.zero && b.zero && c.zero) return DERIV ? T(p.dg0) : T(p.g0);
  double s = 0.0;
  for (int k = 0; k < 8; ++k) {
    const double x1 = (k & 1) ? a.xb : a.xa, x2 = (k & 2) ? b.xb : b.xa, x3 = (k & 4) ? c.xb : c.xa;
    const double g2 = p.g[0] * x1 * x1 + p.g[1] * x2 * x2 + p.g[2] * x3 * x3 +
                      2.0 * (p.g[3] * x1 * x2 + p.g[4] * x1 * x3 + p.g[5] * x2 * x3);
    s += DERIV ? kernel_df<double>(g2, p.kind, p.inv4w2, p.omega)
               : kernel_f<double>(g2, p.kind, p.inv4w2);
  }
  return T(0.125 * s);
}

template <typename T>
struct ColumnConst {
  T bh, bl, ch, cl;
  int flags;  // bit0: tie on axis 2 or 3; bit1: x2 == 0 and x3 == 0
};

template <typename T>
__device__ __forceinline__ ColumnConst<T> column_const(const PairParams& p, const AxisVal& b,
                                                       const AxisVal& c) {
  const double beta = 2.0 * (p.g[3] * b.xa + p.g[4] * c.xa);
  const double gam = p.g[1] * b.xa * b.xa + p.g[2] * c.xa * c.xa + 2.0 * p.g[5] * b.xa * c.xa;
  ColumnConst<T> r;
  r.bh = T(beta);
  r.bl = T(beta - double(r.bh));
  r.ch = T(gam);
  r.cl = T(gam - double(r.ch));
  r.flags = ((b.xa != b.xb) || (c.xa != c.xb) ? 1 : 0) | ((b.zero && c.zero) ? 2 : 0);
  return r;
}

template <typename T>
__device__ __forceinline__ Axis1<T> axis1_entry(const PairParams& p, const AxisVal& a) {
  const double a1 = p.g[0] * a.xa * a.xa;
  Axis1<T> r;
  r.x = T(a.xa);
  r.ah = T(a1);
  r.al = T(a1 - double(r.ah));
  r.flags = axis_flags(a);
  return r;
}

template <typename T, bool DERIV>
__device__ __forceinline__ T fast_bin(const PairParams& p, const Axis1<T>& a, const ColumnConst<T>& c,
                                      int m1, int m2, int m3, const int* Q) {
  if ((a.flags | c.flags) & 1 || ((a.flags & c.flags) & 2)) return slow_bin<T, DERIV>(p, m1, m2, m3, Q);
  const T g2 = (a.ah + a.x * c.bh + c.ch) + (a.al + a.x * c.bl + c.cl);
  return DERIV ? kernel_df<T>(g2, p.kind, T(p.inv4w2), T(p.omega))
               : kernel_f<T>(g2, p.kind, T(p.inv4w2));
}

// ------------------------------------------------------------------ pass A
// plane n1 of field (i, j): rho = conj(psi_j) psi_i e^{-iq.r}; FFT along n3, then n2.
template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N))
pass_a(const cplx_t<T>* __restrict__ psi, cplx_t<T>* __restrict__ S, PairParams p) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* pl = reinterpret_cast<C2*>(smem_raw);   // psi_i plane, then rho / its transform
  C2* qj = pl + N * P;                         // psi_j plane
  C2* ph2 = qj + N * P;
  C2* ph3 = ph2 + N;
  const int n1 = blockIdx.x;
  const int f = blockIdx.y;
  const FieldIdx fi = field_idx(f, p.nocc);
  const int kp = p.kp0 + fi.kpl;
  stage_plane<T, N, P>(pl, psi + (size_t)(p.k * p.nocc + fi.i) * p.ng + (size_t)n1 * N * N);
  stage_plane<T, N, P>(qj, psi + (size_t)(kp * p.nocc + fi.j) * p.ng + (size_t)n1 * N * N);
  cp_async_commit();
  int Q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) Q[d] = p.kint[p.k * 3 + d] - p.kint[kp * 3 + d];
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    ph2[t] = cis_frac<T>((long long)Q[1] * t, (long long)p.D[1] * N, -1);
    ph3[t] = cis_frac<T>((long long)Q[2] * t, (long long)p.D[2] * N, -1);
  }
  const C2 ph1 = cis_frac<T>((long long)Q[0] * n1, (long long)p.D[0] * N, -1);
  cp_async_wait<0>();
  __syncthreads();
  if (threadIdx.x < N) {  // rows (fixed n2 = r): form rho, FFT along n3
    const int r = threadIdx.x;
    const C2 ph12 = cmul<T>(ph1, ph2[r]);
    T re[N], im[N];
    fft::static_for<N>([&](auto I) {
      constexpr int m = decltype(I)::value;
      const C2 v = cmul<T>(cmulc<T>(qj[r * P + m], pl[r * P + m]), cmul<T>(ph12, ph3[m]));
      re[m] = v.x; im[m] = v.y;
    });
    fft::fft_dif<N, -1>(re, im);
    fft::static_for<N>([&](auto I) {
      constexpr int q = decltype(I)::value;
      pl[r * P + fft::dif_rev(N, q)] = mk<T>(re[q], im[q]);
    });
  }
  __syncthreads();
  if (threadIdx.x < N) {  // columns: along n2
    const int c = threadIdx.x;
    T re[N], im[N];
    fft::static_for<N>([&](auto I) {
      constexpr int m = decltype(I)::value;
      const C2 v = pl[m * P + c];
      re[m] = v.x; im[m] = v.y;
    });
    fft::fft_dif<N, -1>(re, im);
    fft::static_for<N>([&](auto I) {
      constexpr int q = decltype(I)::value;
      pl[fft::dif_rev(N, q) * P + c] = mk<T>(re[q], im[q]);
    });
  }
  __syncthreads();
  C2* out = S + (size_t)f * p.ng;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int m3 = e / N, m2 = e - (e / N) * N;
    out[((size_t)m3 * N + n1) * N + m2] = pl[m2 * P + m3];
  }
}

// ------------------------------------------------------------------ pass B
// plane m3 of a field: FFT along n1, multiply by v/(4 pi), inverse along m1, inverse along m2.
template <typename T, int N, bool DOMEGA>
__device__ __forceinline__ void pass_b_body(cplx_t<T>* __restrict__ S, const PairParams& p,
                                            double* dacc) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* plane = reinterpret_cast<C2*>(smem_raw);                 // [n1][m2]
  Axis1<T>* ax1 = reinterpret_cast<Axis1<T>*>(plane + N * P);  // [m1]
  __shared__ double red[4];
  const int m3 = blockIdx.x;
  const int f = blockIdx.y;
  const FieldIdx fi = field_idx(f, p.nocc);
  const int kp = p.kp0 + fi.kpl;
  C2* buf = S + (size_t)f * p.ng + (size_t)m3 * N * N;
  stage_plane<T, N, P>(plane, buf);
  cp_async_commit();
  int Q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) Q[d] = p.kint[p.k * 3 + d] - p.kint[kp * 3 + d];
  for (int t = threadIdx.x; t < N; t += blockDim.x)
    ax1[t] = axis1_entry<T>(p, axis_val(t, Q[0], p.D[0], N));
  const AxisVal a3 = axis_val(m3, Q[2], p.D[2], N);
  cp_async_wait<0>();
  __syncthreads();
  double part = 0.0;
  if (threadIdx.x < N) {  // columns (fixed m2 = c): along n1, kernel, back along m1
    const int c = threadIdx.x;
    const ColumnConst<T> cc = column_const<T>(p, axis_val(c, Q[1], p.D[1], N), a3);
    T re[N], im[N];
    fft::static_for<N>([&](auto I) {
      constexpr int m = decltype(I)::value;
      const C2 v = plane[m * P + c];
      re[m] = v.x; im[m] = v.y;
    });
    fft::fft_dif<N, -1>(re, im);
    if constexpr (DOMEGA) {
      T s = T(0);
      fft::static_for<N>([&](auto I) {
        constexpr int q = decltype(I)::value;
        constexpr int m1 = fft::dif_rev(N, q);
        const T dv = fast_bin<T, true>(p, ax1[m1], cc, m1, c, m3, Q);
        s += dv * (re[q] * re[q] + im[q] * im[q]);
      });
      part = double(s);
    } else {
      fft::static_for<N>([&](auto I) {
        constexpr int q = decltype(I)::value;
        constexpr int m1 = fft::dif_rev(N, q);
        const T v = fast_bin<T, false>(p, ax1[m1], cc, m1, c, m3, Q);
        re[q] *= v;
        im[q] *= v;
      });
      fft::dif_to_natural<N>(re, im);
      fft::fft_dif<N, +1>(re, im);
      fft::static_for<N>([&](auto I) {
        constexpr int q = decltype(I)::value;
        plane[fft::dif_rev(N, q) * P + c] = mk<T>(re[q], im[q]);
      });
    }
  }
  if constexpr (DOMEGA) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(dacc, t);
    }
    return;
  }
  __syncthreads();
  if (threadIdx.x < N) {  // rows: back along m2
    const int r = threadIdx.x;
    T re[N], im[N];
    fft::static_for<N>([&](auto I) {
      constexpr int m = decltype(I)::value;
      const C2 v = plane[r * P + m];
      re[m] = v.x; im[m] = v.y;
    });
    fft::fft_dif<N, +1>(re, im);
    fft::static_for<N>([&](auto I) {
      constexpr int q = decltype(I)::value;
      plane[r * P + fft::dif_rev(N, q)] = mk<T>(re[q], im[q]);
    });
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int r = e / N, c = e - (e / N) * N;
    buf[e] = plane[r * P + c];
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N)) pass_b(cplx_t<T>* __restrict__ S, PairParams p) {
  pass_b_body<T, N, false>(S, p, nullptr);
}

// d E/d omega: the forward half of pass B, accumulating sum_m (dv/d omega)(m) |rho^(m)|^2.
template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N))
pass_b_domega(cplx_t<T>* __restrict__ S, PairParams p, double* dacc) {
  pass_b_body<T, N, true>(S, p, dacc);
}

// ------------------------------------------------------------------ pass C
// plane n1, orbital i: for every j of the wave, inverse along m3, multiply by
// e^{iq.r} psi_{jk'} and accumulate; the gather of field j+1 is in flight while
// field j is transformed (double buffer).
template <typename T, int N, int P>
__device__ __forceinline__ void stage_gather(cplx_t<T>* dst, const cplx_t<T>* src, int n1) {
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int m3 = e / N, n2 = e - (e / N) * N;
    cp_async<sizeof(cplx_t<T>)>(dst + m3 * P + n2, src + ((size_t)m3 * N + n1) * N + n2);
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N))
pass_c(const cplx_t<T>* __restrict__ S, const cplx_t<T>* __restrict__ psi,
       cplx_t<T>* __restrict__ Y, PairParams p) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* g0 = reinterpret_cast<C2*>(smem_raw);   // gather buffers [m3][n2] pitch P
  C2* g1 = g0 + N * P;
  C2* acc = g1 + N * P;                        // [n2][n3] pitch P
  C2* ph2 = acc + N * P;                       // [nkp][N]
  C2* ph3 = ph2 + p.nkp * N;                   // [nkp][N]
  const int n1 = blockIdx.x;
  const int i = blockIdx.y;
  const int nf = p.nkp * p.nocc;               // fields (k', j) summed into this target
  stage_gather<T, N, P>(g0, S + (size_t)(i * p.nocc) * p.ng, n1);   // kpl = 0, j = 0
  cp_async_commit();
  for (int e = threadIdx.x; e < N * P; e += blockDim.x) acc[e] = mk<T>(T(0), T(0));
  for (int t = threadIdx.x; t < p.nkp * N; t += blockDim.x) {
    const int kpl = t / N, x = t - (t / N) * N, kp = p.kp0 + kpl;
    const int q2 = p.kint[p.k * 3 + 1] - p.kint[kp * 3 + 1];
    const int q3 = p.kint[p.k * 3 + 2] - p.kint[kp * 3 + 2];
    ph2[t] = cis_frac<T>((long long)q2 * x, (long long)p.D[1] * N, +1);
    ph3[t] = cis_frac<T>((long long)q3 * x, (long long)p.D[2] * N, +1);
  }
  for (int u = 0; u < nf; ++u) {
    const int kpl = u / p.nocc, j = u - (u / p.nocc) * p.nocc;
    C2* cur = (u & 1) ? g1 : g0;
    if (u + 1 < nf) {
      const int kpl2 = (u + 1) / p.nocc, j2 = (u + 1) - kpl2 * p.nocc;
      const int f2 = (kpl2 * p.nocc + i) * p.nocc + j2;
      stage_gather<T, N, P>((u & 1) ? g0 : g1, S + (size_t)f2 * p.ng, n1);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if (threadIdx.x < N) {
      const int c = threadIdx.x;  // n2
      const int kp = p.kp0 + kpl;
      const int q1 = p.kint[p.k * 3] - p.kint[kp * 3];
      T re[N], im[N];
      fft::static_for<N>([&](auto I) {
        constexpr int m = decltype(I)::value;
        const C2 v = cur[m * P + c];
        re[m] = v.x; im[m] = v.y;
      });
      fft::fft_dif<N, +1>(re, im);
      const C2 ph12 = cmul<T>(cis_frac<T>((long long)q1 * n1, (long long)p.D[0] * N, +1),
                              ph2[kpl * N + c]);
      const C2* pj = psi + (size_t)(kp * p.nocc + j) * p.ng + ((size_t)n1 * N + c) * N;
      const C2* p3 = ph3 + kpl * N;
      fft::static_for<N>([&](auto I) {
        constexpr int q = decltype(I)::value;
        constexpr int n3 = fft::dif_rev(N, q);
        const C2 w = cmul<T>(mk<T>(re[q], im[q]), cmul<T>(ph12, p3[n3]));
        const C2 t = cmul<T>(__ldg(pj + n3), w);
        C2 a = acc[c * P + n3];
        a.x += t.x;
        a.y += t.y;
        acc[c * P + n3] = a;
      });
    }
    __syncthreads();
  }
  C2* y = Y + (size_t)(p.k * p.nocc + i) * p.ng + (size_t)n1 * N * N;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int n2 = e / N, n3 = e - (e / N) * N;
    C2 v = y[e];
    const C2 a = acc[n2 * P + n3];
    v.x += a.x;
    v.y += a.y;
    y[e] = v;
  }
}

template <int N> constexpr size_t smem_a(size_t csz) { return csz * (2 * N * pitch(N) + 2 * N); }
template <int N> constexpr size_t smem_b(size_t csz, size_t tab) { return csz * N * pitch(N) + N * tab; }
inline size_t smem_c(int N, int nkp, size_t csz) {
  return csz * (3 * (size_t)N * pitch(N) + 2 * (size_t)nkp * N);
}

template <typename T, int N>
cudaError_t run_wave(const PairParams& p, const cplx_t<T>* psi, cplx_t<T>* S, cplx_t<T>* Y,
                     cudaStream_t st, cudaEvent_t* ev) {
  using C2 = cplx_t<T>;
  const int nt = threads_for(N);
  const int nf = p.nkp * p.nocc * p.nocc;
  const size_t sa = smem_a<N>(sizeof(C2));
  const size_t sb = smem_b<N>(sizeof(C2), sizeof(Axis1<T>));
  const size_t sc = smem_c(N, p.nkp, sizeof(C2));
  static size_t configured_c = 0;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(pass_a<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    cudaFuncSetAttribute(pass_b<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    configured = true;
  }
  if (sc > configured_c) {
    cudaFuncSetAttribute(pass_c<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    configured_c = sc;
  }
  if (ev) cudaEventRecord(ev[0], st);
  pass_a<T, N><<<dim3(N, nf), nt, sa, st>>>(psi, S, p);
  if (ev) cudaEventRecord(ev[1], st);
  pass_b<T, N><<<dim3(N, nf), nt, sb, st>>>(S, p);
  if (ev) cudaEventRecord(ev[2], st);
  pass_c<T, N><<<dim3(N, p.nocc), nt, sc, st>>>(S, psi, Y, p);
  if (ev) cudaEventRecord(ev[3], st);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t run_domega_wave(const PairParams& p, const cplx_t<T>* psi, cplx_t<T>* S,
                            double* dacc, cudaStream_t st) {
  using C2 = cplx_t<T>;
  const int nt = threads_for(N);
  const int nf = p.nkp * p.nocc * p.nocc;
  const size_t sa = smem_a<N>(sizeof(C2));
  const size_t sb = smem_b<N>(sizeof(C2), sizeof(Axis1<T>));
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(pass_a<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    cudaFuncSetAttribute(pass_b_domega<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sb);
    configured = true;
  }
  pass_a<T, N><<<dim3(N, nf), nt, sa, st>>>(psi, S, p);
  pass_b_domega<T, N><<<dim3(N, nf), nt, sb, st>>>(S, p, dacc);
  return cudaGetLastError();
}

}  // namespace pairs

}  // namespace occri
