// occri_pairs.cuh -- kernel-fused FFT round trips of pair densities (steps c, d).
//
// For output k-point k, a block of k' and every occupied pair (i, j), the field
//   rho(r) = conj(psi_{jk'}(r)) psi_{ik}(r) e^{-iq.r},   q = k - k'      (Eq. aodf)
// is transformed, multiplied by v(|G+q|)/(4 pi) (Eqs. VGao, recipcoul) and
// transformed back; the potential W = e^{iq.r} u accumulates into
//   Y_{ik}(r) += psi_{jk'}(r) W(r)                                       (Eq. occrikinterm).
// The reversed pair (k', k, j, i) has the conjugate field and potential, so each
// unordered pair is transformed once and also feeds Y_{jk'} += psi_{ik} conj(W)
// (the tie-averaged kernel is inversion-symmetric, v_{-q}(-m) = v_q(m)).
//
// A cubic N^3 field does not fit on one SM, so a round trip takes three transform
// passes over a scratch field stored as S[f][m3][n1][m2] (third axis outermost),
// and one accumulation pass:
//   A: plane n1 -- form rho, FFT along n3 then n2, write column-major per m3;
//   B: plane m3 -- FFT along n1, kernel multiply, inverse along m1, inverse along m2;
//   C: plane n1 -- inverse along m3; the potential W overwrites the same addresses,
//      which leaves it in the fields' own point order (n3 N + n1) N + n2
//      (occri_internal.h);
//   D: per grid point, every field of the wave at once: Y_{ik} += sum_j W_ij psi_{jk'}
//      and Y_{jk'} += sum_i conj(W_ij) psi_{ik}, one read-modify-write of Y per wave.
// The orbitals and the accumulators are held as periodic parts (u_ik = e^{-ik.r} psi_ik,
// e^{-ik.r} Y_ik), so no pass multiplies by e^{-+iq.r}: the density conj(u_jk') u_ik is
// periodic, and so is the potential that comes back.
// Passes A-C move whole planes (coalesced) and keep one 1-D transform per thread
// (or per thread pair) in registers (fft_reg.cuh); the planes sit in shared memory
// with an odd pitch so that row and column accesses are conflict-free.
#pragma once

#include <algorithm>
#include <type_traits>

#include "fft_reg.cuh"
#include "occri_device.cuh"
#include "occri_internal.h"

namespace occri {
namespace pairs {

using dev::mk;
using dev::cmul;
using dev::cmulc;
using dev::cis_frac;
using dev::cis_frac_i;
using dev::exp_t;
using dev::expm1_t;

constexpr int pitch(int n) { return (n % 2 == 0) ? n + 1 : n; }
// Even edges use two threads per line (radix-2 split, see line_fft2), odd edges one.
constexpr int line_split(int n) { return (n % 2 == 0) ? 2 : 1; }
constexpr int round32(int n) { return (n + 31) / 32 * 32; }
// Where the two halves of a split line live. true: adjacent lanes of one warp, so that
// both halves' loads of the same element are one shared-memory broadcast (the
// half-dependent twiddle is then computed by both and selected). false: the halves of
// lines 32w..32w+31 in warps 2w (h = 0) and 2w + 1 (h = 1), half-dependent code uniform
// over each warp, every load its own shared-memory access.
constexpr bool kPairLanes = false;
constexpr int threads_for(int n) {
  return line_split(n) == 1 ? round32(n) : (kPairLanes ? round32(2 * n) : 2 * round32(n));
}
// resident CTAs per SM requested from the register allocator
constexpr int min_blocks(int n, int elem_bytes) {
  return elem_bytes > 8 ? (n <= 32 ? 4 : 2) : (n <= 32 ? 8 : 4);
}
// pass A (29 KB of shared memory at 60^3, FP32) runs six CTAs per SM (80 registers, no
// spills): 4 % faster than five at 60^3; a seventh (72 registers) was 7 % slower
constexpr int min_blocks_a(int n, int elem_bytes) {
  return elem_bytes > 8 ? min_blocks(n, elem_bytes) : (n <= 32 ? 8 : 6);
}
// f(|G+q|)/(4 pi) of Eq. recipcoul for |G+q|^2 = g2 = g2h + g2l > 0 (a hi + lo pair).
// The truncated Coulomb kernel (1 - cos(x R_c))/x^2 = 2 sin^2(x R_c/2)/x^2 is evaluated in
// FP64 from the pair in both precisions: x R_c reaches several hundred radians, where the
// FP32 argument alone would be off by 1e-5.
template <typename T>
__device__ __forceinline__ T kernel_f(T g2h, T g2l, int kind, T inv4w2, double rc) {
  if (kind == OCCRI_COULOMB_TRUNC) {
    const double g2 = (double)g2h + (double)g2l;
    const double s = sin(0.5 * sqrt(g2) * rc);
    return T(2.0 * s * s / g2);
  }
  const T g2 = g2h + g2l;
  const T base = T(1) / g2;
  if (kind == OCCRI_COULOMB) return base;
  const T y = g2 * inv4w2;
  if (kind == OCCRI_ERFC) return -base * expm1_t(-y);
  return base * exp_t(-y);
}

// f(|G+q|)/(4 pi) of the truncated erf kernel (Eq. lrtrunc) for |G+q|^2 = g2 > 0, in FP64:
//   [e^{-y} - e^{-omega^2 R_c^2} Re(e^{-i x R_c} w(z)) - erf(omega R_c) cos(x R_c)] / x^2,
// y = x^2/(4 omega^2), z = -x/(2 omega) + i omega R_c, with the Faddeeva function w from
// Weideman's rational approximation (coefficients made on the host).
__device__ __forceinline__ double kernel_lr_trunc(double g2, const PairParams& p) {
  const double x = sqrt(g2), w = p.omega, R = p.rc;
  const double zr = -x / (2.0 * w), zi = w * R;
  // d = L - i z, n = L + i z (i z = -zi + i zr)
  const double L = p.fad_L;
  const double dr = L + zi, di = -zr, nr = L - zi, ni = zr;
  const double den = dr * dr + di * di;
  const double Zr = (nr * dr + ni * di) / den, Zi = (ni * dr - nr * di) / den;
  double pr = p.fad_a[kFadN - 1], pi = 0.0;
#pragma unroll 4
  for (int n = kFadN - 2; n >= 0; --n) {
    const double tr = pr * Zr - pi * Zi + p.fad_a[n];
    pi = pr * Zi + pi * Zr;
    pr = tr;
  }
  const double ir = dr / den, ii = -di / den;            // 1/d
  const double i2r = ir * ir - ii * ii, i2i = 2.0 * ir * ii;
  constexpr double kInvSqrtPi = 0.56418958354775628694807945156077259;
  const double fr = 2.0 * (pr * i2r - pi * i2i) + kInvSqrtPi * ir;
  const double fi = 2.0 * (pr * i2i + pi * i2r) + kInvSqrtPi * ii;
  double sn, cs;
  sincos(x * R, &sn, &cs);
  const double t = exp(-g2 / (4.0 * w * w)) - p.lr_exp * (cs * fr + sn * fi);
  return (t - p.lr_erf * cs) / g2;
}

// (d f/d omega)/(4 pi) = -/+ e^{-x^2/(4 omega^2)} / (2 omega^3) (erfc / erf).
template <typename T>
__device__ __forceinline__ T kernel_df(T g2, int kind, T inv4w2, T omega) {
  if (kind != OCCRI_ERFC && kind != OCCRI_ERF) return T(0);
  const T e = exp_t(-g2 * inv4w2) * T(0.5) / (omega * omega * omega);
  return kind == OCCRI_ERFC ? -e : e;
}

// field f of the wave -> (k' offset, i, j); diagonal waves list i <= j row by row
struct FieldIdx { int kpl, i, j; };
__device__ __forceinline__ FieldIdx field_idx(int f, int nocc, int diag) {
  FieldIdx r;
  if (diag) {
    int i = 0, row = nocc;
    while (f >= row) { f -= row; ++i; --row; }
    r.kpl = 0; r.i = i; r.j = i + f;
    return r;
  }
  r.j = f % nocc;
  r.i = (f / nocc) % nocc;
  r.kpl = f / (nocc * nocc);
  return r;
}
__device__ __forceinline__ int diag_field(int i, int j, int nocc) {  // i <= j
  return i * nocc - i * (i - 1) / 2 + (j - i);
}

// First device error wins: record a bounded wait that gave up.
__device__ __forceinline__ void record_timeout(int* status) {
  if (status && atomicCAS(status, 0, (int)OCCRI_ETIMEOUT) == 0) status[1] = -1;
}

// ------------------------------------------------------------------ async plane staging
// cp.async copies global -> shared without staging through registers, so a whole
// plane is in flight per CTA. 4, 8 or 16 bytes, both addresses aligned to the size.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING));
}

// body(r, c) for every element of an N x N block, in a CTA of threads_for(N) threads:
// thread t < RT N takes column c = t mod N and rows t / N, t / N + RT, ... (RT = the
// threads_for(N) / N rows in flight), so the row is an induction variable and the
// addresses advance by constant steps instead of being re-derived from a flat index.
template <int N, typename F>
__device__ __forceinline__ void plane_loop(F&& body) {
  constexpr int RT = threads_for(N) / N;
  static_assert(RT >= 1, "a thread per column");
  const int t = threadIdx.x;
  if (t < RT * N) {
    const int c = t % N;
#pragma unroll 4
    for (int r = t / N; r < N; r += RT) body(r, c);
  }
}

// Copy a contiguous N x N plane into shared memory with row pitch P.
template <typename T, int N, int P>
__device__ __forceinline__ void stage_plane(cplx_t<T>* dst, const cplx_t<T>* src) {
  plane_loop<N>([&](int r, int c) { cp_async<sizeof(cplx_t<T>)>(dst + r * P + c, src + r * N + c); });
}

// ------------------------------------------------------------------ one line transform
// DFT (e^{-2 pi i m n / N}) of the N elements at base[m * stride], in place, with the
// whole line in registers. The unnormalised inverse (e^{+2 pi i m n / N}) is the same
// transform with output k stored at index (N - k) mod N. post(k, re, im) sees output
// index k (after that reversal) before the store (store is skipped when !store). Every
// call site has its own unrolled copy with a compile-time stride, so no address is
// computed at run time from a stride.
template <typename T, int N, typename Post>
__device__ __forceinline__ void line_fft(cplx_t<T>* base, int stride, bool inverse, bool store,
                                         Post&& post) {
  if constexpr (std::is_same<T, float>::value) {   // packed FP32 core
    fft::pk::u64 x[N];
    fft::static_for<N>([&](auto I) {
      constexpr int m = decltype(I)::value;
      const float2 v = base[m * stride];
      x[m] = fft::pk::pack(v.x, v.y);
    });
    fft::pfft_dif<N, -1>(x);
    fft::static_for<N>([&](auto I) {
      constexpr int q = decltype(I)::value;
      constexpr int k = fft::dif_rev(N, q);
      constexpr int kr = (N - k) % N;
      const int ks = inverse ? kr : k;
      float re, im;
      fft::pk::unpack(x[q], re, im);
      post(ks, re, im);
      if (store) base[ks * stride] = mk<T>(re, im);
    });
  } else {
    T re[N], im[N];
    fft::static_for<N>([&](auto I) {
      constexpr int m = decltype(I)::value;
      const cplx_t<T> v = base[m * stride];
      re[m] = v.x;
      im[m] = v.y;
    });
    fft::fft_dif<N, -1>(re, im);
    fft::static_for<N>([&](auto I) {
      constexpr int q = decltype(I)::value;
      constexpr int k = fft::dif_rev(N, q);
      constexpr int kr = (N - k) % N;
      const int ks = inverse ? kr : k;
      post(ks, re[q], im[q]);
      if (store) base[ks * stride] = mk<T>(re[q], im[q]);
    });
  }
}

// Two threads per line (even N), adjacent lanes or two warps (kPairLanes). Half h forms
//   y_h[n] = (x[n] + (-1)^h x[n + N/2]) e^{-2 pi i h n / N},   n < N/2,
// from the whole line in shared memory and transforms it with an N/2-point register
// FFT, which gives the outputs X[2k + h] (radix-2 decimation in frequency). inverse,
// store and post as in line_fft; `valid` is false for padding threads, which compute
// on a duplicate line but neither store nor call post. The pair synchronises between
// its loads and its stores: __syncwarp for adjacent lanes, else named barrier `bar`
// (1 or 2: at most two pairs of warps per CTA, N <= 64), or with bar = 0 the whole CTA
// (every thread of the CTA then calls it).
struct NoMid {
  __device__ __forceinline__ void operator()() const {}
};

template <typename T, int N, typename Post, typename Mid = NoMid>
__device__ __forceinline__ void line_fft2(cplx_t<T>* base, int stride, bool inverse, bool store,
                                          int h, bool valid, int bar, Post&& post,
                                          Mid&& mid = Mid()) {
  constexpr int M = N / 2;
  auto pair_barrier = [&]() {
    if constexpr (kPairLanes) {
      __syncwarp();
    } else if (bar == 0) {   // warp-uniform; immediate barrier ids
      __syncthreads();
    } else if (bar == 1) {
      asm volatile("bar.sync 1, 64;\n" ::: "memory");
    } else {
      asm volatile("bar.sync 2, 64;\n" ::: "memory");
    }
  };
  if constexpr (std::is_same<T, float>::value) {   // packed FP32 core
    using fft::pk::u64;
    u64 x[M];
    if constexpr (kPairLanes) {   // both halves in one warp: no branch on h
      fft::static_for<M>([&](auto I) {
        constexpr int n = decltype(I)::value;
        constexpr fft::CS w = fft::cs2pi(n, N);     // e^{-2 pi i n / N} = c - i s
        const float2 a = base[n * stride], b = base[(n + M) * stride];
        const u64 pa = fft::pk::pack(a.x, a.y), pb = fft::pk::pack(b.x, b.y);
        if constexpr (n == 0) {
          x[n] = h ? fft::pk::sub(pa, pb) : fft::pk::add(pa, pb);
        } else {
          const u64 t = fft::pk::cmul_const(fft::pk::sub(pa, pb), float(w.c), float(-w.s));
          x[n] = h ? t : fft::pk::add(pa, pb);
        }
      });
    } else if (h == 0) {
      fft::static_for<M>([&](auto I) {
        constexpr int n = decltype(I)::value;
        const float2 a = base[n * stride], b = base[(n + M) * stride];
        x[n] = fft::pk::add(fft::pk::pack(a.x, a.y), fft::pk::pack(b.x, b.y));
      });
    } else {
      fft::static_for<M>([&](auto I) {
        constexpr int n = decltype(I)::value;
        constexpr fft::CS w = fft::cs2pi(n, N);     // e^{-2 pi i n / N} = c - i s
        const float2 a = base[n * stride], b = base[(n + M) * stride];
        const u64 d = fft::pk::sub(fft::pk::pack(a.x, a.y), fft::pk::pack(b.x, b.y));
        if constexpr (n == 0)
          x[n] = d;
        else
          x[n] = fft::pk::cmul_const(d, float(w.c), float(-w.s));
      });
    }
    pair_barrier();
    mid();   // every line of the CTA is in registers when bar == 0
    fft::pfft_dif<M, -1>(x);
    fft::static_for<M>([&](auto I) {
      constexpr int q = decltype(I)::value;
      const int k = 2 * fft::dif_rev(M, q) + h;
      const int ks = inverse ? (k == 0 ? 0 : N - k) : k;
      if (valid) {
        float re, im;
        fft::pk::unpack(x[q], re, im);
        post(ks, re, im);
        if (store) base[ks * stride] = mk<T>(re, im);
      }
    });
  } else {
    T re[M], im[M];
    if (h == 0) {
      fft::static_for<M>([&](auto I) {
        constexpr int n = decltype(I)::value;
        const cplx_t<T> a = base[n * stride], b = base[(n + M) * stride];
        re[n] = a.x + b.x;
        im[n] = a.y + b.y;
      });
    } else {
      fft::static_for<M>([&](auto I) {
        constexpr int n = decltype(I)::value;
        constexpr fft::CS w = fft::cs2pi(n, N);     // e^{-2 pi i n / N} = c - i s
        const cplx_t<T> a = base[n * stride], b = base[(n + M) * stride];
        const T yr = a.x - b.x, yi = a.y - b.y;
        if constexpr (n == 0) {
          re[n] = yr;
          im[n] = yi;
        } else {
          re[n] = yr * T(w.c) + yi * T(w.s);
          im[n] = yi * T(w.c) - yr * T(w.s);
        }
      });
    }
    pair_barrier();
    mid();   // every line of the CTA is in registers when bar == 0
    fft::fft_dif<M, -1>(re, im);
    fft::static_for<M>([&](auto I) {
      constexpr int q = decltype(I)::value;
      const int k = 2 * fft::dif_rev(M, q) + h;
      const int ks = inverse ? (k == 0 ? 0 : N - k) : k;
      if (valid) {
        post(ks, re[q], im[q]);
        if (store) base[ks * stride] = mk<T>(re[q], im[q]);
      }
    });
  }
}

// One transform job over the N lines of a plane (rows: along the contiguous index;
// columns: along the pitched index); every thread of the CTA must call it.
// As run_lines for even N, with the pair barrier made CTA-wide and mid() called after it by
// every thread: the plane in shared memory is free from then on (every line is in registers).
template <typename T, int N, typename Post, typename Mid>
__device__ __forceinline__ void run_lines_then(cplx_t<T>* plane, int P, bool rows, bool inverse,
                                               Post&& post, Mid&& mid) {
  static_assert(line_split(N) == 2, "even edges");
  const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int line0 = kPairLanes ? (int)threadIdx.x >> 1 : (w >> 1) * 32 + lane;
  const int h = kPairLanes ? (int)threadIdx.x & 1 : w & 1;
  const bool valid = line0 < N;
  const int line = valid ? line0 : N - 1;
  line_fft2<T, N>(rows ? plane + line * P : plane + line, rows ? 1 : P, inverse, false, h, valid,
                  0, [&](int k, T& re, T& im) { post(line, k, re, im); }, mid);
}

template <typename T, int N, typename Post>
__device__ __forceinline__ void run_lines(cplx_t<T>* plane, int P, bool rows, bool inverse,
                                          bool store, Post&& post) {
  if constexpr (line_split(N) == 2) {
    const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int line0 = kPairLanes ? (int)threadIdx.x >> 1 : (w >> 1) * 32 + lane;
    const int h = kPairLanes ? (int)threadIdx.x & 1 : w & 1;
    const bool valid = line0 < N;
    const int line = valid ? line0 : N - 1;
    line_fft2<T, N>(rows ? plane + line * P : plane + line, rows ? 1 : P, inverse, store, h,
                    valid, 1 + (w >> 1), [&](int k, T& re, T& im) { post(line, k, re, im); });
  } else {
    if (threadIdx.x < N) {
      const int line = threadIdx.x;
      line_fft<T, N>(rows ? plane + line * P : plane + line, rows ? 1 : P, inverse, store,
                     [&](int k, T& re, T& im) { post(line, k, re, im); });
    }
  }
}

// ------------------------------------------------------------------ kernel values per bin
// Per-CTA table for axis 1 and per-column constants for axes 2, 3 give, for the first
// alias of every axis,
//   |G+q|^2 = a1(m1) + x1(m1) * beta + gamma,  a1 = g11 x1^2,
//   beta = 2 (g12 x2 + g13 x3),  gamma = g22 x2^2 + 2 g23 x2 x3 + g33 x3^2,
// all formed in the working precision: in FP32 the metric is a hi/lo pair and every
// product is error-free (two-product by FMA), so no rounding biases all bins alike and
// no FP64 instruction (1/64 rate) is issued. Bins with an exact tie on some axis, or
// G+q = 0, go to one out-of-line function (flags: bit0 tie, bit1 zero coordinate).

// Reduced coordinate of bin m on one axis as the exact integer X = x*D in
// [-N*D/2, N*D/2), plus tie and zero flags (all integer, |X| < 2^12).
struct AxisInt {
  int X, D, N;
  bool tie, zero;
};
__device__ __forceinline__ AxisInt axis_int(int m, int Q, int D, int N) {
  const int P = N * D;
  int X = m * D + Q;           // |Q| < D, so X in (-P, 2P)
  // subtract P*floor(X/P + 1/2)
  const int twice = 2 * X + P;
  const int fl = (twice >= 0) ? twice / (2 * P) : -((-twice + 2 * P - 1) / (2 * P));
  X -= P * fl;
  AxisInt r;
  r.X = X; r.D = D; r.N = N;
  r.tie = (2 * X == -P);
  r.zero = (X == 0);
  return r;
}
template <typename T> __device__ __forceinline__ T axis_x(const AxisInt& a, bool second) {
  return T(second ? a.X + a.N * a.D : a.X) / T(a.D);
}

// hi/lo parts of the reciprocal metric g_ij (lo = 0 in FP64), and the other launch
// constants in the working precision, read without any double -> float conversion
template <typename T> struct Consts;
template <> struct Consts<double> {
  double h[6], l[6], inv4w2, omega, g0, dg0;
  __device__ __forceinline__ explicit Consts(const PairParams& p) {
#pragma unroll
    for (int i = 0; i < 6; ++i) { h[i] = p.g[i]; l[i] = 0.0; }
    inv4w2 = p.inv4w2; omega = p.omega; g0 = p.g0; dg0 = p.dg0;
  }
};
template <> struct Consts<float> {
  float h[6], l[6], inv4w2, omega, g0, dg0;
  __device__ __forceinline__ explicit Consts(const PairParams& p) {
#pragma unroll
    for (int i = 0; i < 6; ++i) { h[i] = p.gh[i]; l[i] = p.gl[i]; }
    inv4w2 = p.inv4w2_f; omega = p.omega_f; g0 = p.g0_f; dg0 = p.dg0_f;
  }
};
template <typename T> using MetricHL = Consts<T>;

// s (hi, lo) += g * a * b with g = (gh, gl), error-free in the product a*b.
template <typename T>
__device__ __forceinline__ void acc_gab(T gh, T gl, T a, T b, T& hi, T& lo) {
  const T ph = a * b;
  const T pl = fma(a, b, -ph);
  const T t = gh * ph;
  lo += fma(gh, ph, -t) + gh * pl + gl * ph;
  const T s = hi + t;                       // two-sum of hi + t
  const T bb = s - hi;
  lo += (hi - (s - bb)) + (t - bb);
  hi = s;
}

template <typename T>
struct Axis1 {
  T x, ah, al;     // first alias: x and g11 x^2 (hi, lo)
  T xb, bh, bl;    // second alias (== first unless tied)
  int flags;       // bit0 tie, bit1 x == 0
};

template <typename T>
__device__ __forceinline__ Axis1<T> axis1_entry(const Consts<T>& g, const AxisInt& a) {
  Axis1<T> r;
  r.x = axis_x<T>(a, false);
  r.xb = axis_x<T>(a, a.tie);
  T hi = T(0), lo = T(0);
  acc_gab<T>(g.h[0], g.l[0], r.x, r.x, hi, lo);
  r.ah = hi; r.al = lo;
  hi = T(0); lo = T(0);
  acc_gab<T>(g.h[0], g.l[0], r.xb, r.xb, hi, lo);
  r.bh = hi; r.bl = lo;
  r.flags = (a.tie ? 1 : 0) | (a.zero ? 2 : 0);
  return r;
}

// Column constants for up to four (x2, x3) alias variants; nv distinct ones first.
template <typename T>
struct ColumnConst {
  T bh[4], bl[4], ch[4], cl[4];
  int nv;
  int zero;  // x2 == 0 and x3 == 0
};

template <typename T>
__device__ __forceinline__ ColumnConst<T> column_const(const Consts<T>& g, const AxisInt& b,
                                                       const AxisInt& c) {
  ColumnConst<T> r;
  r.nv = (b.tie ? 2 : 1) * (c.tie ? 2 : 1);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    // u -> (alias of x2, alias of x3), listing only the tied axes' second aliases
    const bool s2 = b.tie && (u & 1);
    const bool s3 = c.tie && (b.tie ? (u & 2) : (u & 1));
    const T x2 = axis_x<T>(b, s2), x3 = axis_x<T>(c, s3);
    T bh = T(0), bl = T(0);   // beta = 2 g12 x2 + 2 g13 x3
    acc_gab<T>(g.h[3], g.l[3], T(2), x2, bh, bl);
    acc_gab<T>(g.h[4], g.l[4], T(2), x3, bh, bl);
    T ch = T(0), cl = T(0);   // gamma = g22 x2^2 + g33 x3^2 + 2 g23 x2 x3
    acc_gab<T>(g.h[1], g.l[1], x2, x2, ch, cl);
    acc_gab<T>(g.h[2], g.l[2], x3, x3, ch, cl);
    acc_gab<T>(g.h[5], g.l[5], T(2) * x2, x3, ch, cl);
    r.bh[u] = bh; r.bl[u] = bl; r.ch[u] = ch; r.cl[u] = cl;
  }
  r.zero = (b.zero && c.zero) ? 1 : 0;
  return r;
}

// v/(4 pi) (or its omega-derivative) on one bin, averaged over tied aliases. Called from
// a rolled loop, so the variant handling is inline without growing the unrolled code.
template <typename T, bool DERIV>
__device__ __forceinline__ T bin_value(const PairParams& p, const Consts<T>& k,
                                       const Axis1<T>& a, const ColumnConst<T>& c) {
  if ((a.flags & 2) && c.zero) return DERIV ? k.dg0 : k.g0;
  auto f = [&](T g2h, T g2l) {
    if (!DERIV && p.kind == OCCRI_ERF_TRUNC)
      return T(kernel_lr_trunc((double)g2h + (double)g2l, p));
    return DERIV ? kernel_df<T>(g2h + g2l, p.kind, k.inv4w2, k.omega)
                 : kernel_f<T>(g2h, g2l, p.kind, k.inv4w2, p.rc);
  };
  const bool t1 = (a.flags & 1) != 0;
  T s = T(0);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (u < c.nv) {
      s += f(a.ah + a.x * c.bh[u] + c.ch[u], a.al + a.x * c.bl[u] + c.cl[u]);
      if (t1) s += f(a.bh + a.xb * c.bh[u] + c.ch[u], a.bl + a.xb * c.bl[u] + c.cl[u]);
    }
  }
  return (c.nv == 1 && !t1) ? s : s / T(c.nv * (t1 ? 2 : 1));
}

// v/(4 pi) (DERIV: its omega-derivative) on the bins (m1, m2) of plane m3 for the wave's
// k' = kp0 + kpl: out[m1 N + m2], rows m1 = r0, r0 + rs, ... of every column. ax1 is an
// N-entry scratch table in shared memory; every thread of the CTA calls this (one
// __syncthreads inside, between the axis-1 table and its use).
template <typename T, int N, bool DERIV>
__device__ __forceinline__ void fill_vtab_q(const PairParams& p, const MetricHL<T>& gm, int m3,
                                            const int (&Q)[3], Axis1<T>* ax1, T* out, int r0,
                                            int rs) {
  for (int t = threadIdx.x; t < N; t += blockDim.x)
    ax1[t] = axis1_entry<T>(gm, axis_int(t, Q[0], p.D[0], N));
  __syncthreads();
  // one rolled loop per column (split between the line's threads)
  constexpr int SP = line_split(N);
  const int c = (int)threadIdx.x / SP, h = (int)threadIdx.x % SP;
  if (c < N) {
    const ColumnConst<T> cc = column_const<T>(gm, axis_int(c, Q[1], p.D[1], N),
                                              axis_int(m3, Q[2], p.D[2], N));
#pragma unroll 1
    for (int m1 = r0 + h * rs; m1 < N; m1 += SP * rs)
      out[m1 * N + c] = bin_value<T, DERIV>(p, gm, ax1[m1], cc);
  }
}

// The same for the wave's k' = kp0 + kpl: q = k - k' is Q / D per axis.
template <typename T, int N, bool DERIV>
__device__ __forceinline__ void fill_vtab(const PairParams& p, const MetricHL<T>& gm, int m3,
                                          int kpl, Axis1<T>* ax1, T* out, int r0, int rs) {
  const int kp = p.kp0 + kpl;
  int Q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) Q[d] = p.kint[p.k * 3 + d] - p.kint[kp * 3 + d];
  fill_vtab_q<T, N, DERIV>(p, gm, m3, Q, ax1, out, r0, rs);
}

// The plan's kernel tables: one per integer difference Q = kint[k] - kint[k'], each axis
// in -(D - 1) .. D - 1, stored in row-major (Q_1, Q_2, Q_3) order, each [m3][m1][m2].
// Table index of the wave's k' = kp0 + kpl.
__device__ __forceinline__ long long qtab_index(const PairParams& p, int kpl) {
  const int kp = p.kp0 + kpl;
  long long idx = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    idx = idx * (2 * p.D[d] - 1) + (p.kint[p.k * 3 + d] - p.kint[kp * 3 + d] + p.D[d] - 1);
  return idx;
}

// The wave's kernel tables vt[kpl][m3][m1][m2] = v/(4 pi), once per wave, for pass B to
// copy plane by plane (instead of every pass-B CTA forming the planes it meets). CTA
// (m3, kpl, z) fills rows m1 = z (mod kVtabSplit) of plane m3.
constexpr int kVtabSplit = 4;
template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N))
vtab_kernel(T* __restrict__ vt, PairParams p) {
  __shared__ Axis1<T> ax1[N];
  const int m3 = blockIdx.x, kpl = blockIdx.y;
  const MetricHL<T> gm(p);
  fill_vtab<T, N, false>(p, gm, m3, kpl, ax1, vt + ((size_t)kpl * N + m3) * N * N,
                         (int)blockIdx.z, kVtabSplit);
}

// The plan's kernel tables (qtab_index order), once at plan creation: CTA (t, m3, z) fills
// rows m1 = z (mod kVtabSplit) of plane m3 of table t.
template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N))
qtab_kernel(T* __restrict__ vq, PairParams p) {
  __shared__ Axis1<T> ax1[N];
  const int m3 = blockIdx.y;
  long long t = blockIdx.x;
  int Q[3];
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    const int w = 2 * p.D[d] - 1;
    Q[d] = (int)(t % w) - (p.D[d] - 1);
    t /= w;
  }
  const MetricHL<T> gm(p);
  fill_vtab_q<T, N, false>(p, gm, m3, Q, ax1, vq + ((size_t)blockIdx.x * N + m3) * N * N,
                           (int)blockIdx.z, kVtabSplit);
}

// ------------------------------------------------------------------ pass A
// plane n1 of field (i, j): rho = conj(u_jk') u_ik (= conj(psi_jk') psi_ik e^{-iq.r}, the
// orbitals being held as their periodic parts u); FFT along n3, then n2.
// With ADJ (the adjoint build): the field is sigma = conj(u_jk') g_ik + conj(g_jk') u_ik,
// g being the adjoint orbital field, i.e. the change of rho when u moves along g.
template <typename T, int N, bool ADJ = false>
__global__ void __launch_bounds__(threads_for(N), min_blocks_a(N, sizeof(cplx_t<T>)))
pass_a(const cplx_t<T>* __restrict__ psi, cplx_t<T>* __restrict__ S, PairParams p,
       const cplx_t<T>* __restrict__ gam = nullptr, T* __restrict__ vt = nullptr) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (vt != nullptr) {
    // CTAs past the wave's fields fill the wave's kernel tables vt[kpl][m3][m1][m2] (rows
    // m1 = z mod kVtabSplit of plane m3 = blockIdx.x), alongside the density transforms
    const int nf = wave_fields(p.nocc, p.nkp, p.diag);
    if ((int)blockIdx.y >= nf) {
      const int y = (int)blockIdx.y - nf;
      const int kpl = y / kVtabSplit, z = y % kVtabSplit, m3 = blockIdx.x;
      const MetricHL<T> gm(p);
      fill_vtab<T, N, false>(p, gm, m3, kpl, reinterpret_cast<Axis1<T>*>(smem_raw),
                             vt + ((size_t)kpl * N + m3) * N * N, z, kVtabSplit);
      return;
    }
  }
  C2* pl = reinterpret_cast<C2*>(smem_raw);   // rho, then its 2-D transform
  const int n1 = blockIdx.x;
  const int f = blockIdx.y;
  const FieldIdx fi = field_idx(f, p.nocc, p.diag);
  const int kp = p.kp0 + fi.kpl;
  // plane n1 of the periodic parts: N rows (n3) of N contiguous points (n2)
  const C2* pi = psi + (size_t)(p.k * p.nocc + fi.i) * p.fs + (size_t)n1 * N;
  const C2* pj = psi + (size_t)(kp * p.nocc + fi.j) * p.fs + (size_t)n1 * N;
  if constexpr (ADJ) {
    const C2* gi = gam + (size_t)(p.k * p.nocc + fi.i) * p.fs + (size_t)n1 * N;
    const C2* gj = gam + (size_t)(kp * p.nocc + fi.j) * p.fs + (size_t)n1 * N;
    plane_loop<N>([&](int n3, int n2) {
      const size_t off = (size_t)n3 * N * N + n2;
      const C2 a = cmulc<T>(__ldg(pj + off), __ldg(gi + off));
      const C2 b = cmulc<T>(__ldg(gj + off), __ldg(pi + off));
      pl[n2 * P + n3] = mk<T>(a.x + b.x, a.y + b.y);
    });
  } else if constexpr (std::is_same<T, float>::value && N % 2 == 0) {
    // two points per 16-byte load: N/2 threads per row, more bytes in flight per thread
    // (every plane row starts 16-byte aligned: fs, N and the column are even)
    constexpr int H = N / 2;
    constexpr int RT2 = threads_for(N) / H;
    const int t = threadIdx.x;
    if (t < RT2 * H) {
      const int c = 2 * (t % H);
      const float4* pj4 = reinterpret_cast<const float4*>(pj);
      const float4* pi4 = reinterpret_cast<const float4*>(pi);
#pragma unroll 4
      for (int r = t / H; r < N; r += RT2) {
        const size_t off = ((size_t)r * N * N + c) / 2;
        const float4 a = __ldg(pj4 + off), b = __ldg(pi4 + off);
        pl[c * P + r] = cmulc<T>(make_float2(a.x, a.y), make_float2(b.x, b.y));
        pl[(c + 1) * P + r] = cmulc<T>(make_float2(a.z, a.w), make_float2(b.z, b.w));
      }
    }
  } else {
    plane_loop<N>([&](int n3, int n2) {
      const size_t off = (size_t)n3 * N * N + n2;
      pl[n2 * P + n3] = cmulc<T>(__ldg(pj + off), __ldg(pi + off));
    });
  }
  __syncthreads();
  // columns (line n3, along n2), then rows (line m2, along n3); the rows' outputs go
  // straight to S[f][m3][n1][m2], a warp's lanes on consecutive m2
  run_lines<T, N>(pl, P, false, false, true, [](int, int, T&, T&) {});
  __syncthreads();
  C2* out = S + (size_t)f * p.fs;
  run_lines<T, N>(pl, P, true, false, false, [&](int line, int k, T& re, T& im) {
    out[((size_t)k * N + n1) * N + line] = mk<T>(re, im);
  });
}

// ------------------------------------------------------------------ pass B
// Items (m3, field), m3-major; CTA b takes the contiguous chunk [b c, (b + 1) c) of
// them (c = ceil(items / grid), the grid being the SMs' resident CTA slots), so there is
// no partly filled last round of CTAs. Per item: FFT along n1, multiply by v/(4 pi),
// inverse along m2, inverse along m1. Consecutive items share m3 and (mostly) q, so a
// plane of kernel values is copied in (from the wave's tables, vt) only when (m3, k')
// changes, in the same cp.async group as the item's plane. One plane buffer per CTA: a
// fourth CTA per SM hides the copies better than a second buffer did.
// With DOMEGA: the forward part only, accumulating sum_m (dv/d omega)/(4 pi) |rho^(m)|^2,
// with the derivative's kernel values formed in the CTA.
template <typename T, int N>
__device__ __forceinline__ void copy_table(T* dst, const T* src) {
  // even N: N^2 values are a whole number of 16-byte pieces, and every plane of the
  // tables and of the shared-memory layout starts 16-byte aligned
  constexpr int BYTES = (N % 2 == 0) ? 16 : (int)sizeof(T);
  constexpr int PER = BYTES / (int)sizeof(T);
  for (int e = threadIdx.x; e < N * N / PER; e += blockDim.x)
    cp_async<BYTES>(dst + e * PER, src + e * PER);
}

template <typename T, int N, bool DOMEGA>
__device__ __forceinline__ void pass_b_body(cplx_t<T>* __restrict__ S, const PairParams& p,
                                            const T* __restrict__ vt, double* dacc) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* plane = reinterpret_cast<C2*>(smem_raw);                 // [n1][m2]
  T* vtab = reinterpret_cast<T*>(plane + N * P);               // [m1][m2] v or dv
  Axis1<T>* ax1 = reinterpret_cast<Axis1<T>*>(vtab + N * N);   // [m1] (DOMEGA)
  __shared__ double red[4];
  const int nf = wave_fields(p.nocc, p.nkp, p.diag);
  const int items = N * nf;
  const int per = (items + (int)gridDim.x - 1) / (int)gridDim.x;
  const int i0 = min(items, (int)blockIdx.x * per);
  const int i1 = min(items, i0 + per);
  const MetricHL<T> gm(p);
  int m3_tab = -1, kpl_tab = -1;
  // the item's plane and, where (m3, k') changes, its plane of kernel values
  auto stage = [&](int it) {
    const int m3 = it / nf, f = it - (it / nf) * nf;
    stage_plane<T, N, P>(plane, S + (size_t)f * p.fs + (size_t)m3 * N * N);
    if constexpr (!DOMEGA) {
      const int kpl = field_idx(f, p.nocc, p.diag).kpl;
      if (m3 != m3_tab || kpl != kpl_tab) {   // uniform over the CTA
        m3_tab = m3;
        kpl_tab = kpl;
        const T* tab = p.vq ? static_cast<const T*>(p.vq) + (size_t)qtab_index(p, kpl) * N * N * N
                            : vt + (size_t)kpl * N * N * N;
        copy_table<T, N>(vtab, tab + (size_t)m3 * N * N);
      }
    }
  };
  if (i0 < i1) stage(i0);
  cp_async_commit();
  T dsum = T(0);
#pragma unroll 1
  for (int it = i0; it < i1; ++it) {
    const int m3 = it / nf, f = it - (it / nf) * nf;
    const FieldIdx fi = field_idx(f, p.nocc, p.diag);
    if constexpr (DOMEGA) {
      if (fi.kpl != kpl_tab || m3 != m3_tab) {   // uniform over the CTA
        kpl_tab = fi.kpl;
        m3_tab = m3;
        fill_vtab<T, N, true>(p, gm, m3, fi.kpl, ax1, vtab, 0, 1);
      }
    }
    cp_async_wait<0>();   // this item's plane (and table) have landed
    __syncthreads();
    // an unordered pair stands for itself and its reverse, except (k, k, i, i)
    const T wgt = (p.diag && fi.i == fi.j) ? T(1) : T(2);
    // columns (m2 = line): forward along n1, times v (the only forward transform, so its
    // output indices are constants)
    run_lines<T, N>(plane, P, false, false, !DOMEGA, [&](int line, int k, T& re, T& im) {
      const T v = vtab[k * N + line];
      if constexpr (DOMEGA) {
        dsum += wgt * v * (re * re + im * im);
      } else {
        re *= v;
        im *= v;
      }
    });
    __syncthreads();
    if constexpr (!DOMEGA) {
      // inverse along m2 (rows), then along m1 (columns); the columns' outputs go straight
      // to S[f][m3][n1][n2], a warp's lanes on consecutive n2
      run_lines<T, N>(plane, P, true, true, true, [](int, int, T&, T&) {});
      __syncthreads();
      C2* buf = S + (size_t)f * p.fs + (size_t)m3 * N * N;
      auto out = [&](int line, int k, T& re, T& im) { buf[(size_t)k * N + line] = mk<T>(re, im); };
      if constexpr (line_split(N) == 2) {
        // the next item's copies start as soon as every line of this last transform is in
        // registers, and overlap its arithmetic and stores
        run_lines_then<T, N>(plane, P, false, true, out, [&]() {
          if (it + 1 < i1) stage(it + 1);
          cp_async_commit();
        });
      } else {
        run_lines<T, N>(plane, P, false, true, false, out);
        __syncthreads();   // releases the buffers for the next item's copies
        if (it + 1 < i1) stage(it + 1);
        cp_async_commit();
      }
    } else {
      if (it + 1 < i1) stage(it + 1);
      cp_async_commit();
    }
  }
  if constexpr (DOMEGA) {
    double part = double(dsum);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(dacc, t);
    }
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N), min_blocks(N, sizeof(cplx_t<T>)))
pass_b(cplx_t<T>* __restrict__ S, PairParams p, const T* __restrict__ vt) {
  pass_b_body<T, N, false>(S, p, vt, nullptr);
}

template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N), min_blocks(N, sizeof(cplx_t<T>)))
pass_b_domega(cplx_t<T>* __restrict__ S, PairParams p, double* dacc) {
  pass_b_body<T, N, true>(S, p, nullptr, dacc);
}

// Resident CTA slots of a kernel on this device (SMs x CTAs per SM), at least 1.
template <typename K>
int resident_slots(K kernel, int threads, size_t smem) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  return std::max(1, nsm * std::max(1, per));
}

// ------------------------------------------------------------------ pass C
// plane n1 of a field: inverse along m3, written back over the rows it was read from,
// S[f][n3][n1][n2]. This is the periodic part e^{-iq.r} W of the potential, which is
// what the accumulation of periodic parts needs.
template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N), min_blocks(N, sizeof(cplx_t<T>)))
pass_c(cplx_t<T>* __restrict__ S, PairParams p) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* cur = reinterpret_cast<C2*>(smem_raw);  // [m3][n2], pitch P
  const int n1 = blockIdx.x;
  const int f = blockIdx.y;
  C2* rows = S + (size_t)f * p.fs + (size_t)n1 * N;   // row m3 at rows + m3 N^2
  plane_loop<N>([&](int m3, int n2) {
    cp_async<sizeof(C2)>(cur + m3 * P + n2, rows + (size_t)m3 * N * N + n2);
  });
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  // columns (n2 = line): inverse along m3
  run_lines<T, N>(cur, P, false, true, true, [](int, int, T&, T&) {});
  __syncthreads();
  plane_loop<N>([&](int n3, int n2) { rows[(size_t)n3 * N * N + n2] = cur[n3 * P + n2]; });
}

// ------------------------------------------------------------------ pass D
// One thread per grid point r (fields' point order). For the wave (k, k' in
// [kp0, kp0 + nkp)) with potentials W_f(r) of the fields f = (k', i, j):
//   Y_{ik}(r)  += sum_{k', j} W_{k'ij}(r) psi_{jk'}(r)       (Eq. occrikinterm)
//   Y_{jk'}(r) += sum_i conj(W_{k'ij}(r)) psi_{ik}(r)        (the reversed pair)
// and for a diagonal wave (k, k) with fields i <= j, W_ji = conj(W_ij). All of it runs on
// periodic parts (u = e^{-ik.r} psi, e^{-iq.r} W, e^{-ik.r} Y), for which the same
// relations hold with every phase factor cancelled. NOC >= nocc
// is a compile-time bound so that both sets of per-orbital sums stay in registers;
// the loop body is loads and FMAs only, so the loads of many fields are in flight.
template <typename T, int NOC>
__global__ void __launch_bounds__(256, NOC <= 8 ? 2 : 1)
pass_d(const cplx_t<T>* __restrict__ S, const cplx_t<T>* __restrict__ psi,
       cplx_t<T>* __restrict__ Y, PairParams p) {
  using C2 = cplx_t<T>;
  const long long ng = p.ng;
  const int nocc = p.nocc;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng;
       r += (long long)gridDim.x * blockDim.x) {
    T pr[NOC], pim[NOC], ar[NOC], ai[NOC];
#pragma unroll
    for (int i = 0; i < NOC; ++i) {
      C2 v = mk<T>(T(0), T(0));
      if (i < nocc) v = __ldg(psi + (size_t)(p.k * nocc + i) * p.fs + r);
      pr[i] = v.x; pim[i] = v.y;
      ar[i] = T(0); ai[i] = T(0);
    }
    if (p.diag) {
#pragma unroll
      for (int j = 0; j < NOC; ++j) {
        if (j >= nocc) break;
#pragma unroll
        for (int i = 0; i <= j; ++i) {
          const C2 w = __ldg(S + (size_t)diag_field(i, j, nocc) * p.fs + r);
          ar[i] += w.x * pr[j] - w.y * pim[j];     // W_ij psi_j
          ai[i] += w.x * pim[j] + w.y * pr[j];
          if (i < j) {                             // W_ji psi_i = conj(W_ij) psi_i
            ar[j] += w.x * pr[i] + w.y * pim[i];
            ai[j] += w.x * pim[i] - w.y * pr[i];
          }
        }
      }
    } else {
#pragma unroll 1
      for (int kpl = 0; kpl < p.nkp; ++kpl) {
        const int kp = p.kp0 + kpl;
        const C2* wk = S + (size_t)kpl * nocc * nocc * p.fs + r;
        T qr[NOC], qi[NOC], br[NOC], bi[NOC];
#pragma unroll
        for (int j = 0; j < NOC; ++j) {
          C2 v = mk<T>(T(0), T(0));
          if (j < nocc) v = __ldg(psi + (size_t)(kp * nocc + j) * p.fs + r);
          qr[j] = v.x; qi[j] = v.y;
          br[j] = T(0); bi[j] = T(0);
        }
#pragma unroll
        for (int i = 0; i < NOC; ++i) {
          if (i >= nocc) break;
#pragma unroll
          for (int j = 0; j < NOC; ++j) {
            if (j >= nocc) break;
            const C2 w = __ldg(wk + (size_t)(i * nocc + j) * p.fs);
            ar[i] += w.x * qr[j] - w.y * qi[j];     // W psi_{jk'}
            ai[i] += w.x * qi[j] + w.y * qr[j];
            br[j] += w.x * pr[i] + w.y * pim[i];    // conj(W) psi_{ik}
            bi[j] += w.x * pim[i] - w.y * pr[i];
          }
        }
#pragma unroll
        for (int j = 0; j < NOC; ++j) {
          if (j >= nocc) break;
          C2* y = Y + (size_t)(kp * nocc + j) * p.fs + r;
          C2 v = *y;
          v.x += br[j];
          v.y += bi[j];
          *y = v;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NOC; ++i) {
      if (i >= nocc) break;
      C2* y = Y + (size_t)(p.k * nocc + i) * p.fs + r;
      C2 v = *y;
      v.x += ar[i];
      v.y += ai[i];
      *y = v;
    }
  }
}

// ------------------------------------------------------------------ pass D, bulk-copy form
// The same accumulation with every operand moved by the bulk-copy (TMA) engine, in tiles
// of kBulkTile consecutive points. For a tile, one producer thread (the last warp) copies
// the tile's contiguous points of every field and orbital plane into shared memory,
//   W: nf fields, u_k: nocc planes, u_k': nkp nocc planes, Y_k and Y_k': as many,
// counting the bytes on the buffer's `full` mbarrier. The consumer warps (one point per
// thread) wait for it, compute, store Y with plain coalesced stores and arrive on the
// buffer's `free` mbarrier, after which the producer refills it with the tile kBulkStages
// ahead. The bytes in flight therefore sit in shared memory, not in registers; a CTA
// takes about 100 KB, so two run per SM, or one next to a transform pass of the other
// stream's wave. Every wait is bounded: on timeout the kernel records OCCRI_ETIMEOUT in
// the plan status and leaves.
namespace tma {
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity to complete: gives up after limit_ns
// nanoseconds of the global timer (or 2^22 polls, whichever comes first).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((long long)(global_ns() - t0) > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
}  // namespace tma

constexpr int kBulkTile = 64;    // points per tile = consumer threads (two warps)
constexpr int kBulkStages = 2;   // tile buffers per CTA (one in use, one filling)

template <typename T, int NOC>
__global__ void __launch_bounds__(kBulkTile + 32, 2)
pass_d_bulk(const cplx_t<T>* __restrict__ S, const cplx_t<T>* __restrict__ psi,
            cplx_t<T>* __restrict__ Y, PairParams p) {
  using C2 = cplx_t<T>;
  constexpr int TP = kBulkTile, NS = kBulkStages;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_raw);  // full[NS], free[NS]
  C2* buf0 = reinterpret_cast<C2*>(smem_raw + 128);
  const int nocc = p.nocc;
  const int nf = wave_fields(nocc, p.nkp, p.diag);
  const int nkq = p.diag ? 0 : p.nkp * nocc;   // orbital planes at k'
  const int planes = nf + 2 * nocc + 2 * nkq;  // W, u_k, u_k', Y_k, Y_k'
  const long long ng = p.ng;
  const long long tiles = (ng + TP - 1) / TP;
  const unsigned full0 = tma::smem_u32(&bars[0]), free0 = tma::smem_u32(&bars[NS]);
  if (threadIdx.x == 0) {
    for (int b = 0; b < NS; ++b) {
      tma::mbar_init(full0 + 8 * b, 1);
      tma::mbar_init(free0 + 8 * b, TP);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // plane offsets inside a buffer (in points): W | u_k | u_k' | Y_k | Y_k'
  const int oPk = nf * TP, oPq = oPk + nocc * TP, oYk = oPq + nkq * TP, oYq = oYk + nocc * TP;
  auto buf = [&](int b) { return buf0 + (size_t)b * planes * TP; };

  if (threadIdx.x >= TP) {   // producer warp
    if (threadIdx.x != TP) return;
    // test-only fault: issue no copy at all, so that every consumer's first wait runs out
    // (nothing is in flight when the CTA leaves)
    if (p.fault == OCCRI_FAULT_WAIT) return;
    long long it = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int b = (int)(it % NS);
      // the buffer's previous tile (it - NS) must have been consumed
      if (it >= NS && !tma::mbar_wait(free0 + 8 * b, (unsigned)((it / NS - 1) & 1), p.wait_ns)) {
        record_timeout(p.status);
        return;
      }
      const long long r0 = tile * TP;
      const long long npts = std::min<long long>(TP, ng - r0);
      // bytes per plane, a multiple of 16 (the last tile may read into the field padding)
      const unsigned bytes = (unsigned)(((npts * (long long)sizeof(C2)) + 15) / 16 * 16);
      const unsigned fb = full0 + 8 * b;
      tma::mbar_expect_tx(fb, bytes * (unsigned)planes);
      C2* d = buf(b);
      for (int f = 0; f < nf; ++f)
        tma::bulk_g2s(tma::smem_u32(d + f * TP), S + (size_t)f * p.fs + r0, bytes, fb);
      for (int i = 0; i < nocc; ++i) {
        const size_t src = (size_t)(p.k * nocc + i) * p.fs + r0;
        tma::bulk_g2s(tma::smem_u32(d + oPk + i * TP), psi + src, bytes, fb);
        tma::bulk_g2s(tma::smem_u32(d + oYk + i * TP), Y + src, bytes, fb);
      }
      for (int j = 0; j < nkq; ++j) {
        const size_t src = (size_t)(p.kp0 * nocc + j) * p.fs + r0;
        tma::bulk_g2s(tma::smem_u32(d + oPq + j * TP), psi + src, bytes, fb);
        tma::bulk_g2s(tma::smem_u32(d + oYq + j * TP), Y + src, bytes, fb);
      }
    }
    // every issued copy completes before the consumers release its buffer; wait for the
    // last NS releases so that no copy is in flight when the CTA exits
    for (long long last = std::max<long long>(0, it - NS); last < it; ++last) {
      const int b = (int)(last % NS);
      if (!tma::mbar_wait(free0 + 8 * b, (unsigned)((last / NS) & 1), p.wait_ns)) {
        record_timeout(p.status);
        return;
      }
    }
    return;
  }

  // consumer warps
  const int t = threadIdx.x;
  long long it = 0;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
    const int b = (int)(it % NS);
    if (!tma::mbar_wait(full0 + 8 * b, (unsigned)((it / NS) & 1), p.wait_ns)) {
      record_timeout(p.status);
      return;
    }
    const C2* d = buf(b);
    const long long r = tile * TP + t;
    if (r < ng) {
      T pr[NOC], pim[NOC], ar[NOC], ai[NOC];
#pragma unroll
      for (int i = 0; i < NOC; ++i) {
        C2 v = mk<T>(T(0), T(0));
        if (i < nocc) v = d[oPk + i * TP + t];
        pr[i] = v.x; pim[i] = v.y;
        ar[i] = T(0); ai[i] = T(0);
      }
      if (p.diag) {
#pragma unroll
        for (int j = 0; j < NOC; ++j) {
          if (j >= nocc) break;
#pragma unroll
          for (int i = 0; i <= j; ++i) {
            const C2 w = d[diag_field(i, j, nocc) * TP + t];
            ar[i] += w.x * pr[j] - w.y * pim[j];     // W_ij u_j
            ai[i] += w.x * pim[j] + w.y * pr[j];
            if (i < j) {                             // W_ji u_i = conj(W_ij) u_i
              ar[j] += w.x * pr[i] + w.y * pim[i];
              ai[j] += w.x * pim[i] - w.y * pr[i];
            }
          }
        }
      } else {
#pragma unroll 1
        for (int kpl = 0; kpl < p.nkp; ++kpl) {
          T qr[NOC], qi[NOC], br[NOC], bi[NOC];
#pragma unroll
          for (int j = 0; j < NOC; ++j) {
            C2 v = mk<T>(T(0), T(0));
            if (j < nocc) v = d[oPq + (kpl * nocc + j) * TP + t];
            qr[j] = v.x; qi[j] = v.y;
            br[j] = T(0); bi[j] = T(0);
          }
          const C2* wk = d + (size_t)kpl * nocc * nocc * TP + t;
#pragma unroll
          for (int i = 0; i < NOC; ++i) {
            if (i >= nocc) break;
#pragma unroll
            for (int j = 0; j < NOC; ++j) {
              if (j >= nocc) break;
              const C2 w = wk[(i * nocc + j) * TP];
              ar[i] += w.x * qr[j] - w.y * qi[j];     // W u_{jk'}
              ai[i] += w.x * qi[j] + w.y * qr[j];
              br[j] += w.x * pr[i] + w.y * pim[i];    // conj(W) u_{ik}
              bi[j] += w.x * pim[i] - w.y * pr[i];
            }
          }
#pragma unroll
          for (int j = 0; j < NOC; ++j) {
            if (j >= nocc) break;
            const C2 y = d[oYq + (kpl * nocc + j) * TP + t];
            Y[(size_t)((p.kp0 + kpl) * nocc + j) * p.fs + r] = mk<T>(y.x + br[j], y.y + bi[j]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NOC; ++i) {
        if (i >= nocc) break;
        const C2 y = d[oYk + i * TP + t];
        Y[(size_t)(p.k * nocc + i) * p.fs + r] = mk<T>(y.x + ar[i], y.y + ai[i]);
      }
    }
    tma::mbar_arrive(free0 + 8 * b);
  }
}

// Bytes of shared memory of pass_d_bulk for a wave (two buffers and the barriers), or 0
// when they would not fit next to nothing else on an SM (the register form runs then).
inline size_t bulk_smem(int nocc, int nkp, int diag, size_t csz) {
  const int nf = wave_fields(nocc, nkp, diag);
  const int planes = nf + 2 * nocc + 2 * (diag ? 0 : nkp * nocc);
  const size_t bytes = 128 + (size_t)kBulkStages * planes * kBulkTile * csz;
  return bytes <= 226 * 1024 ? bytes : 0;
}

template <typename T, int NOC>
cudaError_t launch_pass_d_noc(const PairParams& p, const cplx_t<T>* S, const cplx_t<T>* psi,
                              cplx_t<T>* Y, cudaStream_t st) {
  const size_t sm = bulk_smem(p.nocc, p.nkp, p.diag, sizeof(cplx_t<T>));
  if (sm) {
    // the largest shared-memory size set so far for this device, and the resident slots
    // of each shared-memory size actually launched (one cache per wave kind)
    static std::mutex mu;
    static int sm_set[kMaxDevices] = {};
    static DeviceCache slots_cache[2];
    {
      std::lock_guard<std::mutex> lock(mu);
      int& have = sm_set[(p.device >= 0 && p.device < kMaxDevices) ? p.device : 0];
      if ((int)sm > have) {
        if (cudaFuncSetAttribute(pass_d_bulk<T, NOC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
          return cudaGetLastError();
        have = (int)sm;
      }
    }
    const int slots = slots_cache[p.diag ? 0 : 1].get(
        p.device, [&] { return resident_slots(pass_d_bulk<T, NOC>, kBulkTile + 32, sm); });
    const long long tiles = (p.ng + kBulkTile - 1) / kBulkTile;
    pass_d_bulk<T, NOC><<<(unsigned)std::min<long long>(tiles, slots), kBulkTile + 32, sm,
                          st>>>(S, psi, Y, p);
    return cudaGetLastError();
  }
  static DeviceCache slots_reg;
  const int slots = slots_reg.get(p.device, [] { return resident_slots(pass_d<T, NOC>, 256, 0); });
  const unsigned nb = (unsigned)std::min<long long>((p.ng + 255) / 256, slots);
  pass_d<T, NOC><<<nb, 256, 0, st>>>(S, psi, Y, p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass_d(const PairParams& p, const cplx_t<T>* S, const cplx_t<T>* psi,
                          cplx_t<T>* Y, cudaStream_t st) {
  if (p.nocc <= 4) return launch_pass_d_noc<T, 4>(p, S, psi, Y, st);
  if (p.nocc <= 8) return launch_pass_d_noc<T, 8>(p, S, psi, Y, st);
  if (p.nocc <= 16) return launch_pass_d_noc<T, 16>(p, S, psi, Y, st);
  return launch_pass_d_noc<T, 32>(p, S, psi, Y, st);
}

// ------------------------------------------------------------------ pass CD (C and D fused)
// Passes C and D as one kernel, for FP32 waves with nocc <= kCdNoc. A CTA owns the points
// with every n3, one n1 and CdShape::CW consecutive n2 (row pieces). Per batch of
// at most kCdFields fields it copies those pieces of the batch's fields into shared
// memory, transforms every (field, n2) line inversely along m3 in place, and adds the
// batch's terms
//   Y_{ik}  += sum_j W_{k'ij} u_{jk'},      Y_{jk'} += sum_i conj(W_{k'ij}) u_{ik}
// at its points (diagonal waves: fields i <= j, W_ji = conj(W_ij), Y_{k'} = Y_k), so
// the potentials W never go back to global memory. The orbital planes u_k and u_{k'} of
// the CTA's points sit in shared memory beside the batch; the sums for Y stay in
// registers (one point per thread) and are added to Y once per k' (Y_{k'}) and once per
// wave (Y_k). A batch holds whole rows i of the wave's field list, so a row's terms
// land in fixed registers.
constexpr int kCdFields = 32;   // fields per batch
constexpr int kCdNoc = kFusedCdNoc;   // largest nocc of the fused form
// CTA shape: CW n2 columns (CW x 8 bytes per row piece), NT threads (NT >= N CW, and
// kCdFields CW lines per transform round with two threads a line), MB CTAs per SM.
struct CdShape {
  static constexpr int CW = 4, NT = 256, MB = 2;
};
// Plane pitch (points) in shared memory: >= N CW and = CW (mod 16), so that the 8-byte
// loads of a half warp (16 / CW fields x CW columns at one m3) hit 32 distinct banks.
constexpr int cd_pitch(int n, int cw) {
  return n * cw + ((cw - (n * cw) % 16) + 16) % 16;
}
constexpr size_t cd_smem(int n, int cw) {
  return sizeof(float2) * (size_t)cd_pitch(n, cw) * (kCdFields + 2 * kCdNoc);
}

// Rows n3 = 0..N-1 of columns [c0, c0 + CW) at row n1 of np planes (plane pl starts at
// src(pl)) into dst + pl * PP + n3 CW + c; columns >= N are skipped. 16-byte copies
// for even N (the pieces start at even points), 8-byte ones otherwise. Each thread keeps
// one (n3, c) and steps through the planes, NT / (copies per plane) at a time.
template <int N, int CW, int NT, typename Src>
__device__ __forceinline__ void cd_copy(float2* dst, int np, Src src, int n1, int c0) {
  constexpr int PP = cd_pitch(N, CW);
  constexpr int W = (N % 2 == 0) ? 2 : 1;      // points per copy
  constexpr int RW = CW / W;                   // copies per row piece
  constexpr int per = N * RW;                  // copies per plane
  constexpr int PT = NT / per;                 // planes in flight per step
  static_assert(PT >= 1, "a copy per thread and plane");
  const int t = threadIdx.x;
  if (t >= PT * per) return;
  const int r = t % per;
  const int n3 = r / RW, c = (r % RW) * W;
  if (c0 + c >= N) return;
  float2* d = dst + n3 * CW + c;
  const size_t off = ((size_t)n3 * N + n1) * N + c0 + c;
  for (int pl = t / per; pl < np; pl += PT) cp_async<8 * W>(d + pl * PP, src(pl) + off);
}

// A batch of the wave's field list: rows [i0, i1) of k' offset kpl, fields [fa, fa + cnt).
struct CdBatch { int kpl, i0, i1, fa, cnt; };
__device__ __forceinline__ CdBatch cd_batch(int kpl, int i0, int nocc, int diag) {
  CdBatch b;
  b.kpl = kpl;
  b.i0 = i0;
  if (diag) {   // whole rows i <= j, at most kCdFields fields (a row has <= kCdNoc)
    b.fa = diag_field(i0, i0, nocc);
    b.cnt = 0;
    b.i1 = i0;
    while (b.i1 < nocc && b.cnt + (nocc - b.i1) <= kCdFields) b.cnt += nocc - b.i1++;
  } else {
    b.i1 = min(nocc, i0 + max(1, kCdFields / nocc));
    b.fa = kpl * nocc * nocc + i0 * nocc;
    b.cnt = (b.i1 - b.i0) * nocc;
  }
  return b;
}

template <int N, int CW, int NT, int MB>
__global__ void __launch_bounds__(NT, MB)
pass_cd(const float2* __restrict__ S, const float2* __restrict__ psi, float2* __restrict__ Y,
        PairParams p) {
  static_assert(N * CW <= NT, "one point per thread");
  constexpr int PP = cd_pitch(N, CW);
  constexpr int NOC = kCdNoc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Wb = reinterpret_cast<float2*>(smem_raw);   // [field of batch][n3][c], pitch PP
  float2* Uk = Wb + kCdFields * PP;                    // [i][n3][c]
  float2* Uq = Uk + NOC * PP;                          // [j][n3][c]
  const int c0 = blockIdx.x * CW, n1 = blockIdx.y;
  const int nocc = p.nocc;
  const int t = threadIdx.x;
  const int tc = t % CW;
  const bool pvalid = t < N * CW && c0 + tc < N;
  const size_t q = ((size_t)(t / CW) * N + n1) * N + c0 + tc;   // the thread's point
  const int nkl = p.diag ? 1 : p.nkp;
  auto copy_w = [&](float2* dst, const CdBatch& b) {
    cd_copy<N, CW, NT>(dst, b.cnt, [&](int f) { return S + (size_t)(b.fa + f) * p.fs; }, n1, c0);
  };
  auto copy_uq = [&](int kpl) {
    const int kp = p.kp0 + kpl;
    cd_copy<N, CW, NT>(Uq, nocc, [&](int j) { return psi + (size_t)(kp * nocc + j) * p.fs; }, n1,
                       c0);
  };
  float ar[NOC], ai[NOC], br[NOC], bi[NOC];
#pragma unroll
  for (int i = 0; i < NOC; ++i) { ar[i] = ai[i] = br[i] = bi[i] = 0.f; }
  cd_copy<N, CW, NT>(Uk, nocc, [&](int i) { return psi + (size_t)(p.k * nocc + i) * p.fs; }, n1,
                     c0);
  CdBatch cur = cd_batch(0, 0, nocc, p.diag);
  if (!p.diag) copy_uq(0);
  copy_w(Wb, cur);
  cp_async_commit();
#pragma unroll 1
  while (true) {
    const bool more = cur.i1 < nocc || cur.kpl + 1 < nkl;
    const bool end_kpl = cur.i1 >= nocc;
    cp_async_wait<0>();   // this batch (and at its k' change the u_k' planes) has landed
    __syncthreads();
    // inverse along m3 of every (field, column) line of the batch, in place
    {
      const int lines = cur.cnt * CW;
      constexpr int SP = line_split(N);
      constexpr int per_round = NT / SP;
#pragma unroll 1
      for (int l0 = 0; l0 < lines; l0 += per_round) {
        if constexpr (SP == 2) {
          const int w = t >> 5;
          const int line0 = l0 + (w >> 1) * 32 + (t & 31);
          const bool valid = line0 < lines;
          const int line = valid ? line0 : lines - 1;
          line_fft2<float, N>(Wb + (line / CW) * PP + line % CW, CW, true, true, w & 1, valid, 0,
                              [](int, float&, float&) {});
        } else {
          const int line = l0 + t;
          if (line < lines)
            line_fft<float, N>(Wb + (line / CW) * PP + line % CW, CW, true, true,
                               [](int, float&, float&) {});
        }
      }
    }
    __syncthreads();
    // the batch's terms at this thread's point
    const int i0 = cur.i0, i1 = cur.i1, fa = cur.fa;
    if (pvalid) {
      if (p.diag) {
#pragma unroll
        for (int i = 0; i < NOC; ++i) {
          if (i < i0 || i >= i1) continue;
          const float2 ui = Uk[i * PP + t];
#pragma unroll
          for (int j = i; j < NOC; ++j) {
            if (j >= nocc) break;
            const float2 w = Wb[(diag_field(i, j, nocc) - fa) * PP + t];
            const float2 uj = Uk[j * PP + t];
            ar[i] += w.x * uj.x - w.y * uj.y;     // W_ij u_j
            ai[i] += w.x * uj.y + w.y * uj.x;
            if (i < j) {                          // W_ji u_i = conj(W_ij) u_i
              ar[j] += w.x * ui.x + w.y * ui.y;
              ai[j] += w.x * ui.y - w.y * ui.x;
            }
          }
        }
      } else {
        float qr[NOC], qi[NOC];
#pragma unroll
        for (int j = 0; j < NOC; ++j) {
          const float2 v = j < nocc ? Uq[j * PP + t] : make_float2(0.f, 0.f);
          qr[j] = v.x; qi[j] = v.y;
        }
#pragma unroll
        for (int i = 0; i < NOC; ++i) {
          if (i < i0 || i >= i1) continue;
          const float2 ui = Uk[i * PP + t];
          const float2* wrow = Wb + (i - i0) * nocc * PP + t;
#pragma unroll
          for (int j = 0; j < NOC; ++j) {
            if (j >= nocc) break;
            const float2 w = wrow[j * PP];
            ar[i] += w.x * qr[j] - w.y * qi[j];     // W u_{jk'}
            ai[i] += w.x * qi[j] + w.y * qr[j];
            br[j] += w.x * ui.x + w.y * ui.y;       // conj(W) u_{ik}
            bi[j] += w.x * ui.y - w.y * ui.x;
          }
        }
      }
    }
    // add the k' sums to Y_{k'}: all loads before the first store, so that the planes'
    // loads are in flight together
    if (end_kpl && pvalid && !p.diag) {
      const int kp = p.kp0 + cur.kpl;
      float2 v[NOC];
#pragma unroll
      for (int j = 0; j < NOC; ++j)
        if (j < nocc) v[j] = Y[(size_t)(kp * nocc + j) * p.fs + q];
#pragma unroll
      for (int j = 0; j < NOC; ++j) {
        if (j >= nocc) break;
        Y[(size_t)(kp * nocc + j) * p.fs + q] = make_float2(v[j].x + br[j], v[j].y + bi[j]);
        br[j] = bi[j] = 0.f;
      }
    }
    __syncthreads();   // this batch's buffer (and at a k' change the u_{k'} planes) is free
    if (!more) break;
    const CdBatch nxt = end_kpl ? cd_batch(cur.kpl + 1, 0, nocc, p.diag)
                                : cd_batch(cur.kpl, cur.i1, nocc, p.diag);
    if (end_kpl && !p.diag) copy_uq(nxt.kpl);
    copy_w(Wb, nxt);
    cp_async_commit();
    cur = nxt;
  }
  if (pvalid) {
    float2 v[NOC];
#pragma unroll
    for (int i = 0; i < NOC; ++i)
      if (i < nocc) v[i] = Y[(size_t)(p.k * nocc + i) * p.fs + q];
#pragma unroll
    for (int i = 0; i < NOC; ++i) {
      if (i >= nocc) break;
      Y[(size_t)(p.k * nocc + i) * p.fs + q] = make_float2(v[i].x + ar[i], v[i].y + ai[i]);
    }
  }
}

// ------------------------------------------------------------------ omega term of the adjoint
// Plane m3 of field f, after pass A has transformed both the pair density rho (S0) and
// its adjoint density sigma (S1) along n3 and n2: both planes are transformed along n1
// and sum_m (dv/d omega)/(4 pi) Re(conj(sigma^) rho^) is added to *dacc, weight 1/2 for
// a field (k, k, i, i) of a diagonal wave (the only pair that is its own reverse).
template <typename T, int N>
__global__ void __launch_bounds__(threads_for(N), min_blocks(N, sizeof(cplx_t<T>)))
pass_b_domega2(const cplx_t<T>* __restrict__ S0, const cplx_t<T>* __restrict__ S1,
               PairParams p, double* __restrict__ dacc) {
  using C2 = cplx_t<T>;
  constexpr int P = pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* rho = reinterpret_cast<C2*>(smem_raw);                     // [n1][m2]
  C2* sig = rho + N * P;
  Axis1<T>* ax1 = reinterpret_cast<Axis1<T>*>(sig + N * P);     // [m1]
  T* vtab = reinterpret_cast<T*>(ax1 + N);                       // [m1][m2] dv/(4 pi)
  __shared__ double red[4];
  const int m3 = blockIdx.x;
  const int f = blockIdx.y;
  const FieldIdx fi = field_idx(f, p.nocc, p.diag);
  stage_plane<T, N, P>(rho, S0 + (size_t)f * p.fs + (size_t)m3 * N * N);
  stage_plane<T, N, P>(sig, S1 + (size_t)f * p.fs + (size_t)m3 * N * N);
  cp_async_commit();
  const MetricHL<T> gm(p);
  fill_vtab<T, N, true>(p, gm, m3, fi.kpl, ax1, vtab, 0, 1);
  cp_async_wait<0>();
  __syncthreads();
  T dsum = T(0);
#pragma unroll 1
  for (int job = 0; job < 2; ++job) {   // rho^ (stored), then sigma^ (paired with rho^)
    run_lines<T, N>(job == 0 ? rho : sig, P, false, false, job == 0,
                    [&](int line, int k, T& re, T& im) {
                      if (job == 1) {
                        const C2 r = rho[k * P + line];
                        dsum += vtab[k * N + line] * (re * r.x + im * r.y);
                      }
                    });
    __syncthreads();
  }
  double part = double(dsum);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(dacc, (p.diag && fi.i == fi.j) ? 0.5 * t : t);
  }
}

// ------------------------------------------------------------------ pass E (adjoint)
// The adjoint of the Y accumulation and of the pair densities, per grid point (fields'
// point order, periodic parts). With W the potentials of the wave's fields (scratch SW)
// and Z the potentials of their adjoint densities sigma (scratch SZ), g the adjoint
// orbital field and u the orbitals, every unordered pair (k, k', i, j) adds
//   G_ik  += u_jk' Z_ij + g_jk' W_ij,      G_jk' += u_ik conj(Z_ij) + g_ik conj(W_ij),
// a field (k, k, i, i) of a diagonal wave only the first. NOC >= nocc.
template <typename T, int NOC>
__global__ void __launch_bounds__(256)
pass_e(const cplx_t<T>* __restrict__ SW, const cplx_t<T>* __restrict__ SZ,
       const cplx_t<T>* __restrict__ psi, const cplx_t<T>* __restrict__ gam,
       cplx_t<T>* __restrict__ G, PairParams p) {
  using C2 = cplx_t<T>;
  const long long ng = p.ng;
  const int nocc = p.nocc;
  auto mac = [](C2& acc, C2 a, C2 b) {   // acc += a * b
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
  };
  auto macc = [](C2& acc, C2 a, C2 b) {   // acc += a * conj(b)
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.y * b.x - a.x * b.y;
  };
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng;
       r += (long long)gridDim.x * blockDim.x) {
    C2 uk[NOC], gk[NOC], acc[NOC];
#pragma unroll
    for (int i = 0; i < NOC; ++i) {
      uk[i] = gk[i] = acc[i] = mk<T>(T(0), T(0));
      if (i < nocc) {
        uk[i] = __ldg(psi + (size_t)(p.k * nocc + i) * p.fs + r);
        gk[i] = __ldg(gam + (size_t)(p.k * nocc + i) * p.fs + r);
      }
    }
    if (p.diag) {
#pragma unroll
      for (int j = 0; j < NOC; ++j) {
        if (j >= nocc) break;
#pragma unroll
        for (int i = 0; i <= j; ++i) {
          const size_t f = (size_t)diag_field(i, j, nocc) * p.fs + r;
          const C2 w = __ldg(SW + f), z = __ldg(SZ + f);
          mac(acc[i], uk[j], z);
          mac(acc[i], gk[j], w);
          if (i < j) {
            macc(acc[j], uk[i], z);
            macc(acc[j], gk[i], w);
          }
        }
      }
    } else {
#pragma unroll 1
      for (int kpl = 0; kpl < p.nkp; ++kpl) {
        const int kp = p.kp0 + kpl;
        C2 uq[NOC], gq[NOC], accq[NOC];
#pragma unroll
        for (int j = 0; j < NOC; ++j) {
          uq[j] = gq[j] = accq[j] = mk<T>(T(0), T(0));
          if (j < nocc) {
            uq[j] = __ldg(psi + (size_t)(kp * nocc + j) * p.fs + r);
            gq[j] = __ldg(gam + (size_t)(kp * nocc + j) * p.fs + r);
          }
        }
#pragma unroll
        for (int i = 0; i < NOC; ++i) {
          if (i >= nocc) break;
#pragma unroll
          for (int j = 0; j < NOC; ++j) {
            if (j >= nocc) break;
            const size_t f = (size_t)((kpl * nocc + i) * nocc + j) * p.fs + r;
            const C2 w = __ldg(SW + f), z = __ldg(SZ + f);
            mac(acc[i], uq[j], z);
            mac(acc[i], gq[j], w);
            macc(accq[j], uk[i], z);
            macc(accq[j], gk[i], w);
          }
        }
#pragma unroll
        for (int j = 0; j < NOC; ++j) {
          if (j >= nocc) break;
          C2* g = G + (size_t)(kp * nocc + j) * p.fs + r;
          C2 v = *g;
          v.x += accq[j].x;
          v.y += accq[j].y;
          *g = v;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NOC; ++i) {
      if (i >= nocc) break;
      C2* g = G + (size_t)(p.k * nocc + i) * p.fs + r;
      C2 v = *g;
      v.x += acc[i].x;
      v.y += acc[i].y;
      *g = v;
    }
  }
}

template <typename T>
cudaError_t launch_pass_e(const PairParams& p, const cplx_t<T>* SW, const cplx_t<T>* SZ,
                          const cplx_t<T>* psi, const cplx_t<T>* gam, cplx_t<T>* G,
                          cudaStream_t st) {
  const unsigned nb = (unsigned)std::min<long long>((p.ng + 255) / 256, 152LL * 8);
  if (p.nocc <= 4) pass_e<T, 4><<<nb, 256, 0, st>>>(SW, SZ, psi, gam, G, p);
  else if (p.nocc <= 8) pass_e<T, 8><<<nb, 256, 0, st>>>(SW, SZ, psi, gam, G, p);
  else if (p.nocc <= 16) pass_e<T, 16><<<nb, 256, 0, st>>>(SW, SZ, psi, gam, G, p);
  else pass_e<T, 32><<<nb, 256, 0, st>>>(SW, SZ, psi, gam, G, p);
  return cudaGetLastError();
}

template <int N> constexpr size_t smem_a(size_t csz) { return csz * N * pitch(N); }
template <int N> constexpr size_t smem_b(size_t csz, size_t tab) {
  return csz * N * pitch(N) + N * tab + csz / 2 * N * N;
}

template <int N> constexpr size_t smem_c(size_t csz) { return csz * N * pitch(N); }

template <typename T, int N>
cudaError_t run_wave(const PairParams& p, const cplx_t<T>* psi, cplx_t<T>* S, cplx_t<T>* Y,
                     cudaStream_t st, cudaEvent_t* ev, cudaEvent_t ev_y) {
  using C2 = cplx_t<T>;
  const int nt = threads_for(N);
  const int nf = wave_fields(p.nocc, p.nkp, p.diag);
  const size_t sa = smem_a<N>(sizeof(C2));
  const size_t sb = smem_b<N>(sizeof(C2), sizeof(Axis1<T>));
  const size_t sc = smem_c<N>(sizeof(C2));
  static DeviceCache cache;   // per device: attributes set, resident pass-B slots
  const int slots_b = cache.get(p.device, [&] {
    cudaFuncSetAttribute(pass_a<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    cudaFuncSetAttribute(pass_b<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    cudaFuncSetAttribute(pass_c<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    if constexpr (std::is_same<T, float>::value)
      cudaFuncSetAttribute(pass_cd<N, CdShape::CW, CdShape::NT, CdShape::MB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cd_smem(N, CdShape::CW));
    return resident_slots(pass_b<T, N>, nt, sb);
  });
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  if (ev) chk(cudaEventRecord(ev[0], st));
  // pass A; without the plan's tables, the wave's kernel tables in the same launch (extra
  // rows of CTAs fill them)
  T* vt = reinterpret_cast<T*>(reinterpret_cast<char*>(S) + p.vt_off);
  const int tab_rows = p.vq ? 0 : (p.diag ? 1 : p.nkp) * kVtabSplit;
  pass_a<T, N><<<dim3(N, nf + tab_rows), nt, sa, st>>>(psi, S, p, nullptr,
                                                       p.vq ? nullptr : vt);
  if (ev) chk(cudaEventRecord(ev[1], st));
  pass_b<T, N><<<std::min(N * nf, std::max(1, slots_b / std::max(1, p.b_div))), nt, sb, st>>>(
      S, p, vt);
  if (ev) chk(cudaEventRecord(ev[2], st));
  // FP32 waves of nocc <= kCdNoc: passes C and D fused (the potentials stay on chip)
  const bool fused = pair_wave_launches<T>(p.nocc, p.split_cd) == 3;
  if (!fused) pass_c<T, N><<<dim3(N, nf), nt, sc, st>>>(S, p);
  if (ev_y) chk(cudaStreamWaitEvent(st, ev_y, 0));   // the previous wave's Y updates
  if constexpr (std::is_same<T, float>::value) {
    if (fused)
      pass_cd<N, CdShape::CW, CdShape::NT, CdShape::MB>
          <<<dim3((N + CdShape::CW - 1) / CdShape::CW, N), CdShape::NT,
              cd_smem(N, CdShape::CW), st>>>((const float2*)S, (const float2*)psi,
                                                           (float2*)Y, p);
  }
  if (!fused) chk(launch_pass_d<T>(p, S, psi, Y, st));
  if (ev_y) chk(cudaEventRecord(ev_y, st));
  if (ev) chk(cudaEventRecord(ev[3], st));
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int N>
cudaError_t run_domega_wave(const PairParams& p, const cplx_t<T>* psi, cplx_t<T>* S,
                            double* dacc, cudaStream_t st) {
  using C2 = cplx_t<T>;
  const int nt = threads_for(N);
  const int nf = wave_fields(p.nocc, p.nkp, p.diag);
  const size_t sa = smem_a<N>(sizeof(C2));
  const size_t sb = smem_b<N>(sizeof(C2), sizeof(Axis1<T>));
  static DeviceCache cache;   // per device: attributes set, resident pass-B slots
  const int slots_b = cache.get(p.device, [&] {
    cudaFuncSetAttribute(pass_a<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    cudaFuncSetAttribute(pass_b_domega<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sb);
    return resident_slots(pass_b_domega<T, N>, nt, sb);
  });
  pass_a<T, N><<<dim3(N, nf), nt, sa, st>>>(psi, S, p);
  pass_b_domega<T, N><<<std::min(N * nf, slots_b), nt, sb, st>>>(S, p, dacc);
  return cudaGetLastError();
}

// One wave of the adjoint: the forward potentials W into S0, the potentials Z of the
// adjoint densities into S1 (the same three transform passes), then pass E.
template <typename T, int N>
cudaError_t run_vjp_wave(const PairParams& p, const cplx_t<T>* psi, const cplx_t<T>* gam,
                         cplx_t<T>* S0, cplx_t<T>* S1, cplx_t<T>* G, double* dacc,
                         cudaStream_t st) {
  using C2 = cplx_t<T>;
  const int nt = threads_for(N);
  const int nf = wave_fields(p.nocc, p.nkp, p.diag);
  const size_t sa = smem_a<N>(sizeof(C2));
  const size_t sb = smem_b<N>(sizeof(C2), sizeof(Axis1<T>));
  const size_t sc = smem_c<N>(sizeof(C2));
  static DeviceCache cache;   // per device: attributes set, resident pass-B slots
  const int slots_b = cache.get(p.device, [&] {
    cudaFuncSetAttribute(pass_a<T, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sa);
    cudaFuncSetAttribute(pass_a<T, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sa);
    cudaFuncSetAttribute(pass_b<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    cudaFuncSetAttribute(pass_c<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    cudaFuncSetAttribute(pass_b_domega2<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sb + sizeof(C2) * N * pitch(N)));
    return resident_slots(pass_b<T, N>, nt, sb);
  });
  pass_a<T, N, false><<<dim3(N, nf), nt, sa, st>>>(psi, S0, p, nullptr);
  pass_a<T, N, true><<<dim3(N, nf), nt, sa, st>>>(psi, S1, p, gam);
  if (dacc)
    pass_b_domega2<T, N><<<dim3(N, nf), nt, sb + sizeof(C2) * N * pitch(N), st>>>(S0, S1, p,
                                                                                dacc);
  T* vt = reinterpret_cast<T*>(reinterpret_cast<char*>(S0) + p.vt_off);
  if (!p.vq) vtab_kernel<T, N><<<dim3(N, p.diag ? 1 : p.nkp, kVtabSplit), nt, 0, st>>>(vt, p);
  pass_b<T, N><<<std::min(N * nf, slots_b), nt, sb, st>>>(S0, p, vt);
  pass_c<T, N><<<dim3(N, nf), nt, sc, st>>>(S0, p);
  pass_b<T, N><<<std::min(N * nf, slots_b), nt, sb, st>>>(S1, p, vt);
  pass_c<T, N><<<dim3(N, nf), nt, sc, st>>>(S1, p);
  const cudaError_t e = launch_pass_e<T>(p, S0, S1, psi, gam, G, st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The plan's kernel tables into vq: (2 D_1 - 1)(2 D_2 - 1)(2 D_3 - 1) tables of N^3 values.
template <typename T, int N>
cudaError_t run_qtables(const PairParams& p, T* vq, cudaStream_t st) {
  const unsigned nq = (unsigned)((2 * p.D[0] - 1) * (2 * p.D[1] - 1) * (2 * p.D[2] - 1));
  qtab_kernel<T, N><<<dim3(nq, N, kVtabSplit), threads_for(N), 0, st>>>(vq, p);
  return cudaGetLastError();
}

}  // namespace pairs

}  // namespace occri
