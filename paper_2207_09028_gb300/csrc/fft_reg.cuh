// fft_reg.cuh -- one-thread, register-resident mixed-radix FFT of compile-time length.
//
// A length-N transform lives in two register arrays re[], im[]. The decimation-
// in-frequency recursion N = R*M (R in {4,3,5,2}) is unrolled completely at
// compile time, so every index, every twiddle and the final digit permutation
// are constants: twiddles become FMA immediates and the output permutation is a
// register renaming. X[k] = sum_n x[n] e^{SIGN 2 pi i n k / N} with SIGN = -1
// (forward) or +1 (inverse, unnormalised).
//
// Twiddle values come from a constexpr sine/cosine (Taylor series after exact
// integer octant reduction), evaluated by the compiler in double precision.
#pragma once
#include <utility>

#if defined(__CUDACC__)
#define OCCRI_HDI __host__ __device__ __forceinline__
#else
#define OCCRI_HDI inline
#endif

namespace occri {
namespace fft {

// ---------------------------------------------------------------- constexpr trig

constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}

constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}

// cos and sin of 2*pi*num/den with the angle reduced to [0, pi/4] exactly.
struct CS { double c, s; };

constexpr CS cs2pi(long long num, long long den) {
  long long r = num % den;
  if (r < 0) r += den;
  long long u = 8 * r;
  long long o = u / den;
  long long rem = u - o * den;
  double phi = (kPi / 4.0) * (double)rem / (double)den;
  double psi = (kPi / 4.0) * (double)(den - rem) / (double)den;
  double sp = taylor_sin(phi), cp = taylor_cos(phi);
  double sq = taylor_sin(psi), cq = taylor_cos(psi);
  switch (o) {
    case 0: return CS{cp, sp};
    case 1: return CS{sq, cq};
    case 2: return CS{-sp, cp};
    case 3: return CS{-cq, sq};
    case 4: return CS{-cp, -sp};
    case 5: return CS{-sq, -cq};
    case 6: return CS{sp, -cp};
    default: return CS{cq, -sq};
  }
}

// ---------------------------------------------------------------- compile-time loops

template <typename F, int... Is>
OCCRI_HDI void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}

template <int N, typename F>
OCCRI_HDI void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------- radix plan

constexpr bool is_base(int n) { return n == 1 || n == 2 || n == 3 || n == 4 || n == 5; }

constexpr int pick_radix(int n) {
  return is_base(n) ? n : (n % 4 == 0 ? 4 : (n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : 5)));
}

constexpr bool smooth235(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

// Register position p holds output X[dif_rev(N, p)] after dif<N>.
constexpr int dif_rev(int n, int p) {
  if (is_base(n)) return p;
  int r = pick_radix(n), m = n / r;
  return r * dif_rev(m, p % m) + p / m;
}

// Inverse permutation: output index k is held at register position dif_pos(N, k).
constexpr int dif_pos(int n, int k) {
  for (int p = 0; p < n; ++p)
    if (dif_rev(n, p) == k) return p;
  return -1;
}

// ---------------------------------------------------------------- butterflies

template <int SIGN, int A, int S, typename T, int TOT>
OCCRI_HDI void dft2(T (&re)[TOT], T (&im)[TOT]) {
  T ar = re[A], ai = im[A], br = re[A + S], bi = im[A + S];
  re[A] = ar + br; im[A] = ai + bi;
  re[A + S] = ar - br; im[A + S] = ai - bi;
}

template <int SIGN, int A, int S, typename T, int TOT>
OCCRI_HDI void dft3(T (&re)[TOT], T (&im)[TOT]) {
  constexpr double h = 0.86602540378443864676372317075293618;  // sqrt(3)/2
  const T ar = re[A], ai = im[A];
  const T t1r = re[A + S] + re[A + 2 * S], t1i = im[A + S] + im[A + 2 * S];
  const T dr = re[A + S] - re[A + 2 * S], di = im[A + S] - im[A + 2 * S];
  const T t2r = ar - T(0.5) * t1r, t2i = ai - T(0.5) * t1i;
  // i * SIGN * h * d = (-SIGN h di, SIGN h dr)
  const T ur = T(-SIGN * h) * di, ui = T(SIGN * h) * dr;
  re[A] = ar + t1r; im[A] = ai + t1i;
  re[A + S] = t2r + ur; im[A + S] = t2i + ui;
  re[A + 2 * S] = t2r - ur; im[A + 2 * S] = t2i - ui;
}

template <int SIGN, int A, int S, typename T, int TOT>
OCCRI_HDI void dft4(T (&re)[TOT], T (&im)[TOT]) {
  const T s0r = re[A] + re[A + 2 * S], s0i = im[A] + im[A + 2 * S];
  const T d0r = re[A] - re[A + 2 * S], d0i = im[A] - im[A + 2 * S];
  const T s1r = re[A + S] + re[A + 3 * S], s1i = im[A + S] + im[A + 3 * S];
  const T d1r = re[A + S] - re[A + 3 * S], d1i = im[A + S] - im[A + 3 * S];
  // SIGN * i * d1 = (-SIGN d1i, SIGN d1r)
  const T jr = (SIGN > 0) ? -d1i : d1i;
  const T ji = (SIGN > 0) ? d1r : -d1r;
  re[A] = s0r + s1r; im[A] = s0i + s1i;
  re[A + 2 * S] = s0r - s1r; im[A + 2 * S] = s0i - s1i;
  re[A + S] = d0r + jr; im[A + S] = d0i + ji;
  re[A + 3 * S] = d0r - jr; im[A + 3 * S] = d0i - ji;
}

template <int SIGN, int A, int S, typename T, int TOT>
OCCRI_HDI void dft5(T (&re)[TOT], T (&im)[TOT]) {
  constexpr CS w1 = cs2pi(1, 5), w2 = cs2pi(2, 5);
  const T ar = re[A], ai = im[A];
  const T t1r = re[A + S] + re[A + 4 * S], t1i = im[A + S] + im[A + 4 * S];
  const T t2r = re[A + 2 * S] + re[A + 3 * S], t2i = im[A + 2 * S] + im[A + 3 * S];
  const T t3r = re[A + S] - re[A + 4 * S], t3i = im[A + S] - im[A + 4 * S];
  const T t4r = re[A + 2 * S] - re[A + 3 * S], t4i = im[A + 2 * S] - im[A + 3 * S];
  const T c1 = T(w1.c), c2 = T(w2.c), s1 = T(SIGN * w1.s), s2 = T(SIGN * w2.s);
  const T p1r = ar + c1 * t1r + c2 * t2r, p1i = ai + c1 * t1i + c2 * t2i;
  const T p2r = ar + c2 * t1r + c1 * t2r, p2i = ai + c2 * t1i + c1 * t2i;
  const T q1r = s1 * t3r + s2 * t4r, q1i = s1 * t3i + s2 * t4i;   // times i below
  const T q2r = s2 * t3r - s1 * t4r, q2i = s2 * t3i - s1 * t4i;
  re[A] = ar + t1r + t2r; im[A] = ai + t1i + t2i;
  re[A + S] = p1r - q1i; im[A + S] = p1i + q1r;
  re[A + 4 * S] = p1r + q1i; im[A + 4 * S] = p1i - q1r;
  re[A + 2 * S] = p2r - q2i; im[A + 2 * S] = p2i + q2r;
  re[A + 3 * S] = p2r + q2i; im[A + 3 * S] = p2i - q2r;
}

template <int R, int SIGN, int A, int S, typename T, int TOT>
OCCRI_HDI void small_dft(T (&re)[TOT], T (&im)[TOT]) {
  if constexpr (R == 2) dft2<SIGN, A, S>(re, im);
  else if constexpr (R == 3) dft3<SIGN, A, S>(re, im);
  else if constexpr (R == 4) dft4<SIGN, A, S>(re, im);
  else if constexpr (R == 5) dft5<SIGN, A, S>(re, im);
}

// x[P] *= e^{SIGN 2 pi i E / N}
template <int N, int SIGN, int E, int P, typename T, int TOT>
OCCRI_HDI void twiddle(T (&re)[TOT], T (&im)[TOT]) {
  constexpr int e = E % N;
  if constexpr (e == 0) {
  } else if constexpr (2 * e == N) {
    re[P] = -re[P]; im[P] = -im[P];
  } else if constexpr (4 * e == N || 4 * e == 3 * N) {
    // multiply by (+/-) i
    constexpr int sgn = (4 * e == N) ? SIGN : -SIGN;
    const T r = re[P], i = im[P];
    if constexpr (sgn > 0) { re[P] = -i; im[P] = r; } else { re[P] = i; im[P] = -r; }
  } else {
    constexpr CS w = cs2pi(e, N);
    const T c = T(w.c), s = T(SIGN * w.s);
    const T r = re[P], i = im[P];
    re[P] = r * c - i * s;
    im[P] = r * s + i * c;
  }
}

// In-place DIF of the N elements at positions A + S*idx.
template <int N, int SIGN, int A, int S, typename T, int TOT>
OCCRI_HDI void dif(T (&re)[TOT], T (&im)[TOT]) {
  if constexpr (N == 1) {
  } else if constexpr (is_base(N)) {
    small_dft<N, SIGN, A, S>(re, im);
  } else {
    constexpr int R = pick_radix(N), M = N / R;
    static_for<M>([&](auto I1) {
      constexpr int n1 = decltype(I1)::value;
      small_dft<R, SIGN, A + S * n1, S * M>(re, im);
      static_for<R>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        twiddle<N, SIGN, n1 * k1, A + S * (n1 + M * k1)>(re, im);
      });
    });
    static_for<R>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      dif<M, SIGN, A + S * M * k1, S>(re, im);
    });
  }
}

// Full transform: after the call, register p holds X[dif_rev(N, p)].
template <int N, int SIGN, typename T>
OCCRI_HDI void fft_dif(T (&re)[N], T (&im)[N]) {
  static_assert(smooth235(N), "FFT length must be {2,3,5}-smooth");
  dif<N, SIGN, 0, 1>(re, im);
}

// Reorder registers from DIF order to natural order (compile-time renaming).
template <int N, typename T>
OCCRI_HDI void dif_to_natural(T (&re)[N], T (&im)[N]) {
  T r2[N], i2[N];
  static_for<N>([&](auto K) {
    constexpr int k = decltype(K)::value;
    r2[k] = re[dif_pos(N, k)];
    i2[k] = im[dif_pos(N, k)];
  });
  static_for<N>([&](auto K) {
    constexpr int k = decltype(K)::value;
    re[k] = r2[k];
    im[k] = i2[k];
  });
}

// ---------------------------------------------------------------- packed FP32 form
// The same decimation-in-frequency recursion for FP32 with each complex value held as
// one 64-bit register pair {re, im}. Operations that act alike on both halves (sums,
// differences, scaling by a real constant) are single packed f32x2 instructions
// (add/sub/mul/fma.rn.f32x2, sm_100 and later); products with +-i and the twiddles,
// which mix the halves, are scalar operations on the pair's halves. Every packed
// instruction rounds each half exactly as the scalar instruction would.
#if defined(__CUDACC__)
namespace pk {
using u64 = unsigned long long;
__device__ __forceinline__ u64 pack(float re, float im) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(re), "f"(im));
  return r;
}
__device__ __forceinline__ void unpack(u64 v, float& re, float& im) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(re), "=f"(im) : "l"(v));
}
__device__ __forceinline__ u64 add(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma(u64 a, u64 b, u64 c) {   // a * b + c
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ u64 splat(float c) { return pack(c, c); }
// SGN * i * x = (-SGN x.im, SGN x.re)
template <int SGN>
__device__ __forceinline__ u64 mul_i(u64 x) {
  float r, i;
  unpack(x, r, i);
  return SGN > 0 ? pack(-i, r) : pack(i, -r);
}
// x * (c + i s), scalar on the halves so that c and s stay instruction immediates
__device__ __forceinline__ u64 cmul_const(u64 x, float c, float s) {
  float r, i;
  unpack(x, r, i);
  return pack(r * c - i * s, r * s + i * c);
}
}  // namespace pk

template <int SIGN, int A, int S, int TOT>
__device__ __forceinline__ void pdft2(pk::u64 (&x)[TOT]) {
  const pk::u64 a = x[A], b = x[A + S];
  x[A] = pk::add(a, b);
  x[A + S] = pk::sub(a, b);
}

template <int SIGN, int A, int S, int TOT>
__device__ __forceinline__ void pdft3(pk::u64 (&x)[TOT]) {
  constexpr double h = 0.86602540378443864676372317075293618;  // sqrt(3)/2
  const pk::u64 a = x[A];
  const pk::u64 t1 = pk::add(x[A + S], x[A + 2 * S]);
  const pk::u64 d = pk::sub(x[A + S], x[A + 2 * S]);
  const pk::u64 t2 = pk::fma(t1, pk::splat(-0.5f), a);
  float dr, di;
  pk::unpack(d, dr, di);
  // i * SIGN * h * d = (-SIGN h di, SIGN h dr)
  const pk::u64 u = pk::pack(float(-SIGN * h) * di, float(SIGN * h) * dr);
  x[A] = pk::add(a, t1);
  x[A + S] = pk::add(t2, u);
  x[A + 2 * S] = pk::sub(t2, u);
}

template <int SIGN, int A, int S, int TOT>
__device__ __forceinline__ void pdft4(pk::u64 (&x)[TOT]) {
  const pk::u64 s0 = pk::add(x[A], x[A + 2 * S]);
  const pk::u64 d0 = pk::sub(x[A], x[A + 2 * S]);
  const pk::u64 s1 = pk::add(x[A + S], x[A + 3 * S]);
  const pk::u64 d1 = pk::sub(x[A + S], x[A + 3 * S]);
  const pk::u64 j = pk::mul_i<SIGN>(d1);   // SIGN * i * d1
  x[A] = pk::add(s0, s1);
  x[A + 2 * S] = pk::sub(s0, s1);
  x[A + S] = pk::add(d0, j);
  x[A + 3 * S] = pk::sub(d0, j);
}

template <int SIGN, int A, int S, int TOT>
__device__ __forceinline__ void pdft5(pk::u64 (&x)[TOT]) {
  constexpr CS w1 = cs2pi(1, 5), w2 = cs2pi(2, 5);
  const pk::u64 a = x[A];
  const pk::u64 t1 = pk::add(x[A + S], x[A + 4 * S]);
  const pk::u64 t2 = pk::add(x[A + 2 * S], x[A + 3 * S]);
  const pk::u64 t3 = pk::sub(x[A + S], x[A + 4 * S]);
  const pk::u64 t4 = pk::sub(x[A + 2 * S], x[A + 3 * S]);
  const pk::u64 c1 = pk::splat(float(w1.c)), c2 = pk::splat(float(w2.c));
  const pk::u64 s1 = pk::splat(float(SIGN * w1.s)), s2 = pk::splat(float(SIGN * w2.s));
  const pk::u64 p1 = pk::fma(t2, c2, pk::fma(t1, c1, a));
  const pk::u64 p2 = pk::fma(t2, c1, pk::fma(t1, c2, a));
  const pk::u64 q1 = pk::fma(t4, s2, pk::mul(t3, s1));                       // times i below
  const pk::u64 q2 = pk::fma(t4, pk::splat(float(-SIGN * w1.s)), pk::mul(t3, s2));
  const pk::u64 iq1 = pk::mul_i<1>(q1), iq2 = pk::mul_i<1>(q2);
  x[A] = pk::add(pk::add(a, t1), t2);
  x[A + S] = pk::add(p1, iq1);
  x[A + 4 * S] = pk::sub(p1, iq1);
  x[A + 2 * S] = pk::add(p2, iq2);
  x[A + 3 * S] = pk::sub(p2, iq2);
}

template <int R, int SIGN, int A, int S, int TOT>
__device__ __forceinline__ void psmall_dft(pk::u64 (&x)[TOT]) {
  if constexpr (R == 2) pdft2<SIGN, A, S>(x);
  else if constexpr (R == 3) pdft3<SIGN, A, S>(x);
  else if constexpr (R == 4) pdft4<SIGN, A, S>(x);
  else if constexpr (R == 5) pdft5<SIGN, A, S>(x);
}

// x[P] *= e^{SIGN 2 pi i E / N}
template <int N, int SIGN, int E, int P, int TOT>
__device__ __forceinline__ void ptwiddle(pk::u64 (&x)[TOT]) {
  constexpr int e = E % N;
  if constexpr (e == 0) {
  } else if constexpr (2 * e == N) {
    x[P] = pk::sub(pk::splat(0.0f), x[P]);
  } else if constexpr (4 * e == N || 4 * e == 3 * N) {
    constexpr int sgn = (4 * e == N) ? SIGN : -SIGN;
    x[P] = pk::mul_i<sgn>(x[P]);
  } else {
    constexpr CS w = cs2pi(e, N);
    x[P] = pk::cmul_const(x[P], float(w.c), float(SIGN * w.s));
  }
}

template <int N, int SIGN, int A, int S, int TOT>
__device__ __forceinline__ void pdif(pk::u64 (&x)[TOT]) {
  if constexpr (N == 1) {
  } else if constexpr (is_base(N)) {
    psmall_dft<N, SIGN, A, S>(x);
  } else {
    constexpr int R = pick_radix(N), M = N / R;
    static_for<M>([&](auto I1) {
      constexpr int n1 = decltype(I1)::value;
      psmall_dft<R, SIGN, A + S * n1, S * M>(x);
      static_for<R>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        ptwiddle<N, SIGN, n1 * k1, A + S * (n1 + M * k1)>(x);
      });
    });
    static_for<R>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      pdif<M, SIGN, A + S * M * k1, S>(x);
    });
  }
}

// Packed FP32 transform: after the call, x[p] holds X[dif_rev(N, p)].
template <int N, int SIGN>
__device__ __forceinline__ void pfft_dif(pk::u64 (&x)[N]) {
  static_assert(smooth235(N), "FFT length must be {2,3,5}-smooth");
  pdif<N, SIGN, 0, 1>(x);
}
#endif

}  // namespace fft
}  // namespace occri
