// occri_api.cu -- the C ABI (include/occri.h): plan creation, build orchestration,
// the FP64 occ-RI (ACE) assembly (step f) and the E_x adjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "occri_device.cuh"
#include "occri_internal.h"

namespace occri {

static const double kPiD = 3.14159265358979323846;

// Test-only allocation failure (occri_debug_fail_allocation): the number of device
// allocations still to succeed before one fails, or -1 when disarmed.
static std::atomic<long long> g_alloc_countdown{-1};

cudaError_t device_malloc(void** ptr, size_t bytes) {
  long long c = g_alloc_countdown.load();
  while (c >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
      if (c == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(ptr, bytes);
}

bool grid_edge_supported(int n) {
  switch (n) {
#define OCCRI_EDGE_CASE(NN) case NN:
    OCCRI_FOR_EACH_N(OCCRI_EDGE_CASE)
#undef OCCRI_EDGE_CASE
    return true;
    default:
      return false;
  }
}

AOParams Plan::ao_params() const {
  AOParams a;
  a.nk = nk; a.nao = nao; a.nocc = nocc; a.natm = natm; a.nshell = nshell;
  a.ng = ng;
  a.fs = fs;
  for (int d = 0; d < 3; ++d) { a.N[d] = N[d]; a.D[d] = D[d]; }
  a.Dc = D[0] * D[1] * D[2];
  a.shells = shells;
  a.atom_shell0 = atom_shell0;
  a.nimg = nimg;
  a.img_d = img_d; a.img_hi = img_hi; a.img_lo = img_lo; a.img_phase = img_phase;
  a.d0_d = d0_d; a.d0_hi = d0_hi; a.d0_lo = d0_lo; a.t0 = t0; a.kint = kint;
  for (int d = 0; d < 3; ++d) a.nb[d] = nb[d];
  a.nblk = nblk; a.lmax = lmax; a.nsa = nsa; a.blist = blist; a.bpre = bpre;
  a.cs = cs;
  return a;
}

PairParams Plan::pair_params() const {
  PairParams q;
  q.nk = nk; q.nocc = nocc; q.ng = ng; q.fs = fs; q.N1 = N[0];
  q.status = status;
  q.wait_ns = wait_ns;
  q.fault = fault;
  q.device = device;
  q.k = 0; q.kp0 = 0; q.nkp = 1; q.diag = 0;
  q.b_div = b_div;
  q.split_cd = split_cd;
  q.vt_off = (long long)fields_cap * fs * (precision == OCCRI_FP64 ? 16 : 8);
  q.vq = wave_tables ? nullptr : vq;
  for (int d = 0; d < 3; ++d) q.D[d] = D[d];
  q.kint = kint;
  // reciprocal vectors b_i (rows): B = 2 pi (A^{-1})^T
  double inv[3][3];
  const double (*a)[3] = lat;
  const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                     a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                     a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
  inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
  inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
  inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
  inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
  inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
  inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
  inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
  inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
  double b[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b[i][j] = 2.0 * kPiD * inv[j][i];
  auto dot = [&](int i, int j) { return b[i][0] * b[j][0] + b[i][1] * b[j][1] + b[i][2] * b[j][2]; };
  q.g[0] = dot(0, 0); q.g[1] = dot(1, 1); q.g[2] = dot(2, 2);
  q.g[3] = dot(0, 1); q.g[4] = dot(0, 2); q.g[5] = dot(1, 2);
  q.kind = kernel.kind;
  q.omega = kernel.omega;
  const bool has_w = kernel.kind == OCCRI_ERFC || kernel.kind == OCCRI_ERF;
  q.inv4w2 = has_w ? 1.0 / (4.0 * kernel.omega * kernel.omega) : 0.0;
  q.g0 = g0_4pi;
  q.dg0 = dg0_4pi;
  q.rc = rc;
  for (int n = 0; n < kFadN; ++n) q.fad_a[n] = fad_a[n];
  q.fad_L = fad_L;
  q.lr_erf = lr_erf;
  q.lr_exp = lr_exp;
  for (int i = 0; i < 6; ++i) {
    q.gh[i] = (float)q.g[i];
    q.gl[i] = (float)(q.g[i] - (double)q.gh[i]);
  }
  q.inv4w2_f = (float)q.inv4w2;
  q.omega_f = (float)q.omega;
  q.g0_f = (float)q.g0;
  q.dg0_f = (float)q.dg0;
  return q;
}

// ------------------------------------------------------------------ primitives (host)

namespace {

struct Mono { int a, b, c; double v; };

// Real solid harmonics in AO order as monomial lists.
const std::vector<std::vector<Mono>>& solid_table(int l) {
  static const std::vector<std::vector<Mono>> t0 = {{{0, 0, 0, 1.0}}};
  static const std::vector<std::vector<Mono>> t1 = {
      {{1, 0, 0, 1.0}}, {{0, 1, 0, 1.0}}, {{0, 0, 1, 1.0}}};
  static const std::vector<std::vector<Mono>> t2 = {
      {{1, 1, 0, 1.0}},
      {{0, 1, 1, 1.0}},
      {{0, 0, 2, 2.0}, {2, 0, 0, -1.0}, {0, 2, 0, -1.0}},
      {{1, 0, 1, 1.0}},
      {{2, 0, 0, 1.0}, {0, 2, 0, -1.0}}};
  static const std::vector<std::vector<Mono>> t3 = {
      {{2, 1, 0, 3.0}, {0, 3, 0, -1.0}},
      {{1, 1, 1, 1.0}},
      {{0, 1, 2, 4.0}, {2, 1, 0, -1.0}, {0, 3, 0, -1.0}},
      {{0, 0, 3, 2.0}, {2, 0, 1, -3.0}, {0, 2, 1, -3.0}},
      {{1, 0, 2, 4.0}, {3, 0, 0, -1.0}, {1, 2, 0, -1.0}},
      {{2, 0, 1, 1.0}, {0, 2, 1, -1.0}},
      {{3, 0, 0, 1.0}, {1, 2, 0, -3.0}}};
  switch (l) {
    case 0: return t0;
    case 1: return t1;
    case 2: return t2;
    default: return t3;
  }
}

double odd_factorial(int n) {  // (n)!! for odd n >= -1
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

// integral of x^a y^b z^c exp(-p r^2) over R^3
double moment(int a, int b, int c, double p) {
  double r = 1.0;
  const int e[3] = {a, b, c};
  for (int d = 0; d < 3; ++d) {
    if (e[d] % 2) return 0.0;
    r *= odd_factorial(e[d] - 1) / std::pow(2.0 * p, e[d] / 2) * std::sqrt(kPiD / p);
  }
  return r;
}

void shell_norms(int l, double alpha, double* out) {
  const auto& tab = solid_table(l);
  for (size_t m = 0; m < tab.size(); ++m) {
    double s = 0.0;
    for (const Mono& x : tab[m])
      for (const Mono& y : tab[m]) s += x.v * y.v * moment(x.a + y.a, x.b + y.b, x.c + y.c, 2.0 * alpha);
    out[m] = 1.0 / std::sqrt(s);
  }
}

// Radius beyond which N_lm |P_lm| e^{-alpha r^2} < eps for every m (|P_lm| <= sum|coeff| r^l).
double shell_cutoff(int l, double alpha, double eps) {
  double nrm[7];
  shell_norms(l, alpha, nrm);
  const auto& tab = solid_table(l);
  double c = 0.0;
  for (size_t m = 0; m < tab.size(); ++m) {
    double s = 0.0;
    for (const Mono& x : tab[m]) s += std::fabs(x.v);
    c = std::max(c, nrm[m] * s);
  }
  auto f = [&](double r) {
    return std::log(c) + l * std::log(std::max(r, 1e-300)) - alpha * r * r - std::log(eps);
  };
  double lo = (l > 0) ? std::sqrt(l / (2.0 * alpha)) : 0.0;
  if (f(lo) <= 0) return lo;
  double hi = std::max(lo, 1.0);
  while (f(hi) > 0) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (f(mid) > 0) lo = mid; else hi = mid;
  }
  return hi;
}

bool smooth235(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

void inv3(const double a[3][3], double inv[3][3]) {
  const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                     a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                     a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
  inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
  inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
  inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
  inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
  inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
  inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
  inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
  inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
}

// Sums over the lattice with rows L (or, with recip, over its reciprocal lattice) of
// fn(vector) for every nonzero vector, shell by shell (|i|,|j|,|k| <= n with max = n) until a
// whole shell adds less than 1e-17 (from the third shell on).
template <typename F>
double lattice_shell_sum(const double L[3][3], bool recip, F fn) {
  double v[3][3];
  if (recip) {
    double inv[3][3];
    inv3(L, inv);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) v[i][j] = 2.0 * kPiD * inv[j][i];
  } else {
    std::memcpy(v, L, sizeof(v));
  }
  double total = 0.0;
  for (int n = 1; n < 200; ++n) {
    double shell = 0.0;
    for (int i = -n; i <= n; ++i)
      for (int j = -n; j <= n; ++j)
        for (int k = -n; k <= n; ++k) {
          if (std::max(std::abs(i), std::max(std::abs(j), std::abs(k))) != n) continue;
          const double x[3] = {i * v[0][0] + j * v[1][0] + k * v[2][0],
                               i * v[0][1] + j * v[1][1] + k * v[2][1],
                               i * v[0][2] + j * v[1][2] + k * v[2][2]};
          shell += fn(x);
        }
    total += shell;
    if (n > 2 && std::fabs(shell) < 1e-17) break;
  }
  return total;
}

double volume3(const double L[3][3]) {
  return std::fabs(L[0][0] * (L[1][1] * L[2][2] - L[1][2] * L[2][1]) -
                   L[0][1] * (L[1][0] * L[2][2] - L[1][2] * L[2][0]) +
                   L[0][2] * (L[1][0] * L[2][1] - L[1][1] * L[2][0]));
}

// Coefficients of Weideman's rational approximation of the Faddeeva function in the upper
// half plane (J. A. C. Weideman, SIAM J. Numer. Anal. 31 (1994) 1497): with L = (N/sqrt 2)^{1/2}
// and t(theta) = L tan(theta/2), the coefficients are the cosine transform, over the 2M = 4N
// equispaced angles theta = k pi/M, of e^{-t^2} (L^2 + t^2) (zero at theta = -pi):
//   a[n] = (1/2M) sum_k f(theta_k) cos(n theta_k),  n = 1..N,
// and w(z) = 2 sum_n a[n] Z^{n-1} / (L - i z)^2 + 1/(sqrt(pi) (L - i z)), Z = (L + i z)/(L - i z).
// fad[n - 1] receives a[n].
void faddeeva_coefficients(double* fad, double* L_out) {
  const int N = kFadN, M = 2 * N;
  const double L = std::sqrt(N / std::sqrt(2.0));
  for (int n = 1; n <= N; ++n) {
    double s = 0.0;
    for (int k = -M + 1; k < M; ++k) {
      const double theta = k * kPiD / M;
      const double t = L * std::tan(0.5 * theta);
      s += std::exp(-t * t) * (L * L + t * t) * std::cos(n * theta);
    }
    fad[n - 1] = s / (2.0 * M);
  }
  *L_out = L;
}

// Ewald potential at a unit point charge from its periodic images in a uniform neutralising
// background (the lattice's Madelung potential; negative), splitting parameter eta from the
// cell volume.
double madelung_potential(const double L[3][3]) {
  const double vol = volume3(L);
  const double eta = std::sqrt(kPiD) / std::cbrt(vol);
  const double real = lattice_shell_sum(L, false, [&](const double* x) {
    const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    return std::erfc(eta * r) / r;
  });
  const double recip = lattice_shell_sum(L, true, [&](const double* g) {
    const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    return 4.0 * kPiD / vol * std::exp(-g2 / (4.0 * eta * eta)) / g2;
  });
  return real + recip - kPiD / (eta * eta * vol) - 2.0 * eta / std::sqrt(kPiD);
}

// chi of the erf kernel: V 2 w/sqrt(pi) - sum_{G != 0} 4 pi e^{-G^2/(4 w^2)}/G^2 over the
// supercell's reciprocal lattice, and its omega-derivative in *dchi.
double erf_lattice_chi(const double L[3][3], double w, double* dchi) {
  const double vol = volume3(L);
  const double s = lattice_shell_sum(L, true, [&](const double* g) {
    const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    return 4.0 * kPiD * std::exp(-g2 / (4.0 * w * w)) / g2;
  });
  const double ds = lattice_shell_sum(L, true, [&](const double* g) {
    const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    return 2.0 * kPiD * std::exp(-g2 / (4.0 * w * w)) / (w * w * w);
  });
  *dchi = 2.0 * vol / std::sqrt(kPiD) - ds;
  return vol * 2.0 * w / std::sqrt(kPiD) - s;
}

template <typename X>
cudaError_t dalloc(X** p, size_t count, size_t* total) {
  *total += count * sizeof(X);
  return device_malloc((void**)p, std::max<size_t>(count, 1) * sizeof(X));
}

template <typename X>
cudaError_t upload(X** p, const std::vector<X>& v, size_t* total) {
  cudaError_t e = dalloc(p, v.size(), total);
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpy(*p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice);
}

// ------------------------------------------------------------------ step (f) kernels

__device__ void record_status(int* status, int code, int k) {
  if (atomicCAS(status, 0, code) == 0) status[1] = k;
}

// One CTA per k: M = C^H KC (Hermitised), -M = L L^H, xi = KC L^{-H},
// K = -xi xi^H, ek[k] = Re Tr M.
__global__ void __launch_bounds__(256)
ace_kernel(const double2* __restrict__ C, const double2* __restrict__ kc, double2* __restrict__ xi,
           double2* __restrict__ mout, double* __restrict__ ek, double2* __restrict__ K, int nao,
           int nocc, double pivot_tol, int* status) {
  extern __shared__ double2 sm[];
  double2* M = sm;                   // nocc*nocc
  double2* L = sm + nocc * nocc;     // nocc*nocc
  __shared__ int ok;
  const int k = blockIdx.x;
  const double2* Ck = C + (size_t)k * nao * nocc;
  const double2* KCk = kc + (size_t)k * nao * nocc;
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) {
    const int i = e / nocc, j = e - (e / nocc) * nocc;
    double sr = 0.0, si = 0.0;
    for (int mu = 0; mu < nao; ++mu) {
      const double2 c = Ck[(size_t)mu * nocc + i], x = KCk[(size_t)mu * nocc + j];
      sr += c.x * x.x + c.y * x.y;   // conj(c) * x
      si += c.x * x.y - c.y * x.x;
    }
    L[e] = make_double2(sr, si);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) {
    const int i = e / nocc, j = e - (e / nocc) * nocc;
    const double2 a = L[i * nocc + j], b = L[j * nocc + i];
    M[e] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    double tr = 0.0;
    for (int i = 0; i < nocc; ++i) tr += M[i * nocc + i].x;
    ek[k] = tr;
    for (int e = 0; e < nocc * nocc; ++e) mout[(size_t)k * nocc * nocc + e] = M[e];
    // Cholesky of A = -M (lower, complex Hermitian); a pivot at or below
    // pivot_tol * max_j A_jj counts as not positive definite.
    double amax = 0.0;
    for (int j = 0; j < nocc; ++j) amax = fmax(amax, -M[j * nocc + j].x);
    for (int j = 0; j < nocc && ok; ++j) {
      double d = -M[j * nocc + j].x;
      for (int l = 0; l < j; ++l) d -= L[j * nocc + l].x * L[j * nocc + l].x + L[j * nocc + l].y * L[j * nocc + l].y;
      if (!(d > pivot_tol * amax) || !isfinite(d)) { ok = 0; break; }
      const double ljj = sqrt(d);
      L[j * nocc + j] = make_double2(ljj, 0.0);
      for (int i = j + 1; i < nocc; ++i) {
        double ar = -M[i * nocc + j].x, ai = -M[i * nocc + j].y;
        for (int l = 0; l < j; ++l) {  // - L_il conj(L_jl)
          const double2 x = L[i * nocc + l], y = L[j * nocc + l];
          ar -= x.x * y.x + x.y * y.y;
          ai -= x.y * y.x - x.x * y.y;
        }
        L[i * nocc + j] = make_double2(ar / ljj, ai / ljj);
      }
      for (int i = 0; i < j; ++i) L[i * nocc + j] = make_double2(0.0, 0.0);
    }
    if (!ok) record_status(status, OCCRI_ENOTPD, k);
  }
  __syncthreads();
  if (!ok) return;
  // xi L^H = KC  ->  xi_j = (KC_j - sum_{l<j} xi_l conj(L_jl)) / L_jj
  double2* xik = xi + (size_t)k * nao * nocc;
  for (int mu = threadIdx.x; mu < nao; mu += blockDim.x) {
    for (int j = 0; j < nocc; ++j) {
      double2 v = KCk[(size_t)mu * nocc + j];
      for (int l = 0; l < j; ++l) {
        const double2 x = xik[(size_t)mu * nocc + l], y = L[j * nocc + l];
        v.x -= x.x * y.x + x.y * y.y;
        v.y -= x.y * y.x - x.x * y.y;
      }
      const double ljj = L[j * nocc + j].x;
      xik[(size_t)mu * nocc + j] = make_double2(v.x / ljj, v.y / ljj);
    }
  }
  __syncthreads();
  if (K == nullptr) return;
  double2* Kk = K + (size_t)k * nao * nao;
  for (size_t e = threadIdx.x; e < (size_t)nao * nao; e += blockDim.x) {
    const int mu = (int)(e / nao), nu = (int)(e - (e / nao) * nao);
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < nocc; ++j) {  // xi_mu conj(xi_nu)
      const double2 a = xik[(size_t)mu * nocc + j], b = xik[(size_t)nu * nocc + j];
      sr += a.x * b.x + a.y * b.y;
      si += a.y * b.x - a.x * b.y;
    }
    Kk[e] = make_double2(-sr, -si);
  }
}

__global__ void ex_kernel(const double* __restrict__ ek, int nk, double* __restrict__ ex) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nk; ++k) s += ek[k];
    *ex = s / nk;
  }
}

__global__ void scale_copy_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                  long long n, double s) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = make_double2(s * in[e].x, s * in[e].y);
}

__global__ void domega_finish_kernel(const double* __restrict__ acc, double s, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = s * acc[0];
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// Adjoint of the ACE assembly and of E_x, one CTA per k (FP64). With K = KC M^{-1} KC^H,
// M = herm(C^H KC), E_x = (1/N_k) sum_k Re Tr M and the seeds G = dL/dK (gK, or none),
// gKC (or none) and gE = dL/dE_x / N_k, in the convention dL = Re <grad, d.>:
//   grad_KC = G KC M^{-1} + G^H KC M^{-1} - C H + gE C + gKC,
//   grad_C  = -KC H + gE KC   (the part through the assembly), H = herm(M^{-1} KC^H G KC M^{-1}).
// T = G KC and U = G^H KC are formed row by row; T + U is parked in gcf until the row of
// grad_KC has been written.
__global__ void __launch_bounds__(256)
ace_adjoint_kernel(const double2* __restrict__ C, const double2* __restrict__ kc,
                   const double2* __restrict__ mmat, const double2* __restrict__ gK,
                   const double2* __restrict__ gKC, double gE, double2* __restrict__ gkc,
                   double2* __restrict__ gcf, int nao, int nocc, double pivot_tol, int* status) {
  extern __shared__ double2 sm[];
  double2* A = sm;                     // L, then L^{-1}, then herm(H)
  double2* Minv = sm + nocc * nocc;
  double2* Pm = sm + 2 * nocc * nocc;  // KC^H T, then H
  __shared__ int ok;
  const int k = blockIdx.x;
  const double2* Ck = C + (size_t)k * nao * nocc;
  const double2* KCk = kc + (size_t)k * nao * nocc;
  const double2* Mk = mmat + (size_t)k * nocc * nocc;
  double2* gk = gkc + (size_t)k * nao * nocc;
  double2* fk = gcf + (size_t)k * nao * nocc;
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) Pm[e] = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
    // -M = L L^H (as in the assembly), L^{-1}, then M^{-1} = -L^{-H} L^{-1}
    ok = 1;
    double amax = 0.0;
    for (int j = 0; j < nocc; ++j) amax = fmax(amax, -Mk[j * nocc + j].x);
    for (int j = 0; j < nocc && ok; ++j) {
      double d = -Mk[j * nocc + j].x;
      for (int l = 0; l < j; ++l) d -= A[j * nocc + l].x * A[j * nocc + l].x + A[j * nocc + l].y * A[j * nocc + l].y;
      if (!(d > pivot_tol * amax) || !isfinite(d)) { ok = 0; break; }
      const double ljj = sqrt(d);
      A[j * nocc + j] = make_double2(ljj, 0.0);
      for (int i = j + 1; i < nocc; ++i) {
        double ar = -Mk[i * nocc + j].x, ai = -Mk[i * nocc + j].y;
        for (int l = 0; l < j; ++l) {
          const double2 x = A[i * nocc + l], y = A[j * nocc + l];
          ar -= x.x * y.x + x.y * y.y;
          ai -= x.y * y.x - x.x * y.y;
        }
        A[i * nocc + j] = make_double2(ar / ljj, ai / ljj);
      }
    }
    if (ok) {
      // lower-triangular inverse in place, column by column (entries below the diagonal
      // of column j use the diagonal entries of later rows, still those of L)
      for (int j = 0; j < nocc; ++j) {
        const double inv = 1.0 / A[j * nocc + j].x;
        for (int i = j + 1; i < nocc; ++i) {
          double2 acc = make_double2(0.0, 0.0);
          for (int l = j; l < i; ++l) {
            const double2 a = A[i * nocc + l];   // L_il (row i is still L to the left of i)
            const double2 b = (l == j) ? make_double2(inv, 0.0) : A[l * nocc + j];   // Linv_lj
            acc.x += a.x * b.x - a.y * b.y;
            acc.y += a.x * b.y + a.y * b.x;
          }
          const double lii = A[i * nocc + i].x;
          A[i * nocc + j] = make_double2(-acc.x / lii, -acc.y / lii);
        }
      }
      for (int j = 0; j < nocc; ++j) A[j * nocc + j] = make_double2(1.0 / A[j * nocc + j].x, 0.0);
      for (int i = 0; i < nocc; ++i)
        for (int j = 0; j < nocc; ++j) {
          double2 acc = make_double2(0.0, 0.0);
          for (int l = (i > j ? i : j); l < nocc; ++l) {
            const double2 t = zmulc(A[l * nocc + i], A[l * nocc + j]);
            acc.x += t.x;
            acc.y += t.y;
          }
          Minv[i * nocc + j] = make_double2(-acc.x, -acc.y);
        }
    } else {
      record_status(status, OCCRI_ENOTPD, k);
    }
  }
  __syncthreads();
  if (!ok) return;
  if (gK) {   // T + U parked in gcf; Pm += KC^H T
    const double2* Gk = gK + (size_t)k * nao * nao;
    for (int mu = threadIdx.x; mu < nao; mu += blockDim.x) {
      for (int j = 0; j < nocc; ++j) {
        double2 t = make_double2(0.0, 0.0), u = make_double2(0.0, 0.0);
        for (int nu = 0; nu < nao; ++nu) {
          const double2 x = KCk[(size_t)nu * nocc + j];
          const double2 a = zmul(Gk[(size_t)mu * nao + nu], x);
          const double2 b = zmulc(Gk[(size_t)nu * nao + mu], x);
          t.x += a.x; t.y += a.y;
          u.x += b.x; u.y += b.y;
        }
        fk[(size_t)mu * nocc + j] = make_double2(t.x + u.x, t.y + u.y);
        for (int i = 0; i < nocc; ++i) {
          const double2 v = zmulc(KCk[(size_t)mu * nocc + i], t);
          atomicAdd(&Pm[i * nocc + j].x, v.x);
          atomicAdd(&Pm[i * nocc + j].y, v.y);
        }
      }
    }
  }
  __syncthreads();
  // H = M^{-1} Pm M^{-1} (through A), then herm(H) into A
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) {
    const int i = e / nocc, j = e - (e / nocc) * nocc;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < nocc; ++l) {
      const double2 t = zmul(Pm[i * nocc + l], Minv[l * nocc + j]);
      acc.x += t.x; acc.y += t.y;
    }
    A[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) {
    const int i = e / nocc, j = e - (e / nocc) * nocc;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < nocc; ++l) {
      const double2 t = zmul(Minv[i * nocc + l], A[l * nocc + j]);
      acc.x += t.x; acc.y += t.y;
    }
    Pm[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) {
    const int i = e / nocc, j = e - (e / nocc) * nocc;
    const double2 a = Pm[i * nocc + j], b = Pm[j * nocc + i];
    A[e] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
  __syncthreads();
  for (int mu = threadIdx.x; mu < nao; mu += blockDim.x) {
    const size_t row = (size_t)mu * nocc;
    for (int i = 0; i < nocc; ++i) {
      double2 g = make_double2(gE * Ck[row + i].x, gE * Ck[row + i].y);
      if (gKC) {
        g.x += gKC[(size_t)k * nao * nocc + row + i].x;
        g.y += gKC[(size_t)k * nao * nocc + row + i].y;
      }
      for (int l = 0; l < nocc; ++l) {
        const double2 t = zmul(Ck[row + l], A[l * nocc + i]);
        g.x -= t.x; g.y -= t.y;
        if (gK) {
          const double2 v = zmul(fk[row + l], Minv[l * nocc + i]);
          g.x += v.x; g.y += v.y;
        }
      }
      gk[row + i] = g;
    }
    for (int i = 0; i < nocc; ++i) {
      double2 f = make_double2(gE * KCk[row + i].x, gE * KCk[row + i].y);
      for (int l = 0; l < nocc; ++l) {
        const double2 t = zmul(KCk[row + l], A[l * nocc + i]);
        f.x -= t.x; f.y -= t.y;
      }
      fk[row + i] = f;
    }
  }
}

// y += a + b over n complex values (the streams' private accumulators into Y)
template <typename C2>
__global__ void add3_kernel(C2* __restrict__ y, const C2* __restrict__ a, const C2* __restrict__ b,
                            long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    C2 v = y[i];
    const C2 u = a[i], w = b[i];
    v.x += u.x + w.x;
    v.y += u.y + w.y;
    y[i] = v;
  }
}

__global__ void add_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                           double2* __restrict__ out, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = make_double2(a[e].x + b[e].x, a[e].y + b[e].y);
}

void free_plan(Plan* p) {
  if (!p) return;
  void* bufs[] = {p->shells, p->atom_shell0, p->img_d, p->img_hi, p->img_lo, p->img_phase,
                  p->d0_d, p->d0_hi, p->d0_lo, p->t0, p->kint, p->psi, p->Y, p->scratch,
                  p->kc, p->xi, p->mmat, p->ek, p->dacc, p->status, p->h_c, p->h_kc, p->h_k,
                  p->h_ex, p->ao_norm, p->cs, p->blist, p->bpre, p->shell_list_l[0], p->shell_list_l[1], p->shell_list_l[2],
                  p->shell_list_l[3]};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p->scratch2) cudaFree(p->scratch2);
  if (p->scratch3) cudaFree(p->scratch3);
  if (p->vq) cudaFree(p->vq);
  for (void* yx : p->Yx)
    if (yx) cudaFree(yx);
  if (p->asm_scratch) cudaFree(p->asm_scratch);
  for (void* b : {p->gam, p->gpsi, p->cs_g, (void*)p->gkc, (void*)p->gcf, (void*)p->gacc})
    if (b) cudaFree(b);
  for (cudaEvent_t e : {p->ev_fork, p->ev_join, p->ev_y, p->ev_iso, p->ev_join2, p->ev_iso2,
                        p->ev_iso3})
    if (e) cudaEventDestroy(e);
  if (p->aux) cudaStreamDestroy(p->aux);
  if (p->aux2) cudaStreamDestroy(p->aux2);
  if (p->tc) tc_plan_free(p->tc);
  for (cudaEvent_t e : p->ev_used) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_free) cudaEventDestroy(e);
  delete p;
}

}  // namespace

}  // namespace occri

using occri::Plan;

namespace occri_impl {

cudaEvent_t take_event(Plan* p) {
  cudaEvent_t e = nullptr;
  if (!p->ev_free.empty()) {
    e = p->ev_free.back();
    p->ev_free.pop_back();
  } else if (p->ev_used.size() < 200000) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  } else {
    return nullptr;
  }
  p->ev_used.push_back(e);
  return e;
}

// Bracket one stage with a pair of events (no-op when timing is off).
struct StageTimer {
  Plan* p;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageTimer(Plan* pl, bool on, cudaStream_t stream = nullptr)
      : p(pl), st(stream ? stream : pl->stream) {
    if (on) {
      a = take_event(p);
      if (a && cudaEventRecord(a, st) != cudaSuccess) {
        cudaGetLastError();
        a = nullptr;   // this stage goes untimed
      }
    }
  }
  void done(int stage, double units) {
    if (!a) return;
    cudaEvent_t b = take_event(p);
    if (!b) return;
    if (cudaEventRecord(b, st) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    p->ev_pending.push_back(Plan::TimedSpan{a, b, stage, units});
  }
};

template <typename T>
int build_impl(Plan* p, const double2* C, void* KC, void* K, double* Ex) {
  using namespace occri;
  cudaStream_t s = p->stream;
  const bool timed = p->timing_every != 0;   // > 0: sampled waves too; -1: stage spans only
  long long launches = 0;
  const size_t orb = (size_t)p->nk * p->nocc * p->fs;
  if (cudaMemsetAsync(p->Y, 0, orb * sizeof(cplx_t<T>), s) != cudaSuccess) return OCCRI_ECUDA;
  for (void* yx : p->Yx)
    if (yx && cudaMemsetAsync(yx, 0, orb * sizeof(cplx_t<T>), s) != cudaSuccess)
      return OCCRI_ECUDA;
  if (cudaMemsetAsync(p->kc, 0, sizeof(double2) * (size_t)p->nk * p->nao * p->nocc, s) != cudaSuccess)
    return OCCRI_ECUDA;
  {
    StageTimer t(p, timed);
    if (launch_scale_c<T>(*p, C, s) != cudaSuccess) return OCCRI_ECUDA;
    if (launch_orbitals<T>(*p, s) != cudaSuccess) return OCCRI_ECUDA;
    // the pair passes work on the periodic parts u = e^{-ik.r} psi: the pair density
    // conj(u_jk') u_ik is then periodic as it stands, and the accumulated periodic part
    // e^{-ik.r} Y_ik needs no phase either (Y is restored below)
    if (launch_phase_fields<T>(*p, p->psi, -1, s) != cudaSuccess) return OCCRI_ECUDA;
    t.done(OCCRI_STAGE_ORBITALS, p->nk);
    launches += 2 + (p->nocc + kOrbChunk - 1) / kOrbChunk;
  }
  {
    // Waves go round-robin over the plan's stream and one or two auxiliary ones, each with
    // its own scratch; the accumulation passes (which update Y_k) are chained across the
    // streams by ev_y. A sampled wave runs alone (the streams wait for each other around
    // it) so that its pass times are not mixed with another stream's work.
    StageTimer all(p, timed);
    const int ns = p->nstreams;
    cudaStream_t st[3] = {s, p->aux, p->aux2};
    void* sc[3] = {p->scratch, p->scratch2, p->scratch3};
    // with private accumulators per stream, no wave waits for another stream's Y updates
    const bool split_y = p->Yx[0] && p->Yx[1];
    void* yacc[3] = {p->Y, split_y ? p->Yx[0] : p->Y, split_y ? p->Yx[1] : p->Y};
    cudaEvent_t ev_y = split_y ? nullptr : p->ev_y;
    cudaEvent_t join[3] = {nullptr, p->ev_join, p->ev_join2};
    cudaEvent_t iso[3] = {p->ev_iso, p->ev_iso2, p->ev_iso3};
    if (cudaEventRecord(p->ev_fork, s) != cudaSuccess) return OCCRI_ECUDA;
    for (int o = 1; o < ns; ++o)
      if (cudaStreamWaitEvent(st[o], p->ev_fork, 0) != cudaSuccess) return OCCRI_ECUDA;
    // the first wave's accumulation waits on this record (within the same build, which
    // keeps the chain inside a captured graph when the build is captured)
    if (cudaEventRecord(p->ev_y, s) != cudaSuccess) return OCCRI_ECUDA;
    // every other stream's work so far precedes the next work of stream w
    auto isolate = [&](int w) {
      for (int o = 0; o < ns; ++o)
        if (o != w && (cudaEventRecord(iso[o], st[o]) != cudaSuccess ||
                       cudaStreamWaitEvent(st[w], iso[o], 0) != cudaSuccess))
          return false;
      return true;
    };
    double fields = 0.0;
    long long wave = 0;
    for (int k = 0; k < p->nk; ++k)
      for (int kp0 = k; kp0 < p->nk; ++wave) {   // unordered pairs: (k, k), then k' > k
        const int diag = (kp0 == k) ? 1 : 0;
        const int nkp = diag ? 1 : std::min(p->nkp_wave, p->nk - kp0);
        const int w = (int)(wave % ns);
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        bool sample = p->timing_every > 0 && (wave % p->timing_every == 0);
        if (sample)
          for (int i = 0; i < 4 && sample; ++i) sample = (ev[i] = take_event(p)) != nullptr;
        if (sample && !isolate(w)) return OCCRI_ECUDA;   // wait for the other streams' work
        if (launch_pair_wave<T>(*p, k, kp0, nkp, diag, st[w], sc[w], yacc[w],
                                sample ? ev : nullptr, ev_y) != cudaSuccess)
          return OCCRI_ECUDA;
        launches += pair_wave_launches<T>(p->nocc, p->split_cd);
        const double nf = (double)wave_fields(p->nocc, nkp, diag);
        fields += nf;
        if (sample) {   // and keep the other streams waiting until this wave is done
          if (cudaEventRecord(iso[w], st[w]) != cudaSuccess) return OCCRI_ECUDA;
          for (int o = 0; o < ns; ++o)
            if (o != w && cudaStreamWaitEvent(st[o], iso[w], 0) != cudaSuccess) return OCCRI_ECUDA;
          p->ev_pending.push_back(Plan::TimedSpan{ev[0], ev[1], OCCRI_STAGE_PAIR_A, nf});
          p->ev_pending.push_back(Plan::TimedSpan{ev[1], ev[2], OCCRI_STAGE_PAIR_B, nf});
          p->ev_pending.push_back(Plan::TimedSpan{ev[2], ev[3], OCCRI_STAGE_PAIR_C, nf});
        }
        kp0 += nkp;
      }
    for (int o = 1; o < ns; ++o)
      if (cudaEventRecord(join[o], st[o]) != cudaSuccess ||
          cudaStreamWaitEvent(s, join[o], 0) != cudaSuccess)
        return OCCRI_ECUDA;
    if (split_y) {
      add3_kernel<<<8 * 152, 256, 0, s>>>((cplx_t<T>*)p->Y, (const cplx_t<T>*)p->Yx[0],
                                          (const cplx_t<T>*)p->Yx[1], (long long)orb);
      ++launches;
    }
    all.done(OCCRI_STAGE_PAIRS, fields);
  }
  {
    StageTimer t(p, timed);
    if (launch_phase_fields<T>(*p, p->Y, +1, s) != cudaSuccess) return OCCRI_ECUDA;
    ++launches;
    if (p->tc) {
      // the GEMM kernels alone, one span per slab (stage OCCRI_STAGE_CONTRACT_GEMM)
      struct GemmSpans : LaunchHook {
        Plan* p;
        cudaStream_t s;
        bool on;
        StageTimer* t = nullptr;
        GemmSpans(Plan* pl, cudaStream_t st, bool timed) : p(pl), s(st), on(timed) {}
        void before() override {
          if (on) t = new StageTimer(p, true, s);
        }
        void after() override {
          if (t) t->done(OCCRI_STAGE_CONTRACT_GEMM, 1.0);
          delete t;
          t = nullptr;
        }
      } spans(p, s, timed);
      if (launch_contract_tc(*p, s, &spans) != cudaSuccess) return OCCRI_ECUDA;
      launches += tc_plan_launches(p->tc);
    } else {
      if (launch_contract<T>(*p, s) != cudaSuccess) return OCCRI_ECUDA;
      for (int l = 0; l < 4; ++l)
        if (!p->shells_by_l[l].empty())
          launches += (p->nocc + contract_chunk<T>() - 1) / contract_chunk<T>();
    }
    t.done(OCCRI_STAGE_CONTRACT, p->nk);
  }
  {
    StageTimer t(p, timed);
    const size_t sm = 2 * sizeof(double2) * (size_t)p->nocc * p->nocc;
    const double tol = (p->precision == OCCRI_FP64) ? 1e-10 : 1e-5;
    ace_kernel<<<p->nk, 256, sm, s>>>(C, p->kc, p->xi, p->mmat, p->ek, (double2*)K, p->nao,
                                      p->nocc, tol, p->status);
    ++launches;
    if (Ex) {
      ex_kernel<<<1, 32, 0, s>>>(p->ek, p->nk, Ex);
      ++launches;
    }
    t.done(OCCRI_STAGE_ASSEMBLE, p->nk);
  }
  if (KC &&
      cudaMemcpyAsync(KC, p->kc, sizeof(double2) * (size_t)p->nk * p->nao * p->nocc,
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return OCCRI_ECUDA;
  if (cudaGetLastError() != cudaSuccess) return OCCRI_ECUDA;
  p->have_kc = true;
  p->launches_per_build = launches;
  return OCCRI_OK;
}

template <typename T>
int vjp_impl(Plan* p, const double2* C, double gEx, void* gC, double* gomega) {
  using namespace occri;
  cudaStream_t s = p->stream;
  const long long nkc = (long long)p->nk * p->nao * p->nocc;
  if (gC) scale_copy_kernel<<<4 * 152, 256, 0, s>>>(p->kc, (double2*)gC, nkc, gEx * 4.0 / p->nk);
  if (gomega) {
    if (cudaMemsetAsync(p->dacc, 0, 2 * sizeof(double), s) != cudaSuccess) return OCCRI_ECUDA;
    if (p->kernel.kind == OCCRI_ERFC || p->kernel.kind == OCCRI_ERF) {
      // periodic parts of the orbitals of C (the plan's copy may have been replaced by
      // an occri_orbitals call since the build)
      if (launch_scale_c<T>(*p, C, s) != cudaSuccess) return OCCRI_ECUDA;
      if (launch_orbitals<T>(*p, s) != cudaSuccess) return OCCRI_ECUDA;
      if (launch_phase_fields<T>(*p, p->psi, -1, s) != cudaSuccess) return OCCRI_ECUDA;
      for (int k = 0; k < p->nk; ++k)
        for (int kp0 = k; kp0 < p->nk;) {
          const int diag = (kp0 == k) ? 1 : 0;
          const int nkp = diag ? 1 : std::min(p->nkp_wave, p->nk - kp0);
          if (launch_domega_wave<T>(*p, k, kp0, nkp, diag, s) != cudaSuccess) return OCCRI_ECUDA;
          kp0 += nkp;
        }
    }
    const double ngd = (double)p->ng;
    const double sc = -gEx * p->omega_cell * 4.0 * kPiD / ((double)p->nk * p->nk) / (ngd * ngd);
    domega_finish_kernel<<<1, 32, 0, s>>>(p->dacc, sc, gomega);
  }
  return cudaGetLastError() == cudaSuccess ? OCCRI_OK : OCCRI_ECUDA;
}

// Adjoint of the whole build for the seeds gEx, gKC, gK (see occri_vjp_full).
template <typename T>
int vjp_full_impl(Plan* p, const double2* C, double gEx, const double2* gKC, const double2* gK,
                  double2* gC, double* gomega) {
  using namespace occri;
  cudaStream_t s = p->stream;
  const size_t nkc = (size_t)p->nk * p->nao * p->nocc;
  const size_t orb = (size_t)p->nk * p->nocc * p->fs * sizeof(cplx_t<T>);
  const size_t csb = (p->precision == OCCRI_FP64 ? sizeof(double2) : sizeof(float4)) * nkc;
  if (!p->gam) {   // first call: the adjoint workspaces
    bool ok = device_malloc(&p->gam, orb) == cudaSuccess &&
              device_malloc(&p->gpsi, orb) == cudaSuccess &&
              device_malloc(&p->cs_g, csb) == cudaSuccess &&
              device_malloc((void**)&p->gkc, nkc * sizeof(double2)) == cudaSuccess &&
              device_malloc((void**)&p->gcf, nkc * sizeof(double2)) == cudaSuccess &&
              device_malloc((void**)&p->gacc, nkc * sizeof(double2)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      for (void** b : {&p->gam, &p->gpsi, &p->cs_g, (void**)&p->gkc, (void**)&p->gcf,
                       (void**)&p->gacc}) {
        if (*b) cudaFree(*b);
        *b = nullptr;
      }
      return OCCRI_ENOMEM;
    }
  }
  // (f): the assembly's adjoint
  const double tol = (p->precision == OCCRI_FP64) ? 1e-10 : 1e-5;
  const size_t sm = 3 * sizeof(double2) * (size_t)p->nocc * p->nocc;
  ace_adjoint_kernel<<<p->nk, 256, sm, s>>>(C, p->kc, p->mmat, gK, gKC, gEx / p->nk, p->gkc,
                                            p->gcf, p->nao, p->nocc, tol, p->status);
  // the adjoint orbital field g = -sum_mu chi_mu dL/dKC_mu (in units that leave out the
  // contraction's Omega/(N_k N_g)) and the orbitals of C, both as periodic parts
  if (launch_scale_to<T>(*p, p->gkc, p->cs_g, -1.0, s) != cudaSuccess) return OCCRI_ECUDA;
  if (launch_orbitals_to<T>(*p, p->cs_g, p->gam, s) != cudaSuccess) return OCCRI_ECUDA;
  if (launch_phase_fields<T>(*p, p->gam, -1, s) != cudaSuccess) return OCCRI_ECUDA;
  if (launch_scale_c<T>(*p, C, s) != cudaSuccess) return OCCRI_ECUDA;
  if (launch_orbitals<T>(*p, s) != cudaSuccess) return OCCRI_ECUDA;
  if (launch_phase_fields<T>(*p, p->psi, -1, s) != cudaSuccess) return OCCRI_ECUDA;
  // (c)+(d): two round trips per unordered pair, dL/dpsi accumulated (and the omega
  // term of the kernel's derivative, for the erfc and erf kernels)
  if (cudaMemsetAsync(p->gpsi, 0, orb, s) != cudaSuccess) return OCCRI_ECUDA;
  const bool want_w = gomega && (p->kernel.kind == OCCRI_ERFC || p->kernel.kind == OCCRI_ERF);
  if (gomega && cudaMemsetAsync(p->dacc, 0, 2 * sizeof(double), s) != cudaSuccess)
    return OCCRI_ECUDA;
  for (int k = 0; k < p->nk; ++k)
    for (int kp0 = k; kp0 < p->nk;) {
      const int diag = (kp0 == k) ? 1 : 0;
      const int nkp = diag ? 1 : std::min(p->nkp_wave, p->nk - kp0);
      if (launch_vjp_wave<T>(*p, k, kp0, nkp, diag, want_w ? p->dacc : nullptr, s) != cudaSuccess)
        return OCCRI_ECUDA;
      kp0 += nkp;
    }
  // (b): dL/dC_{mu i} = sum_r conj(chi_mu) dL/dpsi_i; the transforms carry N_g/(4 pi)
  // and g carried N_k N_g/Omega, hence the factor 4 pi Omega/(N_k N_g^2)
  if (launch_phase_fields<T>(*p, p->gpsi, +1, s) != cudaSuccess) return OCCRI_ECUDA;
  if (cudaMemsetAsync(p->gacc, 0, nkc * sizeof(double2), s) != cudaSuccess) return OCCRI_ECUDA;
  const double ngd = (double)p->ng;
  const double scale = 4.0 * kPiD * p->omega_cell / ((double)p->nk * ngd * ngd);
  if (launch_contract_field<T>(*p, p->gpsi, p->gacc, scale, s) != cudaSuccess) return OCCRI_ECUDA;
  add_kernel<<<4 * 152, 256, 0, s>>>(p->gcf, p->gacc, gC, (long long)nkc);
  // dL/d omega = Re <dL/dKC, dKC/d omega>: the same units as the gradient of C
  if (gomega) domega_finish_kernel<<<1, 32, 0, s>>>(p->dacc, scale, gomega);
  return cudaGetLastError() == cudaSuccess ? OCCRI_OK : OCCRI_ECUDA;
}

}  // namespace

// A batch of cells built by one graph launch (see occri_batch_create in occri.h).
struct occri_batch {
  int device = 0;                          // the plans' device
  std::vector<occri_plan*> plans;
  cudaStream_t stream = nullptr;           // launch stream (the caller's)
  cudaStream_t cap = nullptr;              // capture origin
  std::vector<cudaStream_t> branch;        // one capture branch per cell
  cudaEvent_t ev_start = nullptr;
  std::vector<cudaEvent_t> ev_end;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the buffers the graph was captured with
  std::vector<const void*> c;
  std::vector<void*> kc, k;
  std::vector<double*> ex;
};

namespace occri_impl {

void batch_release_graph(occri_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void batch_free(occri_batch* b) {
  if (!b) return;
  batch_release_graph(b);
  for (cudaEvent_t e : b->ev_end)
    if (e) cudaEventDestroy(e);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  for (cudaStream_t st : b->branch)
    if (st) cudaStreamDestroy(st);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// Capture one build of every cell into b->graph: the capture starts on b->cap, forks one
// branch per cell (each plan's own two-stream pipeline joins back into its branch), and
// joins all branches on b->cap. Plans run their normal build code with their stream set
// to the branch and timing off.
int batch_capture(occri_batch* b) {
  batch_release_graph(b);
  const size_t n = b->plans.size();
  std::vector<cudaStream_t> saved_stream(n);
  std::vector<int> saved_timing(n);
  for (size_t i = 0; i < n; ++i) {
    Plan* p = b->plans[i]->p;
    saved_stream[i] = p->stream;
    saved_timing[i] = p->timing_every;
    p->timing_every = 0;
  }
  int st = OCCRI_OK;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    st = OCCRI_ECUDA;
  } else {
    if (cudaEventRecord(b->ev_start, b->cap) != cudaSuccess) st = OCCRI_ECUDA;
    for (size_t i = 0; i < n && st == OCCRI_OK; ++i) {
      Plan* p = b->plans[i]->p;
      if (cudaStreamWaitEvent(b->branch[i], b->ev_start, 0) != cudaSuccess) {
        st = OCCRI_ECUDA;
        break;
      }
      p->stream = b->branch[i];
      const double2* C = (const double2*)b->c[i];
      st = p->precision == OCCRI_FP64 ? build_impl<double>(p, C, b->kc[i], b->k[i], b->ex[i])
                                      : build_impl<float>(p, C, b->kc[i], b->k[i], b->ex[i]);
      if (st == OCCRI_OK && (cudaEventRecord(b->ev_end[i], b->branch[i]) != cudaSuccess ||
                             cudaStreamWaitEvent(b->cap, b->ev_end[i], 0) != cudaSuccess))
        st = OCCRI_ECUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st == OCCRI_OK && (e != cudaSuccess || !g)) st = OCCRI_ECUDA;
    if (st == OCCRI_OK) {
      b->graph = g;
      if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = OCCRI_ECUDA;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  for (size_t i = 0; i < n; ++i) {
    Plan* p = b->plans[i]->p;
    p->stream = saved_stream[i];
    p->timing_every = saved_timing[i];
  }
  if (st != OCCRI_OK) {
    cudaGetLastError();
    batch_release_graph(b);
  }
  return st;
}

// ---------------------------------------------------------------- autotuner
// Launch configurations of the pair loop, timed on the plan's own buffers and cached per
// (device, grid edge, nocc, precision, N_k, scratch capacity) for the life of the process.
struct TuneCfg {
  int nkp, nstreams, b_div, split_cd;
};

std::mutex g_tune_mu;
std::vector<std::pair<std::vector<long long>, occri_tune_t>> g_tune_cache;

std::vector<long long> tune_key(const Plan* p) {
  return {p->device, p->N[0], p->nocc, p->precision, p->nk, p->nkp_cap};
}

// The third stream, its scratch and events, made on first use.
int ensure_third_stream(Plan* p) {
  if (p->scratch3) return OCCRI_OK;
  cudaError_t e = occri::device_malloc(&p->scratch3, p->scratch_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_iso3, cudaEventDisableTiming);
  if (e == cudaSuccess) return OCCRI_OK;
  cudaGetLastError();
  if (p->scratch3) cudaFree(p->scratch3);
  for (void* yx : p->Yx)
    if (yx) cudaFree(yx);
  if (p->aux2) cudaStreamDestroy(p->aux2);
  if (p->ev_join2) cudaEventDestroy(p->ev_join2);
  if (p->ev_iso3) cudaEventDestroy(p->ev_iso3);
  p->scratch3 = nullptr;
  p->aux2 = nullptr;
  p->ev_join2 = p->ev_iso3 = nullptr;
  return e == cudaErrorMemoryAllocation ? OCCRI_ENOMEM : OCCRI_ECUDA;
}

int apply_tune(Plan* p, const occri_tune_t& t) {
  if (t.streams == 3) {
    const int st = ensure_third_stream(p);
    if (st != OCCRI_OK) return st;
  }
  p->nkp_wave = std::max(1, std::min(t.k_per_wave, p->nkp_cap));
  p->nstreams = std::max(1, std::min(t.streams, 3));
  p->b_div = std::max(1, t.pass_b_div);
  p->split_cd = t.split_cd ? 1 : 0;
  p->tuned = 1;
  return OCCRI_OK;   // wave_tables is set by occri_plan_set_tuning only
}

bool tune_lookup(Plan* p, occri_tune_t* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const auto key = tune_key(p);
  for (const auto& e : g_tune_cache)
    if (e.first == key) {
      if (out) *out = e.second;
      return true;
    }
  return false;
}

// Microseconds per pair field of `reps` consecutive waves of the build's loop (the waves of
// k = 0 with k' = 1, 2, ... wrapped over the mesh; diagonal waves where N_k = 1), under cfg.
template <typename T>
int tune_time(Plan* p, const TuneCfg& cfg, int reps, double* us_per_field) {
  const TuneCfg keep{p->nkp_wave, p->nstreams, p->b_div, p->split_cd};
  p->nkp_wave = cfg.nkp;
  p->nstreams = cfg.nstreams;
  p->b_div = cfg.b_div;
  p->split_cd = cfg.split_cd;
  cudaStream_t s = p->stream;
  cudaStream_t st[3] = {s, p->aux, p->aux2};
  void* sc[3] = {p->scratch, p->scratch2, p->scratch3};
  cudaEvent_t join[3] = {nullptr, p->ev_join, p->ev_join2};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = OCCRI_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = OCCRI_ECUDA;
  double fields = 0.0;
  if (rc == OCCRI_OK) {
    bool ok = cudaEventRecord(e0, s) == cudaSuccess && cudaEventRecord(p->ev_fork, s) == cudaSuccess;
    for (int o = 1; o < cfg.nstreams && ok; ++o)
      ok = cudaStreamWaitEvent(st[o], p->ev_fork, 0) == cudaSuccess;
    ok = ok && cudaEventRecord(p->ev_y, s) == cudaSuccess;
    int kp0 = p->nk > 1 ? 1 : 0;
    for (int w = 0; w < reps && ok; ++w) {
      const int diag = p->nk > 1 ? 0 : 1;
      const int nkp = diag ? 1 : std::min(cfg.nkp, p->nk - kp0);
      const int sw = w % cfg.nstreams;
      const bool split_y = p->Yx[0] && p->Yx[1];
      void* ya = split_y && sw > 0 ? p->Yx[sw - 1] : p->Y;
      ok = occri::launch_pair_wave<T>(*p, 0, kp0, nkp, diag, st[sw], sc[sw], ya, nullptr,
                                      split_y ? nullptr : p->ev_y) == cudaSuccess;
      fields += (double)occri::wave_fields(p->nocc, nkp, diag);
      if (!diag) {
        kp0 += nkp;
        if (kp0 >= p->nk) kp0 = 1;
      }
    }
    for (int o = 1; o < cfg.nstreams && ok; ++o)
      ok = cudaEventRecord(join[o], st[o]) == cudaSuccess &&
           cudaStreamWaitEvent(s, join[o], 0) == cudaSuccess;
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess;
    float ms = 0.f;
    ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      rc = OCCRI_ECUDA;
    } else {
      *us_per_field = 1e3 * (double)ms / std::max(1.0, fields);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  p->nkp_wave = keep.nkp;
  p->nstreams = keep.nstreams;
  p->b_div = keep.b_div;
  p->split_cd = keep.split_cd;
  return rc;
}

template <typename T>
int autotune(Plan* p, occri_tune_t* out) {
  std::vector<int> nkps;
  for (int v = 1; v < p->nkp_cap; v *= 2) nkps.push_back(v);
  nkps.push_back(p->nkp_cap);
  const bool can_fuse = occri::pair_wave_launches<T>(p->nocc, 0) == 3;
  const bool has_third = ensure_third_stream(p) == OCCRI_OK;   // else two streams at most
  // enough waves for every candidate to cover the same fields (and both streams)
  const int reps = std::max(12, 2 * p->nkp_cap);
  const TuneCfg def{p->nkp_cap, 3, 1, 0};
  double t_def = 0.0, best = 0.0;
  TuneCfg pick = def;
  int count = 0;
  for (int nkp : nkps)
    for (int ns = 1; ns <= (has_third ? 3 : 2); ++ns)
      for (int bd = 1; bd <= 2; ++bd)
        for (int sp = 0; sp <= (can_fuse ? 1 : 0); ++sp) {
          const TuneCfg c{nkp, ns, bd, sp};
          const int r = std::max(1, reps * p->nkp_cap / nkp);   // equal fields per candidate
          double us = 0.0;
          int st = tune_time<T>(p, c, 1, &us);   // warm-up (attributes, caches)
          if (st == OCCRI_OK) st = tune_time<T>(p, c, r, &us);
          if (st != OCCRI_OK) return st;
          ++count;
          const bool is_def = c.nkp == def.nkp && c.nstreams == def.nstreams &&
                              c.b_div == def.b_div && c.split_cd == def.split_cd;
          if (is_def) t_def = us;
          if (count == 1 || us < best) {
            best = us;
            pick = c;
          }
        }
  // the build leaves Y to be overwritten; the timed waves only touched scratch and Y
  occri_tune_t t{};
  t.k_per_wave = pick.nkp;
  t.streams = pick.nstreams;
  t.pass_b_div = pick.b_div;
  t.split_cd = pick.split_cd;
  t.wave_tables = (p->wave_tables || !p->vq) ? 1 : 0;
  t.us_per_field = best;
  t.us_default = t_def;
  t.candidates = count;
  const int st = apply_tune(p, t);
  if (st != OCCRI_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto key = tune_key(p);
    bool found = false;
    for (auto& e : g_tune_cache)
      if (e.first == key) {
        e.second = t;
        found = true;
      }
    if (!found) g_tune_cache.emplace_back(key, t);
  }
  if (out) *out = t;
  return OCCRI_OK;
}

}  // namespace occri_impl

extern "C" {

const char* occri_status_string(int status) {
  switch (status) {
    case OCCRI_OK: return "ok";
    case OCCRI_EINVAL: return "invalid argument";
    case OCCRI_ENOMEM: return "device allocation failed";
    case OCCRI_ENOTPD: return "-C^H K C is not positive definite";
    case OCCRI_ECUDA: return "CUDA runtime error";
    case OCCRI_ETIMEOUT: return "bounded device wait timed out";
    case OCCRI_EUNSUPPORTED: return "unsupported by this build";
    default: return "unknown status";
  }
}

int occri_plan_create(occri_plan** out, const occri_cell* cell, const occri_kmesh* kmesh,
                      const occri_basis* basis, int nocc, const int grid[3],
                      const occri_kernel* kernel, int precision, void* cuda_stream) {
  using namespace occri;
  if (!out) return OCCRI_EINVAL;
  *out = nullptr;
  if (!cell || !kmesh || !basis || !grid || !kernel) return OCCRI_EINVAL;
  if (cell->natm < 1 || !cell->xyz) return OCCRI_EINVAL;
  if (kmesh->nk < 1 || !kmesh->kfrac) return OCCRI_EINVAL;
  if (basis->nshell < 1 || !basis->atom || !basis->l || !basis->alpha) return OCCRI_EINVAL;
  if (precision != OCCRI_FP64 && precision != OCCRI_MIXED && precision != OCCRI_MIXED_TC)
    return OCCRI_EINVAL;
  if (kernel->kind < 0 || kernel->kind > 4) return OCCRI_EINVAL;
  if ((kernel->kind == OCCRI_ERFC || kernel->kind == OCCRI_ERF ||
       kernel->kind == OCCRI_ERF_TRUNC) && !(kernel->omega > 0.0))
    return OCCRI_EINVAL;
  if (kernel->g0_mode < 0 || kernel->g0_mode > 2) return OCCRI_EINVAL;
  if (kernel->g0_mode == 1 && kernel->kind != OCCRI_ERFC && kernel->kind != OCCRI_COULOMB_TRUNC &&
      kernel->kind != OCCRI_ERF_TRUNC)
    return OCCRI_EINVAL;
  if (kernel->g0_mode == 2 && kernel->kind != OCCRI_COULOMB && kernel->kind != OCCRI_ERF)
    return OCCRI_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (grid[d] < 4 || grid[d] > 64 || !smooth235(grid[d])) return OCCRI_EINVAL;
  int nao = 0;
  for (int s = 0; s < basis->nshell; ++s) {
    if (basis->l[s] < 0 || basis->l[s] > 3) return OCCRI_EINVAL;
    if (basis->atom[s] < 0 || basis->atom[s] >= cell->natm) return OCCRI_EINVAL;
    if (!(basis->alpha[s] > 0.0) || !std::isfinite(basis->alpha[s])) return OCCRI_EINVAL;
    if (s > 0 && basis->atom[s] < basis->atom[s - 1]) return OCCRI_EINVAL;  // atom-major order
    nao += 2 * basis->l[s] + 1;
  }
  if (nocc < 1 || nocc > nao) return OCCRI_EINVAL;
  double lat[3][3], inv[3][3];
  std::memcpy(lat, cell->a, sizeof(lat));
  const double det = lat[0][0] * (lat[1][1] * lat[2][2] - lat[1][2] * lat[2][1]) -
                     lat[0][1] * (lat[1][0] * lat[2][2] - lat[1][2] * lat[2][0]) +
                     lat[0][2] * (lat[1][0] * lat[2][1] - lat[1][1] * lat[2][0]);
  if (!(std::fabs(det) > 1e-8) || !std::isfinite(det)) return OCCRI_EINVAL;
  if (grid[0] != grid[1] || grid[0] != grid[2]) return OCCRI_EUNSUPPORTED;
  if (nocc > 32) return OCCRI_EUNSUPPORTED;   // assembly keeps C^H KC in shared memory
  if (!grid_edge_supported(grid[0])) return OCCRI_EUNSUPPORTED;
  inv3(lat, inv);

  Plan* p = new (std::nothrow) Plan();
  if (!p) return OCCRI_ENOMEM;
  p->nk = kmesh->nk; p->nao = nao; p->nocc = nocc; p->natm = cell->natm;
  p->nshell = basis->nshell; p->precision = precision;
  for (int d = 0; d < 3; ++d) p->N[d] = grid[d];
  p->ng = (long long)grid[0] * grid[1] * grid[2];
  std::memcpy(p->lat, lat, sizeof(lat));
  p->omega_cell = std::fabs(det);
  p->kernel = *kernel;
  p->stream = (cudaStream_t)cuda_stream;

  // k-points as rationals K/D per axis (D <= 64)
  p->kint_h.assign((size_t)p->nk * 3, 0);
  for (int d = 0; d < 3; ++d) {
    int found = 0;
    for (int D = 1; D <= 64 && !found; ++D) {
      bool okd = true;
      for (int k = 0; k < p->nk && okd; ++k) {
        const double v = kmesh->kfrac[k * 3 + d] * D;
        if (std::fabs(v - std::nearbyint(v)) > 1e-9) okd = false;
      }
      if (okd) found = D;
    }
    if (!found) { delete p; return OCCRI_EUNSUPPORTED; }
    p->D[d] = found;
    for (int k = 0; k < p->nk; ++k) {
      long long v = std::llround(kmesh->kfrac[k * 3 + d] * found);
      v %= found;
      if (v < 0) v += found;
      p->kint_h[k * 3 + d] = (int)v;
    }
  }
  const int Dc = p->D[0] * p->D[1] * p->D[2];

  // the G+q = 0 value (Eq. VGao's chi) and the truncation radius, from the k-mesh's
  // supercell D_1 a_1 x D_2 a_2 x D_3 a_3
  {
    double sc[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) sc[i][j] = lat[i][j] * p->D[i];
    const double vsc = std::fabs(det) * Dc;
    p->rc = std::cbrt(3.0 * vsc / (4.0 * kPiD));
    const double w = kernel->omega;
    double g0 = 0.0, dg0 = 0.0;
    if (kernel->g0_mode == 1 && kernel->kind == OCCRI_ERFC) {
      g0 = kPiD / (w * w);
      dg0 = -2.0 * kPiD / (w * w * w);
    } else if (kernel->g0_mode == 1 && kernel->kind == OCCRI_COULOMB_TRUNC) {
      g0 = 2.0 * kPiD * p->rc * p->rc;
    } else if (kernel->g0_mode == 1 && kernel->kind == OCCRI_ERF_TRUNC) {
      // 4 pi int_0^R_c erf(omega r) r dr
      const double R = p->rc;
      g0 = 4.0 * kPiD * ((R * R / 2.0 - 1.0 / (4.0 * w * w)) * std::erf(w * R) +
                         R * std::exp(-w * w * R * R) / (2.0 * w * std::sqrt(kPiD)));
    } else if (kernel->g0_mode == 2 && kernel->kind == OCCRI_COULOMB) {
      g0 = -vsc * madelung_potential(sc);
    } else if (kernel->g0_mode == 2 && kernel->kind == OCCRI_ERF) {
      g0 = erf_lattice_chi(sc, w, &dg0);
    }
    p->g0_4pi = g0 / (4.0 * kPiD);
    p->dg0_4pi = dg0 / (4.0 * kPiD);
    if (kernel->kind == OCCRI_ERF_TRUNC) {
      faddeeva_coefficients(p->fad_a, &p->fad_L);
      p->lr_erf = std::erf(w * p->rc);
      p->lr_exp = std::exp(-w * w * p->rc * p->rc);
    }
  }

  // shells, cutoffs, AO offsets
  const double eps = (precision == OCCRI_FP64) ? 1e-16 : 1e-11;
  std::vector<ShellDev> sh(p->nshell);
  std::vector<double> rcut(p->nshell);
  double rcut_max = 0.0;
  int ao = 0;
  for (int s = 0; s < p->nshell; ++s) {
    ShellDev& x = sh[s];
    std::memset(&x, 0, sizeof(x));
    x.l = basis->l[s];
    x.atom = basis->atom[s];
    x.ao = ao;
    x.alpha = basis->alpha[s];
    x.alpha_f = (float)x.alpha;
    x.alpha_lo = (float)(x.alpha - (double)x.alpha_f);
    // Tight primitives reach one or two images per point, so FP32 rounding of
    // r^2 and alpha r^2 does not average out there; they get a double-float exponent.
    x.exact_arg = (precision != OCCRI_FP64 && x.alpha >= 0.5) ? 1 : 0;
    shell_norms(x.l, x.alpha, x.norm);
    for (int m = 0; m < 2 * x.l + 1; ++m) x.norm_f[m] = (float)x.norm[m];
    rcut[s] = shell_cutoff(x.l, x.alpha, eps);
    x.rcut2 = rcut[s] * rcut[s];
    x.rcut2_f = (float)x.rcut2;
    rcut_max = std::max(rcut_max, rcut[s]);
    ao += 2 * x.l + 1;
    p->shells_by_l[x.l].push_back(s);
  }
  std::vector<double> ao_norm(nao);
  for (int s = 0; s < p->nshell; ++s)
    for (int m = 0; m < 2 * sh[s].l + 1; ++m) ao_norm[sh[s].ao + m] = sh[s].norm[m];
  std::vector<int> atom_shell0(p->natm + 1, 0);
  for (int a = 0, s = 0; a <= p->natm; ++a) {
    while (s < p->nshell && basis->atom[s] < a) ++s;
    atom_shell0[a] = s;
  }

  // Point blocks of 2 x 4 x 4 grid points (one warp each, ragged at the edges). Every
  // point of a block shares the block's T0, the lattice vector that brings the block
  // centre minus A into the Wigner-Seitz cell; d0 = r - A - T0 per (atom, point).
  const long long ng = p->ng;
  const int BD[3] = {2, 4, 4};
  for (int d = 0; d < 3; ++d) p->nb[d] = (grid[d] + BD[d] - 1) / BD[d];
  const int nblk = p->nb[0] * p->nb[1] * p->nb[2];
  p->nblk = nblk;
  std::vector<double> d0((size_t)p->natm * 3 * ng);
  std::vector<int> t0((size_t)p->natm * nblk);
  std::vector<double> bcen((size_t)p->natm * nblk * 3);  // block centre - A - T0
  std::vector<double> brad(nblk, 0.0);                     // max |r - centre| in the block
  double rbound = 0.0;
  for (int a = 0; a < p->natm; ++a) {
    const double* A = cell->xyz + 3 * a;
    double af[3];
    for (int d = 0; d < 3; ++d) af[d] = A[0] * inv[0][d] + A[1] * inv[1][d] + A[2] * inv[2][d];
    for (int b1 = 0; b1 < p->nb[0]; ++b1)
      for (int b2 = 0; b2 < p->nb[1]; ++b2)
        for (int b3 = 0; b3 < p->nb[2]; ++b3) {
          const int blk = (b1 * p->nb[1] + b2) * p->nb[2] + b3;
          const int lo[3] = {BD[0] * b1, BD[1] * b2, BD[2] * b3};
          int hi[3];
          for (int d = 0; d < 3; ++d) hi[d] = std::min(lo[d] + BD[d], grid[d]) - 1;
          double fc[3];
          for (int d = 0; d < 3; ++d) fc[d] = 0.5 * (lo[d] + hi[d]) / grid[d] - af[d];
          int base[3];
          for (int d = 0; d < 3; ++d) base[d] = (int)std::floor(fc[d] + 0.5);
          double best = 1e300;
          int bt[3] = {base[0], base[1], base[2]};
          double bc[3] = {0, 0, 0};
          for (int e0 = -1; e0 <= 1; ++e0)
            for (int e1 = -1; e1 <= 1; ++e1)
              for (int e2 = -1; e2 <= 1; ++e2) {
                const int t[3] = {base[0] + e0, base[1] + e1, base[2] + e2};
                const double g[3] = {fc[0] - t[0], fc[1] - t[1], fc[2] - t[2]};
                double c[3];
                for (int d = 0; d < 3; ++d) c[d] = g[0] * lat[0][d] + g[1] * lat[1][d] + g[2] * lat[2][d];
                const double r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                if (r2 < best) {
                  best = r2;
                  for (int d = 0; d < 3; ++d) { bt[d] = t[d]; bc[d] = c[d]; }
                }
              }
          t0[(size_t)a * nblk + blk] = dev::pack_t0(bt[0], bt[1], bt[2]);
          for (int d = 0; d < 3; ++d) bcen[((size_t)a * nblk + blk) * 3 + d] = bc[d];
          for (int n1 = lo[0]; n1 <= hi[0]; ++n1)
            for (int n2 = lo[1]; n2 <= hi[1]; ++n2)
              for (int n3 = lo[2]; n3 <= hi[2]; ++n3) {
                const long long n = ((long long)n1 * grid[1] + n2) * grid[2] + n3;
                const double f[3] = {(double)n1 / grid[0] - af[0] - bt[0],
                                     (double)n2 / grid[1] - af[1] - bt[1],
                                     (double)n3 / grid[2] - af[2] - bt[2]};
                double c[3];
                for (int d = 0; d < 3; ++d) c[d] = f[0] * lat[0][d] + f[1] * lat[1][d] + f[2] * lat[2][d];
                for (int d = 0; d < 3; ++d) d0[((size_t)a * 3 + d) * ng + n] = c[d];
                rbound = std::max(rbound, std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]));
                const double e[3] = {c[0] - bc[0], c[1] - bc[1], c[2] - bc[2]};
                brad[blk] = std::max(brad[blk], std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]));
              }
        }
  }
  rbound += 1e-9;

  // master image list T' sorted by length, |T'| <= rcut_max + rbound
  const double rimg = rcut_max + rbound;
  int nb[3];
  for (int d = 0; d < 3; ++d) {
    const double bn = std::sqrt(inv[0][d] * inv[0][d] + inv[1][d] * inv[1][d] + inv[2][d] * inv[2][d]);
    nb[d] = (int)std::ceil(rimg * bn) + 1;
  }
  struct Img { double len, x, y, z; int n[3]; };
  std::vector<Img> imgs;
  for (int i = -nb[0]; i <= nb[0]; ++i)
    for (int j = -nb[1]; j <= nb[1]; ++j)
      for (int k = -nb[2]; k <= nb[2]; ++k) {
        Img m;
        m.x = i * lat[0][0] + j * lat[1][0] + k * lat[2][0];
        m.y = i * lat[0][1] + j * lat[1][1] + k * lat[2][1];
        m.z = i * lat[0][2] + j * lat[1][2] + k * lat[2][2];
        m.len = std::sqrt(m.x * m.x + m.y * m.y + m.z * m.z);
        m.n[0] = i; m.n[1] = j; m.n[2] = k;
        if (m.len <= rimg) imgs.push_back(m);
      }
  std::sort(imgs.begin(), imgs.end(), [](const Img& a, const Img& b) { return a.len < b.len; });
  const int nimg = (int)imgs.size();
  p->nimg = nimg;
  for (int s = 0; s < p->nshell; ++s) {
    const double lim = rcut[s] + rbound;
    int c = 0;
    while (c < nimg && imgs[c].len <= lim) ++c;
    sh[s].nimg = c;
  }
  // per (atom, block): master images sorted by distance from the block centre, and
  // per shell the prefix within the shell's radius plus the block radius
  int nsa = 0;
  for (int a = 0; a < p->natm; ++a) nsa = std::max(nsa, atom_shell0[a + 1] - atom_shell0[a]);
  p->nsa = nsa;
  std::vector<std::vector<unsigned short>> lists((size_t)p->natm * nblk);
  std::vector<unsigned short> bpre((size_t)p->natm * nblk * std::max(nsa, 1), 0);
  int lmax = 1;
  {
    std::vector<std::pair<double, int>> cand;
    for (int a = 0; a < p->natm; ++a) {
      double rmax_a = 0.0;
      for (int s2 = atom_shell0[a]; s2 < atom_shell0[a + 1]; ++s2) rmax_a = std::max(rmax_a, rcut[s2]);
      for (int blk = 0; blk < nblk; ++blk) {
        const double* c = &bcen[((size_t)a * nblk + blk) * 3];
        const double reach = rmax_a + brad[blk] + 1e-9;
        cand.clear();
        for (int j = 0; j < nimg; ++j) {
          const double e[3] = {c[0] - imgs[j].x, c[1] - imgs[j].y, c[2] - imgs[j].z};
          const double dist = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
          if (dist <= reach) cand.push_back({dist, j});
        }
        std::sort(cand.begin(), cand.end());
        auto& L = lists[(size_t)a * nblk + blk];
        L.resize(cand.size());
        for (size_t u = 0; u < cand.size(); ++u) L[u] = (unsigned short)cand[u].second;
        for (int s2 = atom_shell0[a]; s2 < atom_shell0[a + 1]; ++s2) {
          const double lim = rcut[s2] + brad[blk] + 1e-9;
          int cnt = 0;
          while (cnt < (int)cand.size() && cand[cnt].first <= lim) ++cnt;
          bpre[((size_t)a * nblk + blk) * nsa + (s2 - atom_shell0[a])] = (unsigned short)cnt;
        }
        lmax = std::max(lmax, (int)cand.size());
      }
    }
  }
  p->lmax = lmax;
  std::vector<unsigned short> blist((size_t)p->natm * nblk * lmax, 0);
  for (size_t q = 0; q < lists.size(); ++q)
    std::copy(lists[q].begin(), lists[q].end(), blist.begin() + q * lmax);
  if (nimg >= 65536) { delete p; return OCCRI_EUNSUPPORTED; }
  std::vector<double> img_d((size_t)3 * nimg);
  std::vector<float> img_hi((size_t)3 * nimg), img_lo((size_t)3 * nimg);
  for (int j = 0; j < nimg; ++j) {
    const double v[3] = {imgs[j].x, imgs[j].y, imgs[j].z};
    for (int d = 0; d < 3; ++d) {
      img_d[(size_t)d * nimg + j] = v[d];
      img_hi[(size_t)d * nimg + j] = (float)v[d];
      img_lo[(size_t)d * nimg + j] = (float)(v[d] - (double)(float)v[d]);
    }
  }
  // e^{i k.T'} with exact integer reduction of the phase
  std::vector<double2> ph_d;
  std::vector<float2> ph_f;
  const int nk_pad = (p->nk + kPhasePadK - 1) / kPhasePadK * kPhasePadK;   // zero rows past nk
  if (precision == OCCRI_FP64) ph_d.assign((size_t)nk_pad * nimg, make_double2(0.0, 0.0));
  else ph_f.assign((size_t)nk_pad * nimg, make_float2(0.f, 0.f));
  for (int k = 0; k < p->nk; ++k)
    for (int j = 0; j < nimg; ++j) {
      long long num = 0;
      for (int d = 0; d < 3; ++d)
        num += (long long)p->kint_h[k * 3 + d] * imgs[j].n[d] * (Dc / p->D[d]);
      num %= Dc;
      if (num < 0) num += Dc;
      const double ang = 2.0 * kPiD * (double)num / (double)Dc;
      if (precision == OCCRI_FP64) ph_d[(size_t)k * nimg + j] = make_double2(std::cos(ang), std::sin(ang));
      else ph_f[(size_t)k * nimg + j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }

  // device tables and workspaces, on the current device
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return OCCRI_ECUDA;
  }
  size_t tot = 0;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess && x != cudaSuccess) e = x; };
  chk(upload(&p->shells, sh, &tot));
  chk(upload(&p->atom_shell0, atom_shell0, &tot));
  for (int l = 0; l < 4; ++l) chk(upload(&p->shell_list_l[l], p->shells_by_l[l], &tot));
  chk(upload(&p->kint, p->kint_h, &tot));
  chk(upload(&p->ao_norm, ao_norm, &tot));
  {
    unsigned char* b = nullptr;
    const size_t csb = (precision == OCCRI_FP64 ? sizeof(double2) : sizeof(float4)) *
                       (size_t)p->nk * nao * nocc;
    chk(dalloc(&b, csb, &tot));
    p->cs = b;
  }
  chk(upload(&p->t0, t0, &tot));
  chk(upload(&p->blist, blist, &tot));
  chk(upload(&p->bpre, bpre, &tot));
  if (precision == OCCRI_FP64) {
    chk(upload(&p->img_d, img_d, &tot));
    chk(upload(&p->d0_d, d0, &tot));
    double2* ph = nullptr;
    chk(upload(&ph, ph_d, &tot));
    p->img_phase = ph;
  } else {
    chk(upload(&p->img_hi, img_hi, &tot));
    chk(upload(&p->img_lo, img_lo, &tot));
    std::vector<float> hi(d0.size()), lo(d0.size());
    for (size_t i = 0; i < d0.size(); ++i) {
      hi[i] = (float)d0[i];
      lo[i] = (float)(d0[i] - (double)hi[i]);
    }
    chk(upload(&p->d0_hi, hi, &tot));
    chk(upload(&p->d0_lo, lo, &tot));
    float2* ph = nullptr;
    chk(upload(&ph, ph_f, &tot));
    p->img_phase = ph;
  }
  const size_t csz = (precision == OCCRI_FP64) ? sizeof(double2) : sizeof(float2);
  p->fs = (ng + 63) / 64 * 64;
  const size_t field_bytes = csz * (size_t)p->fs;
  const size_t per_kp = field_bytes * (size_t)nocc * nocc;
  const size_t budget = (size_t)kWaveBudgetMB << 20;
  int nkp = (int)std::max<size_t>(1, budget / per_kp);
  nkp = std::min(nkp, p->nk);
  nkp = std::max(1, std::min(nkp, 65535 / (nocc * nocc)));   // grid.y limit of the passes
  p->nkp_wave = nkp;
  p->nkp_cap = nkp;
  p->fields_cap = nkp * nocc * nocc;
  const size_t orb = (size_t)p->nk * nocc * p->fs;
  {
    unsigned char* b = nullptr;
    chk(dalloc(&b, orb * csz, &tot)); p->psi = b; b = nullptr;
    chk(dalloc(&b, orb * csz, &tot)); p->Y = b; b = nullptr;
    // the second and third streams' private accumulators, where they cost at most 16 GiB
    if (2 * orb * csz <= ((size_t)16 << 30)) {
      chk(dalloc(&b, orb * csz, &tot)); p->Yx[0] = b; b = nullptr;
      chk(dalloc(&b, orb * csz, &tot)); p->Yx[1] = b; b = nullptr;
    }
    // behind each scratch buffer, the kernel tables v/(4 pi) of one wave (one per k')
    const size_t sbytes = (size_t)p->fields_cap * field_bytes + (size_t)nkp * ng * (csz / 2);
    p->scratch_bytes = sbytes;
    chk(dalloc(&b, sbytes, &tot)); p->scratch = b; b = nullptr;
    chk(dalloc(&b, sbytes, &tot)); p->scratch2 = b; b = nullptr;
    // three waves in flight by default: one more scratch buffer (a wave, ~110 MB at 60^3
    // FP32) measured 1.5 % faster builds at 6x6x6 k than two
    chk(dalloc(&b, sbytes, &tot)); p->scratch3 = b; b = nullptr;
    // the kernel tables of every k - k', where they fit: waves then form none of their own
    const size_t qbytes = (size_t)(2 * p->D[0] - 1) * (2 * p->D[1] - 1) * (2 * p->D[2] - 1) *
                          (size_t)ng * (csz / 2);
    if (qbytes <= kQTabMaxBytes) {
      chk(dalloc(&b, qbytes, &tot)); p->vq = b; b = nullptr;
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux2, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&p->ev_fork, &p->ev_join, &p->ev_y, &p->ev_iso, &p->ev_iso2,
                          &p->ev_join2, &p->ev_iso3})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  p->nstreams = 3;
  chk(dalloc(&p->kc, (size_t)p->nk * nao * nocc, &tot));
  chk(dalloc(&p->xi, (size_t)p->nk * nao * nocc, &tot));
  chk(dalloc(&p->mmat, (size_t)p->nk * nocc * nocc, &tot));
  chk(dalloc(&p->ek, (size_t)p->nk, &tot));
  chk(dalloc(&p->dacc, 2, &tot));
  chk(dalloc(&p->status, 2, &tot));
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, 2 * sizeof(int));
  if (e == cudaSuccess && p->vq)
    e = precision == OCCRI_FP64 ? launch_qtables<double>(*p, p->stream)
                                : launch_qtables<float>(*p, p->stream);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? OCCRI_ENOMEM : OCCRI_ECUDA;
    cudaGetLastError();
    free_plan(p);
    return code;
  }
  if (precision == OCCRI_MIXED_TC) {
    const int st = tc_plan_create(p, sh, cell->xyz, rcut, &tot);
    if (st != OCCRI_OK) {
      free_plan(p);
      return st;
    }
  }
  p->workspace_bytes = tot;
  {
    occri_tune_t t{};
    if (occri_impl::tune_lookup(p, &t) && occri_impl::apply_tune(p, t) != OCCRI_OK)
      p->nstreams = 2;   // the cached choice needed memory that is not there: keep the default
  }
  occri_plan* h = new (std::nothrow) occri_plan;
  if (!h) { free_plan(p); return OCCRI_ENOMEM; }
  h->p = p;
  *out = h;
  return OCCRI_OK;
}

int occri_plan_destroy(occri_plan* plan) {
  if (!plan) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  occri::free_plan(plan->p);
  delete plan;
  return OCCRI_OK;
}

int occri_plan_info(const occri_plan* plan, occri_plan_info_t* info) {
  if (!plan || !info) return OCCRI_EINVAL;
  const Plan* p = plan->p;
  info->nk = p->nk; info->nao = p->nao; info->nocc = p->nocc; info->natm = p->natm;
  info->nshell = p->nshell;
  for (int d = 0; d < 3; ++d) info->grid[d] = p->N[d];
  info->ng = p->ng;
  info->precision = p->precision;
  info->workspace_bytes = p->workspace_bytes;
  info->fields_per_wave = p->nkp_wave * p->nocc * p->nocc;
  info->launches_per_build = p->launches_per_build;
  info->contraction_tc = p->tc ? 1 : 0;
  info->tc_stages = tc_plan_stages(p->tc);
  info->tc_flops_per_stage = p->tc ? occri::tc_flops_per_stage() : 0.0;
  return OCCRI_OK;
}

int occri_plan_set_timing(occri_plan* plan, int every) {
  if (!plan || every < -1) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  if (every == 0) {
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return OCCRI_ECUDA;
    p->ev_pending.clear();
    for (cudaEvent_t e : p->ev_used) p->ev_free.push_back(e);
    p->ev_used.clear();
  }
  p->timing_every = every;
  return OCCRI_OK;
}

int occri_plan_stage_times(occri_plan* plan, double* ms, long long* launches, double* units) {
  if (!plan || !ms || !launches || !units) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return OCCRI_ECUDA;
  for (const Plan::TimedSpan& sp : p->ev_pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, sp.a, sp.b) != cudaSuccess) return OCCRI_ECUDA;
    p->stage_ms[sp.stage] += t;
    p->stage_n[sp.stage] += 1;
    p->stage_units[sp.stage] += sp.units;
  }
  p->ev_pending.clear();
  for (cudaEvent_t e : p->ev_used) p->ev_free.push_back(e);
  p->ev_used.clear();
  for (int i = 0; i < OCCRI_NSTAGES; ++i) {
    ms[i] = p->stage_ms[i];
    launches[i] = p->stage_n[i];
    units[i] = p->stage_units[i];
    p->stage_ms[i] = 0.0;
    p->stage_n[i] = 0;
    p->stage_units[i] = 0.0;
  }
  return OCCRI_OK;
}

int occri_plan_set_stream(occri_plan* plan, void* cuda_stream) {
  if (!plan) return OCCRI_EINVAL;
  plan->p->stream = (cudaStream_t)cuda_stream;
  return OCCRI_OK;
}

int occri_plan_sync(occri_plan* plan, int* bad_k) {
  if (bad_k) *bad_k = -1;
  if (!plan) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return OCCRI_ECUDA;
  int st[2] = {0, -1};
  if (cudaMemcpy(st, p->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return OCCRI_ECUDA;
  if (st[0] != 0) {
    if (cudaMemset(p->status, 0, sizeof(st)) != cudaSuccess) return OCCRI_ECUDA;
    if (bad_k) *bad_k = st[1];
    return st[0];
  }
  return OCCRI_OK;
}


int occri_k_build(occri_plan* plan, const void* C_dev, void* KC_dev, void* K_dev, double* Ex_dev) {
  if (!plan || !C_dev) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  return p->precision == OCCRI_FP64
             ? occri_impl::build_impl<double>(p, (const double2*)C_dev, KC_dev, K_dev, Ex_dev)
             : occri_impl::build_impl<float>(p, (const double2*)C_dev, KC_dev, K_dev, Ex_dev);
}

int occri_plan_autotune(occri_plan* plan, int flags, occri_tune_t* chosen) {
  if (!plan || (flags & ~OCCRI_TUNE_FORCE)) return OCCRI_EINVAL;
  Plan* p = plan->p;
  occri::DeviceGuard guard(p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  occri_tune_t t{};
  if (!(flags & OCCRI_TUNE_FORCE) && occri_impl::tune_lookup(p, &t)) {
    const int st = occri_impl::apply_tune(p, t);
    if (st != OCCRI_OK) return st;
    t.candidates = 0;
    if (chosen) *chosen = t;
    return OCCRI_OK;
  }
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return OCCRI_ECUDA;
  }
  const int st = p->precision == OCCRI_FP64 ? occri_impl::autotune<double>(p, chosen)
                                            : occri_impl::autotune<float>(p, chosen);
  if (st != OCCRI_OK) return st;
  // timing may have left a device status (none is expected); report it like a build would
  return occri_plan_sync(plan, nullptr);
}

int occri_plan_set_tuning(occri_plan* plan, const occri_tune_t* cfg) {
  if (!plan || !cfg) return OCCRI_EINVAL;
  if (cfg->k_per_wave < 1 || cfg->streams < 1 || cfg->streams > 3 ||
      (cfg->pass_b_div != 1 && cfg->pass_b_div != 2) || (cfg->split_cd != 0 && cfg->split_cd != 1) ||
      (cfg->wave_tables != 0 && cfg->wave_tables != 1))
    return OCCRI_EINVAL;
  Plan* p = plan->p;
  occri::DeviceGuard guard(p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  const int st = occri_impl::apply_tune(p, *cfg);
  if (st != OCCRI_OK) return st;
  p->wave_tables = cfg->wave_tables ? 1 : 0;
  p->tuned = 0;
  return OCCRI_OK;
}

int occri_plan_tuning(const occri_plan* plan, occri_tune_t* current) {
  if (!plan || !current) return OCCRI_EINVAL;
  const Plan* p = plan->p;
  *current = occri_tune_t{};
  current->k_per_wave = p->nkp_wave;
  current->streams = p->nstreams;
  current->pass_b_div = p->b_div;
  current->split_cd = p->split_cd;
  current->wave_tables = (p->wave_tables || !p->vq) ? 1 : 0;
  current->candidates = p->tuned ? -1 : 0;
  return OCCRI_OK;
}

int occri_k_assemble_paper(occri_plan* plan, int ncol, const void* S_dev, const void* C_dev,
                           const void* KC_dev, void* K_dev) {
  if (!plan || !S_dev || !C_dev || !KC_dev || !K_dev) return OCCRI_EINVAL;
  Plan* p = plan->p;
  if (ncol < 1 || ncol > p->nao) return OCCRI_EINVAL;
  occri::DeviceGuard guard(p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  const cudaError_t e = occri::launch_assemble_paper(*p, ncol, (const double2*)S_dev,
                                                     (const double2*)C_dev, (const double2*)KC_dev,
                                                     (double2*)K_dev);
  if (e == cudaErrorMemoryAllocation) return OCCRI_ENOMEM;
  return e == cudaSuccess ? OCCRI_OK : OCCRI_ECUDA;
}

int occri_k_build_conduction(occri_plan* plan_all, occri_plan* plan_r, const void* C_all_dev,
                             void* KCr_dev) {
  if (!plan_all || !plan_r || !C_all_dev || !KCr_dev || plan_all == plan_r) return OCCRI_EINVAL;
  Plan* pa = plan_all->p;
  Plan* pr = plan_r->p;
  // the two plans must describe the same cell, k-mesh, basis, grid, kernel and precision
  bool same = pa->nk == pr->nk && pa->nao == pr->nao && pa->natm == pr->natm &&
              pa->nshell == pr->nshell && pa->precision == pr->precision &&
              pa->device == pr->device && pa->nocc > pr->nocc &&
              pa->kernel.kind == pr->kernel.kind && pa->kernel.omega == pr->kernel.omega &&
              pa->g0_4pi == pr->g0_4pi && pa->rc == pr->rc;
  for (int d = 0; d < 3; ++d) same = same && pa->N[d] == pr->N[d] && pa->D[d] == pr->D[d];
  for (int i = 0; i < 3 && same; ++i)
    for (int j = 0; j < 3; ++j) same = same && pa->lat[i][j] == pr->lat[i][j];
  same = same && pa->kint_h == pr->kint_h;
  if (!same) return OCCRI_EINVAL;
  occri::DeviceGuard guard(pa->device);
  if (!guard.ok) return OCCRI_ECUDA;
  const int nr = pr->nocc, nocc = pa->nocc - nr;
  const long long rows = (long long)pa->nk * pa->nao;
  void* buf = nullptr;
  const size_t b_all = sizeof(double2) * (size_t)rows * pa->nocc;
  const size_t b_r = sizeof(double2) * (size_t)rows * nr;
  if (occri::device_malloc(&buf, b_all + 2 * b_r) != cudaSuccess) {
    cudaGetLastError();
    return OCCRI_ENOMEM;
  }
  double2* kc_all = (double2*)buf;
  double2* c_r = (double2*)((unsigned char*)buf + b_all);
  double2* kc_r = (double2*)((unsigned char*)buf + b_all + b_r);
  int st = OCCRI_OK;
  // both builds run on plan_all's stream, one after the other
  cudaStream_t keep = pr->stream;
  pr->stream = pa->stream;
  if (occri::launch_gather_cols((const double2*)C_all_dev, c_r, rows, nocc, nr, pa->stream) !=
      cudaSuccess)
    st = OCCRI_ECUDA;
  if (st == OCCRI_OK) st = occri_k_build(plan_all, C_all_dev, kc_all, nullptr, nullptr);
  if (st == OCCRI_OK) st = occri_k_build(plan_r, c_r, kc_r, nullptr, nullptr);
  if (st == OCCRI_OK &&
      occri::launch_band_diff(kc_all, kc_r, (double2*)KCr_dev, rows, nocc, nr, pa->stream) !=
          cudaSuccess)
    st = OCCRI_ECUDA;
  if (cudaStreamSynchronize(pa->stream) != cudaSuccess && st == OCCRI_OK) st = OCCRI_ECUDA;
  pr->stream = keep;
  cudaFree(buf);
  if (st != OCCRI_OK) {
    cudaGetLastError();
    return st;
  }
  const int s1 = occri_plan_sync(plan_all, nullptr);
  const int s2 = occri_plan_sync(plan_r, nullptr);
  return s1 != OCCRI_OK ? s1 : s2;
}

int occri_k_build_once(const occri_cell* cell, const occri_kmesh* kmesh,
                       const occri_basis* basis, const void* C_dev, int nocc, const int grid[3],
                       const occri_kernel* kernel, int precision, void* K_dev, double* Ex_dev,
                       void* cuda_stream) {
  if (!C_dev) return OCCRI_EINVAL;
  occri_plan* plan = nullptr;
  int st = occri_plan_create(&plan, cell, kmesh, basis, nocc, grid, kernel, precision,
                             cuda_stream);
  if (st != OCCRI_OK) return st;
  st = occri_k_build(plan, C_dev, nullptr, K_dev, Ex_dev);
  const int st_sync = occri_plan_sync(plan, nullptr);
  occri_plan_destroy(plan);
  return st != OCCRI_OK ? st : st_sync;
}

int occri_plan_inject_fault(occri_plan* plan, int fault, double wait_limit_ms) {
  if (!plan) return OCCRI_EINVAL;
  if (fault != OCCRI_FAULT_NONE && fault != OCCRI_FAULT_WAIT) return OCCRI_EINVAL;
  if (!(wait_limit_ms > 0.0) || wait_limit_ms > 60000.0) return OCCRI_EINVAL;
  plan->p->fault = fault;
  plan->p->wait_ns = (long long)(wait_limit_ms * 1e6);
  return OCCRI_OK;
}

int occri_debug_fail_allocation(int nth) {
  occri::g_alloc_countdown.store(nth >= 1 ? (long long)(nth - 1) : -1LL);
  return OCCRI_OK;
}

int occri_k_build_host(occri_plan* plan, const void* C_host, void* KC_host, void* K_host,
                       double* Ex_host) {
  if (!plan || !C_host) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  const size_t nc = (size_t)p->nk * p->nao * p->nocc;
  const size_t nkk = (size_t)p->nk * p->nao * p->nao;
  if (!p->h_c) {
    if (occri::device_malloc((void**)&p->h_c, nc * sizeof(double2)) != cudaSuccess ||
        occri::device_malloc((void**)&p->h_kc, nc * sizeof(double2)) != cudaSuccess ||
        occri::device_malloc((void**)&p->h_ex, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      for (void** b : {(void**)&p->h_c, (void**)&p->h_kc, (void**)&p->h_ex}) {
        if (*b) cudaFree(*b);
        *b = nullptr;
      }
      return OCCRI_ENOMEM;
    }
  }
  if (K_host && !p->h_k) {
    if (occri::device_malloc((void**)&p->h_k, nkk * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      p->h_k = nullptr;
      return OCCRI_ENOMEM;
    }
  }
  cudaStream_t s = p->stream;
  if (cudaMemcpyAsync(p->h_c, C_host, nc * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return OCCRI_ECUDA;
  int st = occri_k_build(plan, p->h_c, KC_host ? p->h_kc : nullptr, K_host ? p->h_k : nullptr,
                         Ex_host ? p->h_ex : nullptr);
  if (st != OCCRI_OK) return st;
  if (KC_host && cudaMemcpyAsync(KC_host, p->h_kc, nc * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return OCCRI_ECUDA;
  if (K_host && cudaMemcpyAsync(K_host, p->h_k, nkk * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return OCCRI_ECUDA;
  if (Ex_host && cudaMemcpyAsync(Ex_host, p->h_ex, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return OCCRI_ECUDA;
  return occri_plan_sync(plan, nullptr);
}

int occri_orbitals(occri_plan* plan, const void* C_dev, void* psi_dev) {
  if (!plan || !C_dev || !psi_dev) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  cudaError_t e;
  if (p->precision == OCCRI_FP64) {
    e = occri::launch_scale_c<double>(*p, (const double2*)C_dev, p->stream);
    if (e == cudaSuccess) e = occri::launch_orbitals<double>(*p, p->stream);
    if (e == cudaSuccess) e = occri::launch_widen<double>(*p, psi_dev, p->stream);
  } else {
    e = occri::launch_scale_c<float>(*p, (const double2*)C_dev, p->stream);
    if (e == cudaSuccess) e = occri::launch_orbitals<float>(*p, p->stream);
    if (e == cudaSuccess) e = occri::launch_widen<float>(*p, psi_dev, p->stream);
  }
  return e == cudaSuccess ? OCCRI_OK : OCCRI_ECUDA;
}

int occri_vjp_full(occri_plan* plan, const void* C_dev, double gEx, const void* gKC_dev,
                   const void* gK_dev, void* gC_dev, double* gomega_dev) {
  if (!plan || !C_dev || !gC_dev) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  if (!p->have_kc) return OCCRI_EINVAL;
  if (gomega_dev && p->kernel.kind == OCCRI_ERF_TRUNC) return OCCRI_EUNSUPPORTED;
  const double2* C = (const double2*)C_dev;
  const double2* gKC = (const double2*)gKC_dev;
  const double2* gK = (const double2*)gK_dev;
  double2* gC = (double2*)gC_dev;
  return p->precision == OCCRI_FP64
             ? occri_impl::vjp_full_impl<double>(p, C, gEx, gKC, gK, gC, gomega_dev)
             : occri_impl::vjp_full_impl<float>(p, C, gEx, gKC, gK, gC, gomega_dev);
}

int occri_vjp(occri_plan* plan, const void* C_dev, double gEx, void* gC_dev, double* gomega_dev) {
  if (!plan || !C_dev) return OCCRI_EINVAL;
  occri::DeviceGuard guard(plan->p->device);
  if (!guard.ok) return OCCRI_ECUDA;
  Plan* p = plan->p;
  if (!p->have_kc) return OCCRI_EINVAL;
  if (gomega_dev && p->kernel.kind == OCCRI_ERF_TRUNC) return OCCRI_EUNSUPPORTED;
  const double2* C = (const double2*)C_dev;
  return p->precision == OCCRI_FP64 ? occri_impl::vjp_impl<double>(p, C, gEx, gC_dev, gomega_dev)
                                    : occri_impl::vjp_impl<float>(p, C, gEx, gC_dev, gomega_dev);
}

int occri_batch_create(occri_batch** out, occri_plan* const* plans, int nplans,
                       void* cuda_stream) {
  if (!out) return OCCRI_EINVAL;
  *out = nullptr;
  if (!plans || nplans < 1) return OCCRI_EINVAL;
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i]) return OCCRI_EINVAL;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return OCCRI_EINVAL;
  }
  const int dev = plans[0]->p->device;
  for (int i = 1; i < nplans; ++i)
    if (plans[i]->p->device != dev) return OCCRI_EINVAL;
  occri::DeviceGuard guard(dev);
  if (!guard.ok) return OCCRI_ECUDA;
  occri_batch* b = new occri_batch();
  b->device = dev;
  b->plans.assign(plans, plans + nplans);
  b->stream = (cudaStream_t)cuda_stream;
  b->branch.assign(nplans, nullptr);
  b->ev_end.assign(nplans, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < nplans && ok; ++i)
    ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_end[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    occri_impl::batch_free(b);
    return OCCRI_ECUDA;
  }
  *out = b;
  return OCCRI_OK;
}

int occri_batch_build(occri_batch* b, const void* const* C_dev, void* const* KC_dev,
                      void* const* K_dev, double* const* Ex_dev) {
  if (!b || !C_dev) return OCCRI_EINVAL;
  occri::DeviceGuard guard(b->device);
  if (!guard.ok) return OCCRI_ECUDA;
  const size_t n = b->plans.size();
  std::vector<const void*> c(n);
  std::vector<void*> kc(n, nullptr), k(n, nullptr);
  std::vector<double*> ex(n, nullptr);
  for (size_t i = 0; i < n; ++i) {
    if (!C_dev[i]) return OCCRI_EINVAL;
    c[i] = C_dev[i];
    if (KC_dev) kc[i] = KC_dev[i];
    if (K_dev) k[i] = K_dev[i];
    if (Ex_dev) ex[i] = Ex_dev[i];
  }
  if (!b->exec || c != b->c || kc != b->kc || k != b->k || ex != b->ex) {
    b->c = c;
    b->kc = kc;
    b->k = k;
    b->ex = ex;
    const int st = occri_impl::batch_capture(b);
    if (st != OCCRI_OK) {
      b->c.clear();
      return st;
    }
  }
  return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? OCCRI_OK : OCCRI_ECUDA;
}

int occri_batch_sync(occri_batch* b, int* bad_cell, int* bad_k) {
  if (bad_cell) *bad_cell = -1;
  if (bad_k) *bad_k = -1;
  if (!b) return OCCRI_EINVAL;
  occri::DeviceGuard guard(b->device);
  if (!guard.ok) return OCCRI_ECUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return OCCRI_ECUDA;
  int first = OCCRI_OK;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    Plan* p = b->plans[i]->p;
    int st[2] = {0, -1};
    if (cudaMemcpy(st, p->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
      return OCCRI_ECUDA;
    if (st[0] != 0) {
      if (cudaMemset(p->status, 0, sizeof(st)) != cudaSuccess) return OCCRI_ECUDA;
      if (first == OCCRI_OK) {
        first = st[0];
        if (bad_cell) *bad_cell = (int)i;
        if (bad_k) *bad_k = st[1];
      }
    }
  }
  return first;
}

int occri_batch_destroy(occri_batch* b) {
  if (!b) return OCCRI_EINVAL;
  occri::DeviceGuard guard(b->device);
  if (!guard.ok) return OCCRI_ECUDA;
  cudaStreamSynchronize(b->stream);
  occri_impl::batch_free(b);
  return OCCRI_OK;
}

}  // extern "C"
