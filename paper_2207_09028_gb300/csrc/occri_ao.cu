// occri_ao.cu -- Bloch-summed AOs evaluated on the fly (integral-direct, Algorithm 4):
//   (a)+(b) psi_{ik}(r) = sum_mu C^k_{mu i} chi_{mu k}(r)                  (Eq. occmo)
//   (e)     K_{mu i}(k) = -(Omega/(N_k N_g)) sum_r conj(chi_{mu k}(r)) Y_{ik}(r)  (Eq. occrik)
// with chi_{mu k}(r) = sum_T e^{i k.T} phi_mu(r - A - T) (Sec. II.A).
//
// The image sum is split as T = T0(r, A) + T': T0 brings r - A into the
// Wigner-Seitz cell (precomputed per grid point and atom), T' runs over one
// master list of lattice vectors sorted by length. Every thread of a warp walks
// the same prefix of that list (a shell's prefix covers its screening radius
// plus the largest |r - A - T0|), so the image offsets and the phase table
// e^{i k.T'} are warp-uniform loads. chi itself is never stored.
//
// In FP32 the displacement r - A - T is formed from hi/lo float pairs so that
// it is accurate to an ulp of its own size, not of |T|.
#include <cuda_runtime.h>

#include <mutex>

#include "occri_device.cuh"
#include "occri_internal.h"

namespace occri {
namespace ao {

using dev::cis_frac;
using dev::exp_t;

// Unnormalised real solid harmonics, m = -l..l (p: x, y, z).
template <typename T, int L>
__device__ __forceinline__ void solid(T x, T y, T z, T (&P)[2 * L + 1]) {
  if constexpr (L == 0) {
    P[0] = T(1);
  } else if constexpr (L == 1) {
    P[0] = x; P[1] = y; P[2] = z;
  } else if constexpr (L == 2) {
    P[0] = x * y;
    P[1] = y * z;
    P[2] = T(2) * z * z - x * x - y * y;
    P[3] = x * z;
    P[4] = x * x - y * y;
  } else {
    const T x2 = x * x, y2 = y * y, z2 = z * z;
    P[0] = y * (T(3) * x2 - y2);
    P[1] = x * y * z;
    P[2] = y * (T(4) * z2 - x2 - y2);
    P[3] = z * (T(2) * z2 - T(3) * x2 - T(3) * y2);
    P[4] = x * (T(4) * z2 - x2 - y2);
    P[5] = z * (x2 - y2);
    P[6] = x * (x2 - T(3) * y2);
  }
}

// r_n - A - T0 for one grid point and atom, in the working precision.
template <typename T> struct Disp;
template <> struct Disp<double> { double x, y, z; };
template <> struct Disp<float> { float xh, yh, zh, xl, yl, zl; };

__device__ __forceinline__ void load_disp(const AOParams& p, int atom, long long n, Disp<double>* d) {
  const double* b = p.d0_d + (size_t)atom * 3 * p.ng;
  d->x = b[n];
  d->y = b[p.ng + n];
  d->z = b[2 * p.ng + n];
}
__device__ __forceinline__ void load_disp(const AOParams& p, int atom, long long n, Disp<float>* d) {
  const float* h = p.d0_hi + (size_t)atom * 3 * p.ng;
  const float* l = p.d0_lo + (size_t)atom * 3 * p.ng;
  d->xh = h[n]; d->yh = h[p.ng + n]; d->zh = h[2 * p.ng + n];
  d->xl = l[n]; d->yl = l[p.ng + n]; d->zl = l[2 * p.ng + n];
}

__device__ __forceinline__ void image_disp(const AOParams& p, const Disp<double>& d, int j,
                                           double* x, double* y, double* z) {
  *x = d.x - p.img_d[j];
  *y = d.y - p.img_d[p.nimg + j];
  *z = d.z - p.img_d[2 * p.nimg + j];
}
__device__ __forceinline__ void image_disp(const AOParams& p, const Disp<float>& d, int j,
                                           float* x, float* y, float* z) {
  *x = (d.xh - p.img_hi[j]) + (d.xl - p.img_lo[j]);
  *y = (d.yh - p.img_hi[p.nimg + j]) + (d.yl - p.img_lo[p.nimg + j]);
  *z = (d.zh - p.img_hi[2 * p.nimg + j]) + (d.zl - p.img_lo[2 * p.nimg + j]);
}

// Exact-argument Gaussian for FP32: x = (d0 - T') as an unevaluated hi + lo sum (two-diff
// of the hi parts plus the lo parts), r^2 and alpha r^2 as hi + lo pairs (FMA
// two-products, two-sums), and e^{-alpha r^2} = e^{-ah} (1 - al). Returns r^2 (hi) for
// the cutoff test and the coordinates rounded to FP32 for the polynomial.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float exact_gauss(const AOParams& p, const Disp<float>& d, int j,
                                             float ah_, float al_, float* r2h, float* x,
                                             float* y, float* z) {
  float c[3], cl[3];
  const float dh[3] = {d.xh, d.yh, d.zh}, dl[3] = {d.xl, d.yl, d.zl};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float s, e;
    two_sum(dh[q], -p.img_hi[q * p.nimg + j], s, e);
    c[q] = s;
    cl[q] = e + (dl[q] - p.img_lo[q * p.nimg + j]);
  }
  float ph[3], pl[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    ph[q] = c[q] * c[q];
    pl[q] = fmaf(c[q], c[q], -ph[q]) + 2.0f * c[q] * cl[q];
  }
  float s1, e1, s2, e2;
  two_sum(ph[0], ph[1], s1, e1);
  two_sum(s1, ph[2], s2, e2);
  const float rl = (e1 + e2) + (pl[0] + pl[1] + pl[2]);
  *r2h = s2;
  const float ah = ah_ * s2;
  const float al = fmaf(ah_, s2, -ah) + ah_ * rl + al_ * s2;
  *x = c[0] + cl[0];
  *y = c[1] + cl[1];
  *z = c[2] + cl[2];
  return expf(-ah) * (1.0f - al);
}

template <typename T> __device__ __forceinline__ T sh_alpha(const ShellDev& s);
template <> __device__ __forceinline__ double sh_alpha<double>(const ShellDev& s) { return s.alpha; }
template <> __device__ __forceinline__ float sh_alpha<float>(const ShellDev& s) { return s.alpha_f; }
template <typename T> __device__ __forceinline__ T sh_alpha_lo(const ShellDev& s);
template <> __device__ __forceinline__ double sh_alpha_lo<double>(const ShellDev&) { return 0.0; }
template <> __device__ __forceinline__ float sh_alpha_lo<float>(const ShellDev& s) { return s.alpha_lo; }
template <typename T> __device__ __forceinline__ T sh_rcut2(const ShellDev& s);
template <> __device__ __forceinline__ double sh_rcut2<double>(const ShellDev& s) { return s.rcut2; }
template <> __device__ __forceinline__ float sh_rcut2<float>(const ShellDev& s) { return s.rcut2_f; }

// Grid point of `lane` in point block `blk` (2 x 4 x 4 points, ragged at the grid edge);
// lanes outside the grid get a clamped in-range point and *valid = false.
// Point `lane` of block `blk`: its natural index n = (n1 N2 + n2) N3 + n3 (the
// geometry tables) and its index in the orbital/accumulator fields, which are stored
// with the third axis outermost, q = (n3 N1 + n1) N2 + n2 (see occri_internal.h).
// Lanes run along n2 first so that four consecutive lanes touch contiguous elements.
// Points past the grid edge (ragged blocks) are clamped and flagged invalid.
__device__ __forceinline__ long long block_point(const AOParams& p, int blk, int lane, bool* valid,
                                                 long long* q) {
  const int b3 = blk % p.nb[2], b2 = (blk / p.nb[2]) % p.nb[1], b1 = blk / (p.nb[1] * p.nb[2]);
  int n1 = 2 * b1 + (lane >> 4), n2 = 4 * b2 + (lane & 3), n3 = 4 * b3 + ((lane >> 2) & 3);
  *valid = n1 < p.N[0] && n2 < p.N[1] && n3 < p.N[2];
  n1 = min(n1, p.N[0] - 1);
  n2 = min(n2, p.N[1] - 1);
  n3 = min(n3, p.N[2] - 1);
  *q = ((long long)n3 * p.N[0] + n1) * p.N[1] + n2;
  return ((long long)n1 * p.N[1] + n2) * p.N[2] + n3;
}

// e^{i k.T0} for the T0 shared by the points of block `blk` for this atom.
template <typename T>
__device__ __forceinline__ cplx_t<T> phase_t0(const AOParams& p, int atom, int blk, int k) {
  int t[3];
  dev::unpack_t0(p.t0[(size_t)atom * p.nblk + blk], &t[0], &t[1], &t[2]);
  long long num = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    num += (long long)p.kint[k * 3 + d] * t[d] * (p.Dc / p.D[d]);
  return cis_frac<T>(num, p.Dc, +1);
}

// chi_{mu k}(r_n) / N_mu for the 2L+1 functions of one shell, without the e^{i k.T0}
// factor (the normalisation is applied in FP64 outside: folded into C for (b), into
// the reduction for (e)). The images are the first np entries of the block's list,
// identical for all lanes of the warp. In FP32 the exponent uses alpha = alpha_f + alpha_lo.
template <typename T, int L>
__device__ __forceinline__ void shell_values(const AOParams& p, const ShellDev& sh, int k,
                                             const Disp<T>& d, const unsigned short* list, int np,
                                             T (&cr)[2 * L + 1], T (&ci)[2 * L + 1]) {
  const cplx_t<T>* ph = reinterpret_cast<const cplx_t<T>*>(p.img_phase) + (size_t)k * p.nimg;
  const T alpha = sh_alpha<T>(sh), alo = sh_alpha_lo<T>(sh), rc2 = sh_rcut2<T>(sh);
#pragma unroll
  for (int m = 0; m < 2 * L + 1; ++m) {
    cr[m] = T(0);
    ci[m] = T(0);
  }
  const bool exact = (sizeof(T) == 4) && sh.exact_arg;
  for (int j = 0; j < np; ++j) {
    const int idx = list[j];
    T x, y, z, r2, e;
    if constexpr (sizeof(T) == 4) {
      if (exact) {
        e = exact_gauss(p, d, idx, alpha, alo, &r2, &x, &y, &z);
      } else {
        image_disp(p, d, idx, &x, &y, &z);
        r2 = x * x + y * y + z * z;
        e = exp_t(-(alpha * r2 + alo * r2));
      }
    } else {
      image_disp(p, d, idx, &x, &y, &z);
      r2 = x * x + y * y + z * z;
      e = exp_t(-(alpha * r2 + alo * r2));
    }
    if (r2 <= rc2) {
      T P[2 * L + 1];
      solid<T, L>(x, y, z, P);
      const cplx_t<T> w = ph[idx];
#pragma unroll
      for (int m = 0; m < 2 * L + 1; ++m) {
        const T v = P[m] * e;
        cr[m] += w.x * v;
        ci[m] += w.y * v;
      }
    }
  }
}

// chi_{mu k}(r_n)/N_mu for KB consecutive k-points (rows k0..k0+KB-1 of the padded
// phase table); the image geometry, exponential and polynomial are computed once.
template <typename T, int L, int KB>
__device__ __forceinline__ void shell_values_kb(const AOParams& p, const ShellDev& sh, int k0,
                                                const Disp<T>& d, const unsigned short* list,
                                                int np, T (&cr)[KB][2 * L + 1],
                                                T (&ci)[KB][2 * L + 1]) {
  const cplx_t<T>* ph = reinterpret_cast<const cplx_t<T>*>(p.img_phase) + (size_t)k0 * p.nimg;
  const T alpha = sh_alpha<T>(sh), alo = sh_alpha_lo<T>(sh), rc2 = sh_rcut2<T>(sh);
#pragma unroll
  for (int b = 0; b < KB; ++b)
#pragma unroll
    for (int m = 0; m < 2 * L + 1; ++m) {
      cr[b][m] = T(0);
      ci[b][m] = T(0);
    }
  const bool exact = (sizeof(T) == 4) && sh.exact_arg;
  for (int j = 0; j < np; ++j) {
    const int idx = list[j];
    T x, y, z, r2, e;
    if constexpr (sizeof(T) == 4) {
      if (exact) {
        e = exact_gauss(p, d, idx, alpha, alo, &r2, &x, &y, &z);
      } else {
        image_disp(p, d, idx, &x, &y, &z);
        r2 = x * x + y * y + z * z;
        e = exp_t(-(alpha * r2 + alo * r2));
      }
    } else {
      image_disp(p, d, idx, &x, &y, &z);
      r2 = x * x + y * y + z * z;
      e = exp_t(-(alpha * r2 + alo * r2));
    }
    if (r2 <= rc2) {
      T P[2 * L + 1];
      solid<T, L>(x, y, z, P);
#pragma unroll
      for (int m = 0; m < 2 * L + 1; ++m) P[m] *= e;
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const cplx_t<T> w = ph[(size_t)b * p.nimg + idx];
#pragma unroll
        for (int m = 0; m < 2 * L + 1; ++m) {
          cr[b][m] += w.x * P[m];
          ci[b][m] += w.y * P[m];
        }
      }
    }
  }
}


// psi += (N_mu C_mu i) chi_mu / N_mu; in FP32 the scaled coefficient is a hi/lo pair.
__device__ __forceinline__ void cmac(const double2* cs, size_t idx, double xr, double xi,
                                     double& ar, double& ai) {
  const double2 c = cs[idx];
  ar += c.x * xr - c.y * xi;
  ai += c.x * xi + c.y * xr;
}
__device__ __forceinline__ void cmac(const float4* cs, size_t idx, float xr, float xi, float& ar,
                                     float& ai) {
  const float4 c = cs[idx];
  ar += (c.x * xr - c.y * xi) + (c.z * xr - c.w * xi);
  ai += (c.x * xi + c.y * xr) + (c.z * xi + c.w * xr);
}
template <typename T> struct CsType;
template <> struct CsType<double> { using type = double2; };
template <> struct CsType<float> { using type = float4; };

template <typename T, int L, int NI, int KB>
__device__ __forceinline__ void orbital_shell(const AOParams& p, const ShellDev& sh, int k0,
                                              const Disp<T>& d, const unsigned short* list,
                                              int np, const cplx_t<T> (&ph0)[KB], int i0,
                                              T (&ar)[KB][NI], T (&ai)[KB][NI]) {
  using CS = typename CsType<T>::type;
  const CS* cs = reinterpret_cast<const CS*>(p.cs);
  T cr[KB][2 * L + 1], ci[KB][2 * L + 1];
  shell_values_kb<T, L, KB>(p, sh, k0, d, list, np, cr, ci);
#pragma unroll
  for (int b = 0; b < KB; ++b) {
    if (k0 + b >= p.nk) break;
#pragma unroll
    for (int m = 0; m < 2 * L + 1; ++m) {
      const T xr = cr[b][m] * ph0[b].x - ci[b][m] * ph0[b].y;
      const T xi = cr[b][m] * ph0[b].y + ci[b][m] * ph0[b].x;
      const size_t row = ((size_t)(k0 + b) * p.nao + sh.ao + m) * p.nocc;
#pragma unroll
      for (int i = 0; i < NI; ++i)
        if (i0 + i < p.nocc) cmac(cs, row + i0 + i, xr, xi, ar[b][i], ai[b][i]);
    }
  }
}

// Scaled coefficients N_mu C^k_{mu i}, formed in FP64 (and split hi/lo for FP32).
__global__ void scale_c_kernel_d(const double2* __restrict__ C, const double* __restrict__ nrm,
                                 double2* __restrict__ out, int nao, int nocc, long long n,
                                 double factor = 1.0) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double s = factor * nrm[(e / nocc) % nao];
    out[e] = make_double2(s * C[e].x, s * C[e].y);
  }
}
__global__ void scale_c_kernel_f(const double2* __restrict__ C, const double* __restrict__ nrm,
                                 float4* __restrict__ out, int nao, int nocc, long long n,
                                 double factor = 1.0) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double s = factor * nrm[(e / nocc) % nao];
    const double x = s * C[e].x, y = s * C[e].y;
    const float xh = (float)x, yh = (float)y;
    out[e] = make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
  }
}

// One warp per point block, four blocks per CTA; KB k-points per thread. Three CTAs per SM
// (168 registers, a 104-byte spill in FP32) were 7 % faster than two (255 registers).
template <typename T, int NI, int KB>
__global__ void __launch_bounds__(128, 3)
orbitals_kernel(AOParams p, cplx_t<T>* __restrict__ psi, int i0, int kbase = 0) {
  const int blk = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (blk >= p.nblk) return;
  bool valid;
  long long q;
  const long long n = block_point(p, blk, threadIdx.x & 31, &valid, &q);
  const int k0 = kbase + blockIdx.y * KB;
  T ar[KB][NI], ai[KB][NI];
#pragma unroll
  for (int b = 0; b < KB; ++b)
#pragma unroll
    for (int i = 0; i < NI; ++i) { ar[b][i] = T(0); ai[b][i] = T(0); }
  for (int a = 0; a < p.natm; ++a) {
    Disp<T> d;
    load_disp(p, a, n, &d);
    cplx_t<T> ph0[KB];
#pragma unroll
    for (int b = 0; b < KB; ++b)
      ph0[b] = (k0 + b < p.nk) ? phase_t0<T>(p, a, blk, k0 + b) : cplx_t<T>{T(0), T(0)};
    const size_t ab = (size_t)a * p.nblk + blk;
    const unsigned short* list = p.blist + ab * p.lmax;
    const unsigned short* pre = p.bpre + ab * p.nsa;
    const int s0 = p.atom_shell0[a];
    for (int s = s0; s < p.atom_shell0[a + 1]; ++s) {
      const ShellDev sh = p.shells[s];
      const int np = pre[s - s0];
      switch (sh.l) {
        case 0: orbital_shell<T, 0, NI, KB>(p, sh, k0, d, list, np, ph0, i0, ar, ai); break;
        case 1: orbital_shell<T, 1, NI, KB>(p, sh, k0, d, list, np, ph0, i0, ar, ai); break;
        case 2: orbital_shell<T, 2, NI, KB>(p, sh, k0, d, list, np, ph0, i0, ar, ai); break;
        default: orbital_shell<T, 3, NI, KB>(p, sh, k0, d, list, np, ph0, i0, ar, ai); break;
      }
    }
  }
  if (!valid) return;
#pragma unroll
  for (int b = 0; b < KB; ++b) {
    if (k0 + b >= p.nk) break;
#pragma unroll
    for (int i = 0; i < NI; ++i)
      if (i0 + i < p.nocc)
        psi[((size_t)(k0 + b) * p.nocc + i0 + i) * p.fs + q] = cplx_t<T>{ar[b][i], ai[b][i]};
  }
}

// ------------------------------------------------------------------ (e)

template <typename T, int L, int NI>
__global__ void __launch_bounds__(256)
contract_kernel(AOParams p, const cplx_t<T>* __restrict__ Y, double2* __restrict__ kc,
                const int* __restrict__ shell_list, int i0, long long chunk, double scale,
                int kbase) {
  constexpr int NM = 2 * L + 1;
  constexpr int NV = 2 * NM * NI;
  const int s = shell_list[blockIdx.z];
  const int k = kbase + blockIdx.y;
  const ShellDev sh = p.shells[s];
  const int start = blockIdx.x * (int)chunk;
  const int end = min(p.nblk, start + (int)chunk);
  const int s0 = p.atom_shell0[sh.atom];
  T ar[NM][NI], ai[NM][NI];
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int i = 0; i < NI; ++i) { ar[m][i] = T(0); ai[m][i] = T(0); }
  for (int blk = start + (int)(threadIdx.x >> 5); blk < end; blk += (int)(blockDim.x >> 5)) {
    bool valid;
    long long q;
    const long long n = block_point(p, blk, threadIdx.x & 31, &valid, &q);
    Disp<T> d;
    load_disp(p, sh.atom, n, &d);
    const cplx_t<T> ph0 = phase_t0<T>(p, sh.atom, blk, k);
    const size_t ab = (size_t)sh.atom * p.nblk + blk;
    T cr[NM], ci[NM];
    shell_values<T, L>(p, sh, k, d, p.blist + ab * p.lmax, p.bpre[ab * p.nsa + (s - s0)], cr, ci);
    T yr[NI], yi[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      if (valid && i0 + i < p.nocc) {
        const cplx_t<T> y = Y[((size_t)k * p.nocc + i0 + i) * p.fs + q];
        yr[i] = y.x; yi[i] = y.y;
      } else {
        yr[i] = T(0); yi[i] = T(0);
      }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const T xr = cr[m] * ph0.x - ci[m] * ph0.y;
      const T xi = cr[m] * ph0.y + ci[m] * ph0.x;
#pragma unroll
      for (int i = 0; i < NI; ++i) {  // conj(chi) * y
        ar[m][i] += xr * yr[i] + xi * yi[i];
        ai[m][i] += xr * yi[i] - xi * yr[i];
      }
    }
  }
  __shared__ double red[8][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      double vr = double(ar[m][i]), vi = double(ai[m][i]);
      for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (lane == 0) {
        red[warp][2 * (m * NI + i)] = vr;
        red[warp][2 * (m * NI + i) + 1] = vi;
      }
    }
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += blockDim.x) {
    const int mi = v >> 1, m = mi / NI, i = mi - (mi / NI) * NI;
    if (i0 + i >= p.nocc) continue;
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][v];
    double* dst = reinterpret_cast<double*>(kc + ((size_t)k * p.nao + sh.ao + m) * p.nocc + i0 + i);
    atomicAdd(dst + (v & 1), scale * sh.norm[m] * t);
  }
}

// Widen the fields to c128 and put them back in natural point order:
// out[f][(n1 N + n2) N + n3] = in[f][(n3 N + n1) N + n2] (cubic grid of edge N; input
// fields fs points apart, output fields N^3 apart).
template <typename T>
__global__ void widen_kernel(const cplx_t<T>* __restrict__ in, double2* __restrict__ out,
                             long long n, int N, long long fs) {
  const long long ng = (long long)N * N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long f = e / ng, r = e - f * ng;
    const int n3 = (int)(r % N), n2 = (int)((r / N) % N), n1 = (int)(r / ((long long)N * N));
    const cplx_t<T> v = in[f * fs + ((long long)n3 * N + n1) * N + n2];
    out[e] = make_double2(double(v.x), double(v.y));
  }
}


// F[k][i][q] *= e^{sign i k.r_q} for every orbital field of every k-point (fields'
// point order q = (n3 N + n1) N + n2, cubic grid of edge N). With sign = -1 this turns
// the Bloch orbitals psi_ik into their periodic parts u_ik = e^{-ik.r} psi_ik, with
// sign = +1 it turns the accumulated periodic parts back into Y_ik. The phase is
// 2 pi sum_d kint_d n_d / (D_d N), reduced exactly in integers.
template <typename T>
__global__ void phase_fields_kernel(cplx_t<T>* __restrict__ F, const int* __restrict__ kint,
                                    int k0, int nk, int nocc, int N, long long fs, int D0, int D1,
                                    int D2, int sign) {
  const long long ng = (long long)N * N * N;
  const long long Dc = (long long)D0 * D1 * D2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nk * ng;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = k0 + (int)(e / ng);
    const long long q = e - (long long)(k - k0) * ng;
    const int n3 = (int)(q / ((long long)N * N));
    const int rem = (int)(q - (long long)n3 * N * N);
    const int n1 = rem / N, n2 = rem - (rem / N) * N;
    const long long num = (long long)kint[3 * k] * n1 * (Dc / D0) +
                          (long long)kint[3 * k + 1] * n2 * (Dc / D1) +
                          (long long)kint[3 * k + 2] * n3 * (Dc / D2);
    const cplx_t<T> ph = dev::cis_frac<T>(num, Dc * N, sign);
    cplx_t<T>* f = F + (size_t)k * nocc * fs + q;
    for (int i = 0; i < nocc; ++i) {
      const cplx_t<T> v = f[(size_t)i * fs];
      f[(size_t)i * fs] = cplx_t<T>{v.x * ph.x - v.y * ph.y, v.x * ph.y + v.y * ph.x};
    }
  }
}

}  // namespace ao

template <>
cudaError_t launch_scale_c<double>(const Plan& p, const double2* C, cudaStream_t s) {
  const long long n = (long long)p.nk * p.nao * p.nocc;
  ao::scale_c_kernel_d<<<2 * 152, 256, 0, s>>>(C, p.ao_norm, (double2*)p.cs, p.nao, p.nocc, n);
  return cudaGetLastError();
}
template <>
cudaError_t launch_scale_c<float>(const Plan& p, const double2* C, cudaStream_t s) {
  const long long n = (long long)p.nk * p.nao * p.nocc;
  ao::scale_c_kernel_f<<<2 * 152, 256, 0, s>>>(C, p.ao_norm, (float4*)p.cs, p.nao, p.nocc, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_phase_fields(const Plan& p, void* F, int sign, cudaStream_t s, int k0, int nkk) {
  if (nkk < 0) nkk = p.nk - k0;
  ao::phase_fields_kernel<T><<<8 * 152, 256, 0, s>>>((cplx_t<T>*)F, p.kint, k0, nkk, p.nocc,
                                                      p.N[0], p.fs, p.D[0], p.D[1], p.D[2], sign);
  return cudaGetLastError();
}
template cudaError_t launch_phase_fields<float>(const Plan&, void*, int, cudaStream_t, int, int);
template cudaError_t launch_phase_fields<double>(const Plan&, void*, int, cudaStream_t, int, int);

template <typename T>
cudaError_t launch_orbitals_to(const Plan& p, const void* cs, void* out, cudaStream_t s, int k0,
                               int nkk) {
  constexpr int NI = kOrbChunk, KB = orbital_kbatch<T>();
  if (nkk < 0) nkk = p.nk - k0;
  AOParams ap = p.ao_params();
  ap.cs = cs;
  dim3 grid((unsigned)((p.nblk + 3) / 4), (nkk + KB - 1) / KB);
  for (int i0 = 0; i0 < p.nocc; i0 += NI)
    ao::orbitals_kernel<T, NI, KB><<<grid, 128, 0, s>>>(ap, (cplx_t<T>*)out, i0, k0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_orbitals(const Plan& p, cudaStream_t s) {
  return launch_orbitals_to<T>(p, p.cs, p.psi, s, 0, -1);
}

// Scaled coefficients factor N_mu X^k_{mu i} of any [nk][nao][nocc] c128 array X, in the
// plan's coefficient format, into `out` (sized like the plan's own coefficients).
template <>
cudaError_t launch_scale_to<double>(const Plan& p, const double2* X, void* out, double factor,
                                    cudaStream_t s) {
  const long long n = (long long)p.nk * p.nao * p.nocc;
  ao::scale_c_kernel_d<<<2 * 152, 256, 0, s>>>(X, p.ao_norm, (double2*)out, p.nao, p.nocc, n,
                                               factor);
  return cudaGetLastError();
}
template <>
cudaError_t launch_scale_to<float>(const Plan& p, const double2* X, void* out, double factor,
                                   cudaStream_t s) {
  const long long n = (long long)p.nk * p.nao * p.nocc;
  ao::scale_c_kernel_f<<<2 * 152, 256, 0, s>>>(X, p.ao_norm, (float4*)out, p.nao, p.nocc, n,
                                               factor);
  return cudaGetLastError();
}

template <typename T, int L>
static void launch_contract_l(const Plan& p, const AOParams& ap, const void* Yf, double2* out,
                              double scale, cudaStream_t s, int k0, int nkk) {
  constexpr int NI = contract_chunk<T>();
  const int ns = (int)p.shells_by_l[L].size();
  if (ns == 0) return;
  const long long target = 4LL * 152 * 8;   // CTAs to fill the GPU several times over
  long long parts = (target + (long long)nkk * ns - 1) / ((long long)nkk * ns);
  const long long maxparts = (p.nblk + 31) / 32;   // at least 32 point blocks per CTA
  if (parts > maxparts) parts = maxparts;
  if (parts < 1) parts = 1;
  const long long chunk = (p.nblk + parts - 1) / parts;
  for (int i0 = 0; i0 < p.nocc; i0 += NI)
    ao::contract_kernel<T, L, NI><<<dim3((unsigned)parts, nkk, ns), 256, 0, s>>>(
        ap, (const cplx_t<T>*)Yf, out, p.shell_list_l[L], i0, chunk, scale, k0);
}

// out[k][mu][i] += scale N_mu sum_r conj(chi~_{mu k}(r)) F_ik(r) for an orbital-shaped field F
template <typename T>
cudaError_t launch_contract_field(const Plan& p, const void* F, double2* out, double scale,
                                  cudaStream_t s, int k0, int nkk) {
  if (nkk < 0) nkk = p.nk - k0;
  const AOParams ap = p.ao_params();
  launch_contract_l<T, 0>(p, ap, F, out, scale, s, k0, nkk);
  launch_contract_l<T, 1>(p, ap, F, out, scale, s, k0, nkk);
  launch_contract_l<T, 2>(p, ap, F, out, scale, s, k0, nkk);
  launch_contract_l<T, 3>(p, ap, F, out, scale, s, k0, nkk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_contract(const Plan& p, cudaStream_t s, int k0, int nkk) {
  // Y carries N_g/(4 pi) (see PairParams), hence -Omega 4 pi / (N_k N_g^2)
  const double scale = -p.omega_cell * 4.0 * 3.14159265358979323846 /
                       ((double)p.nk * (double)p.ng * (double)p.ng);
  return launch_contract_field<T>(p, p.Y, p.kc, scale, s, k0, nkk);
}

template <typename T>
cudaError_t launch_widen(const Plan& p, void* out, cudaStream_t s) {
  const long long n = (long long)p.nk * p.nocc * p.ng;
  ao::widen_kernel<T><<<4 * 152, 256, 0, s>>>((const cplx_t<T>*)p.psi, (double2*)out, n, p.N[0],
                                               p.fs);
  return cudaGetLastError();
}

template cudaError_t launch_orbitals<float>(const Plan&, cudaStream_t);
template cudaError_t launch_orbitals<double>(const Plan&, cudaStream_t);
template cudaError_t launch_orbitals_to<float>(const Plan&, const void*, void*, cudaStream_t, int,
                                               int);
template cudaError_t launch_orbitals_to<double>(const Plan&, const void*, void*, cudaStream_t, int,
                                                int);
template cudaError_t launch_contract_field<float>(const Plan&, const void*, double2*, double,
                                                  cudaStream_t, int, int);
template cudaError_t launch_contract_field<double>(const Plan&, const void*, double2*, double,
                                                   cudaStream_t, int, int);
template cudaError_t launch_contract<float>(const Plan&, cudaStream_t, int, int);
template cudaError_t launch_contract<double>(const Plan&, cudaStream_t, int, int);
template cudaError_t launch_widen<float>(const Plan&, void*, cudaStream_t);
template cudaError_t launch_widen<double>(const Plan&, void*, cudaStream_t);

}  // namespace occri

// ------------------------------------------------------------------ orbitals without allocation
//
// occri_orbitals_noalloc runs the same kernels as occri_orbitals but keeps its
// scratch -- the normalised coefficients N_mu C^k_{mu i} and the orbitals in the
// plan's working precision before widening -- in this file-scope device array
// instead of the plan's workspaces. Every GPU that loads the library reserves
// OCCRI_STATIC_SCRATCH_BYTES of device memory for it until the process exits.
static __device__ __align__(256) unsigned char occri_static_scratch[OCCRI_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

size_t round_up_256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the static array for the current device (looked up once per device,
// with that device current; the host-side symbol itself is not a device address). The
// caller has made the plan's device current.
int static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return OCCRI_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return OCCRI_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, occri_static_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return OCCRI_ECUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return OCCRI_OK;
}

template <typename T>
int orbitals_noalloc_impl(const occri::Plan& p, const double2* C, void* psi_out, void* base) {
  using namespace occri;
  using CS = typename ao::CsType<T>::type;
  const long long ncs = (long long)p.nk * p.nao * p.nocc;
  const long long npsi = (long long)p.nk * p.nocc * p.ng;   // outputs (natural order)
  CS* cs = reinterpret_cast<CS*>(base);
  cplx_t<T>* psi = reinterpret_cast<cplx_t<T>*>(static_cast<unsigned char*>(base) +
                                                round_up_256(sizeof(CS) * ncs));
  cudaStream_t s = p.stream;
  if constexpr (sizeof(T) == 8)
    ao::scale_c_kernel_d<<<2 * 152, 256, 0, s>>>(C, p.ao_norm, cs, p.nao, p.nocc, ncs);
  else
    ao::scale_c_kernel_f<<<2 * 152, 256, 0, s>>>(C, p.ao_norm, cs, p.nao, p.nocc, ncs);
  AOParams ap = p.ao_params();
  ap.cs = cs;
  constexpr int KB = orbital_kbatch<T>();
  const dim3 grid((unsigned)((p.nblk + 3) / 4), (p.nk + KB - 1) / KB);
  for (int i0 = 0; i0 < p.nocc; i0 += kOrbChunk)
    ao::orbitals_kernel<T, kOrbChunk, KB><<<grid, 128, 0, s>>>(ap, psi, i0);
  ao::widen_kernel<T><<<4 * 152, 256, 0, s>>>(psi, (double2*)psi_out, npsi, p.N[0], p.fs);
  return cudaGetLastError() == cudaSuccess ? OCCRI_OK : OCCRI_ECUDA;
}

}  // namespace

extern "C" int occri_orbitals_noalloc(const occri_plan* plan, const void* C_dev, void* psi_dev) {
  if (!plan || !C_dev || !psi_dev) return OCCRI_EINVAL;
  const occri::Plan& p = *plan->p;
  // the plan's device is made current, so the scratch address below is that device's
  occri::DeviceGuard guard(p.device);
  if (!guard.ok) return OCCRI_ECUDA;
  const bool fp64 = p.precision == OCCRI_FP64;
  const size_t ncs = (size_t)p.nk * p.nao * p.nocc;
  const size_t npsi = (size_t)p.nk * p.nocc * p.fs;   // internal fields, fs points apart
  const size_t need = round_up_256((fp64 ? sizeof(double2) : sizeof(float4)) * ncs) +
                      (fp64 ? sizeof(double2) : sizeof(float2)) * npsi;
  if (need > (size_t)OCCRI_STATIC_SCRATCH_BYTES) return OCCRI_EINVAL;
  void* base = nullptr;
  const int st = static_scratch_address(&base);
  if (st != OCCRI_OK) return st;
  return fp64 ? orbitals_noalloc_impl<double>(p, (const double2*)C_dev, psi_dev, base)
              : orbitals_noalloc_impl<float>(p, (const double2*)C_dev, psi_dev, base);
}
