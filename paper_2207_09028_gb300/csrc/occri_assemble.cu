// occri_assemble.cu -- the paper's form of the occ-RI assembly and the conduction-band
// columns (Sec. II.C, Eq. occrikop; Sec. II.D, conduction-band paragraph), in FP64.
//
// From the AO-occupied block KC = <mu|K|j> (Eq. occrik) and the S-orthonormal orbitals C of
// each k, with P = C C^H S the projector on span(C) and Q = 1 - P:
//   K ~ PKP + PKQ + QKP = KC (S C)^H + (S C) KC^H - (S C) M (S C)^H,   M = herm(C^H KC).
// Three kernels per call: M (one thread per entry), then T = S C and D = KC - T M per block
// of AO rows, then K = D T^H + T KC^H per 16 x 16 tile.
//
// Conduction bands: K_{mu p} for p among chosen conduction bands R, with the sum over the
// occupied orbitals only, is the difference of two ordinary builds: one whose orbitals are
// occupied + R (every orbital summed over) and one whose orbitals are R alone (the R terms
// of the first). band_diff_kernel takes that difference.
#include <cuda_runtime.h>

#include "occri_internal.h"

namespace occri {
namespace {

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // a b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {  // conj(a) b + c
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfmbc(double2 a, double2 b, double2 c) {  // a conj(b) + c
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.y, b.x, fma(-a.x, b.y, c.y)));
}

// M[k][a][b] = sum_mu conj(C[mu][a]) KC[mu][b] (not yet Hermitised)
__global__ void paper_m_kernel(const double2* __restrict__ C, const double2* __restrict__ KC,
                               double2* __restrict__ M, int nao, int ncol) {
  const int k = blockIdx.x;
  const int e = blockIdx.y * blockDim.x + threadIdx.x;
  if (e >= ncol * ncol) return;
  const int a = e / ncol, b = e - a * ncol;
  const double2* c = C + (size_t)k * nao * ncol;
  const double2* kc = KC + (size_t)k * nao * ncol;
  double2 s = make_double2(0.0, 0.0);
  for (int mu = 0; mu < nao; ++mu) s = cfmac(c[(size_t)mu * ncol + a], kc[(size_t)mu * ncol + b], s);
  M[((size_t)k * ncol + a) * ncol + b] = s;
}

constexpr int kRowBlock = 16;

// For AO rows [16 blockIdx.y, +16): T = S C, then D = KC - T herm(M).
__global__ void paper_t_kernel(const double2* __restrict__ S, const double2* __restrict__ C,
                               const double2* __restrict__ KC, const double2* __restrict__ M,
                               double2* __restrict__ T, double2* __restrict__ D, int nao,
                               int ncol) {
  const int k = blockIdx.x;
  const int r0 = blockIdx.y * kRowBlock;
  const int rows = min(kRowBlock, nao - r0);
  const double2* s = S + (size_t)k * nao * nao;
  const double2* c = C + (size_t)k * nao * ncol;
  const double2* kc = KC + (size_t)k * nao * ncol;
  const double2* m = M + (size_t)k * ncol * ncol;
  double2* t = T + (size_t)k * nao * ncol;
  double2* d = D + (size_t)k * nao * ncol;
  for (int e = threadIdx.x; e < rows * ncol; e += blockDim.x) {
    const int mu = r0 + e / ncol, a = e % ncol;
    double2 acc = make_double2(0.0, 0.0);
    for (int nu = 0; nu < nao; ++nu)
      acc = cfma(s[(size_t)mu * nao + nu], c[(size_t)nu * ncol + a], acc);
    t[(size_t)mu * ncol + a] = acc;
  }
  __syncthreads();   // this block's rows of T are written (and visible to the block)
  for (int e = threadIdx.x; e < rows * ncol; e += blockDim.x) {
    const int mu = r0 + e / ncol, a = e % ncol;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < ncol; ++b) {
      const double2 mba = m[(size_t)b * ncol + a], mab = m[(size_t)a * ncol + b];
      const double2 h = make_double2(0.5 * (mba.x + mab.x), 0.5 * (mba.y - mab.y));
      acc = cfma(t[(size_t)mu * ncol + b], h, acc);
    }
    const double2 x = kc[(size_t)mu * ncol + a];
    d[(size_t)mu * ncol + a] = make_double2(x.x - acc.x, x.y - acc.y);
  }
}

// K[mu][nu] = sum_a D[mu][a] conj(T[nu][a]) + T[mu][a] conj(KC[nu][a])
__global__ void paper_k_kernel(const double2* __restrict__ T, const double2* __restrict__ D,
                               const double2* __restrict__ KC, double2* __restrict__ K, int nao,
                               int ncol) {
  const int k = blockIdx.x;
  const int mu = blockIdx.y * 16 + threadIdx.y, nu = blockIdx.z * 16 + threadIdx.x;
  if (mu >= nao || nu >= nao) return;
  const double2* t = T + (size_t)k * nao * ncol;
  const double2* d = D + (size_t)k * nao * ncol;
  const double2* kc = KC + (size_t)k * nao * ncol;
  double2 acc = make_double2(0.0, 0.0);
  for (int a = 0; a < ncol; ++a) {
    acc = cfmbc(d[(size_t)mu * ncol + a], t[(size_t)nu * ncol + a], acc);
    acc = cfmbc(t[(size_t)mu * ncol + a], kc[(size_t)nu * ncol + a], acc);
  }
  K[((size_t)k * nao + mu) * nao + nu] = acc;
}

// out[k][mu][r] = all[k][mu][nocc + r] - rr[k][mu][r]
__global__ void band_diff_kernel(const double2* __restrict__ all, const double2* __restrict__ rr,
                                 double2* __restrict__ out, long long rows, int nocc, int nr) {
  const long long n = rows * nr;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / nr;
    const int r = (int)(e - row * nr);
    const double2 a = all[row * (nocc + nr) + nocc + r], b = rr[e];
    out[e] = make_double2(a.x - b.x, a.y - b.y);
  }
}

// c_r[k][mu][r] = C_all[k][mu][nocc + r]
__global__ void gather_cols_kernel(const double2* __restrict__ all, double2* __restrict__ cr,
                                   long long rows, int nocc, int nr) {
  const long long n = rows * nr;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / nr;
    cr[e] = all[row * (nocc + nr) + nocc + (int)(e - row * nr)];
  }
}

}  // namespace

cudaError_t launch_assemble_paper(Plan& p, int ncol, const double2* S, const double2* C,
                                  const double2* KC, double2* K) {
  const size_t need = sizeof(double2) * ((size_t)p.nk * ncol * ncol + 2 * (size_t)p.nk * p.nao * ncol);
  if (p.asm_bytes < need) {
    if (p.asm_scratch) {
      // the previous call's kernels may still read the old buffer
      if (cudaStreamSynchronize(p.stream) != cudaSuccess) return cudaGetLastError();
      cudaFree(p.asm_scratch);
      p.asm_scratch = nullptr;
      p.asm_bytes = 0;
    }
    cudaError_t e = device_malloc(&p.asm_scratch, need);
    if (e != cudaSuccess) return e;
    p.asm_bytes = need;
  }
  double2* M = (double2*)p.asm_scratch;
  double2* T = M + (size_t)p.nk * ncol * ncol;
  double2* D = T + (size_t)p.nk * p.nao * ncol;
  const dim3 gm(p.nk, (ncol * ncol + 255) / 256);
  paper_m_kernel<<<gm, 256, 0, p.stream>>>(C, KC, M, p.nao, ncol);
  const dim3 gt(p.nk, (p.nao + kRowBlock - 1) / kRowBlock);
  paper_t_kernel<<<gt, 256, 0, p.stream>>>(S, C, KC, M, T, D, p.nao, ncol);
  const dim3 gk(p.nk, (p.nao + 15) / 16, (p.nao + 15) / 16);
  paper_k_kernel<<<gk, dim3(16, 16), 0, p.stream>>>(T, D, KC, K, p.nao, ncol);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(const double2* all, double2* cr, long long rows, int nocc, int nr,
                               cudaStream_t s) {
  gather_cols_kernel<<<1216, 256, 0, s>>>(all, cr, rows, nocc, nr);
  return cudaGetLastError();
}

cudaError_t launch_band_diff(const double2* all, const double2* rr, double2* out, long long rows,
                             int nocc, int nr, cudaStream_t s) {
  band_diff_kernel<<<1216, 256, 0, s>>>(all, rr, out, rows, nocc, nr);
  return cudaGetLastError();
}

}  // namespace occri
