// occri_contract_tc.cu -- step (e), K_{mu i}(k) = -(Omega/(N_k N_g)) sum_r conj(chi_{mu k}(r))
// Y_ik(r) (Eq. occrik, the last step of Algorithm 3), as one dense GEMM on the tensor cores.
//
// Formulation. Let D_d be the k denominators (kappa_{k,d} = kint_d / D_d), L_l = sum_d l_d a_d
// for l_d in [0, D_d) the cell offsets of the D1 x D2 x D3 supercell, and
// Phi_mu(x) = sum_S phi_mu(x - A_mu - S) the AO periodised over the supercell lattice S
// (e^{ik.S} = 1 there). Then conj(chi_{mu k}(r)) = sum_l e^{-ik.L_l} Phi_mu(r - L_l), and
//   K_{mu i}(k) = scale sum_l e^{-ik.L_l} P_l[mu, (k,i)],   P_l = sum_r Phi_mu(r - L_l) Y_ik(r).
// P_l is a real-by-complex GEMM: rows mu (128 AOs per tile, sorted by screening radius so that
// tight AOs share tiles), columns the (Re, Im) of 128 (k, i) pairs (N = 256), reduction over the
// cell's grid points, 32 per stage. Its A operand Phi (real, generated on the fly from the
// Gaussians, never stored) and its B operand (Y converted once per build to FP16 hi/lo pairs
// in the tensor cores' shared-memory layout) are split hi + lo, and three FP16 MMAs
// (hi.hi + hi.lo + lo.hi) with FP32 accumulation give FP32-level products. The sum over l
// with the phases e^{-ik.L_l} is applied to each P_l in tensor memory by the epilogue warps
// (acc -> running sum), and the running sums go to K_{mu i} by FP64 atomics. Stages where no
// AO of the tile reaches the points (r - L_l) are skipped: tight AOs are sparse here.
//
// Warp roles (one CTA per SM, persistent over a host-made list of work chunks):
//   warp 0      TMEM allocation; lane 0 issues the MMAs and commits them to mbarriers
//   warp 1      lane 0 copies each stage's B block (32 KB) with the bulk-copy engine
//   warps 2-9   generate the A tile of each stage (FP16 hi/lo) into shared memory
//   warps 10-13 epilogue: P_l from tensor memory, phases, running sums, FP64 atomics
// Every mbarrier wait is bounded by the plan's wait limit; on timeout the kernel records
// OCCRI_ETIMEOUT and the CTA leaves (each role stops issuing; no copy is left in flight
// unless its own wait failed).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "occri_device.cuh"
#include "occri_internal.h"
#include "occri_tc.cuh"

namespace occri {
namespace tcc {

constexpr int kM = 128;             // AO rows per tile (TMEM lanes)
constexpr int kNC = 128;            // complex (k, i) columns per tile
constexpr int kN = 2 * kNC;         // real columns (Re, Im)
constexpr int kKP = 32;             // grid points per stage (MMA K, two slices of 16)
constexpr int kStages = 4;
constexpr int kChunkTiles = 16;     // point tiles per work chunk (its B blocks stay in L2)
constexpr int kFlushChunks = 8;     // chunks summed in FP32 before the FP64 atomics
constexpr int kMaxImg = 512;        // supercell images of one stage, all atoms
constexpr int kAWarps = 8, kEWarps = 4;
constexpr int kThreads = 32 * (2 + kAWarps + kEWarps);
constexpr int kASlice = kM * 16 * 2;          // bytes of one K slice of A (hi or lo)
constexpr int kBSlice = kN * 16 * 2;          // bytes of one K slice of B
constexpr int kABytes = 2 * kASlice;          // A hi (or lo) of a stage
constexpr int kBBytes = 2 * kBSlice;          // B hi (or lo) of a stage
constexpr int kBBlock = 2 * kBBytes;          // one converted Y block (hi then lo): 32 KB
constexpr int kStageBytes = 2 * kABytes + kBBlock;
constexpr uint32_t kIdesc = tc::idesc_f16_f32(kM, kN);
// Descriptor strides of the no-swizzle K-major layout used below: inside one 16-wide K slice,
// an 8-row group holds its two 8-column core matrices at +0 and +128 bytes and groups follow
// every 256 bytes.
constexpr uint32_t kLBO = 128, kSBO = 256;
constexpr float kScaleTarget = 8192.f;        // operands scaled to |x| < 2^13 (FP16 max 65504)

// byte offset of element (row, k) inside one operand of a stage (slices of 16 along K)
__host__ __device__ constexpr int op_off(int row, int k, int slice_bytes) {
  return (k >> 4) * slice_bytes + (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 +
         (k & 7) * 2;
}

struct TcShell {        // the rows of one shell inside a tile
  float alpha, alpha_lo, rcut2;
  int atom, l, row0, m0, nm;
};

struct TcParams {
  int nk, nao, nocc, natm, N, ncol, n_ct, ntile_r, nl, nwords;
  int D[3], w[3];
  long long ng;
  const unsigned char* yh;       // converted Y blocks [ct][rt][32 KB]
  const TcShell* shells;
  const int* tile_shell0;        // shells of tile t: [tile_shell0[t], tile_shell0[t+1])
  const float* rowscale;         // [tile*128 + row]
  const double* rowf;            // N_mu / rowscale, 0 on pad rows
  const int* perm;               // tile row -> AO (or -1)
  const float* reach;            // [tile][natm] largest screening radius of the tile's shells
  const float4* rtiles;          // [ntile_r] centre (x, y, z) and radius of the point tile
  const unsigned* active;        // [tile][ntile_r][nwords] bit l: the tile reaches r - L_l
  const int4* chunks;            // (tile, ct, offset into chunk_rt, count | flags << 8)
  const int* chunk_rt;           // point tiles of each chunk
  const int* cta_chunk0;         // chunks of CTA b: [cta_chunk0[b], cta_chunk0[b+1])
  const int* kint;               // [nk][3]
  const unsigned* colmax;        // [ncol] max over r of |Re Y| + |Im Y| (float bits)
  double2* kc;
  double scale;
  float lat[9], sc[9], scinv[9]; // rows a_d; supercell rows D_d a_d; cart -> supercell frac
  int aint[kMaxTcAtoms][3];
  float arem_hi[kMaxTcAtoms][3], arem_lo[kMaxTcAtoms][3], axyz[kMaxTcAtoms][3];
  int* status;
  long long wait_ns;
};

enum { kFirstSum = 1 << 8, kToGlobal = 1 << 9 };

__device__ __forceinline__ void fail(int* status) {
  if (status && atomicCAS(status, 0, (int)OCCRI_ETIMEOUT) == 0) status[1] = -1;
}

// Unnormalised real solid harmonics (m = -l..l; p: x, y, z), as the AO kernels.
template <int L>
__device__ __forceinline__ void solid_h(float x, float y, float z, float (&P)[2 * L + 1]) {
  if constexpr (L == 0) {
    P[0] = 1.f;
  } else if constexpr (L == 1) {
    P[0] = x; P[1] = y; P[2] = z;
  } else if constexpr (L == 2) {
    P[0] = x * y;
    P[1] = y * z;
    P[2] = 2.f * z * z - x * x - y * y;
    P[3] = x * z;
    P[4] = x * x - y * y;
  } else {
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    P[0] = y * (3.f * x2 - y2);
    P[1] = x * y * z;
    P[2] = y * (4.f * z2 - x2 - y2);
    P[3] = z * (2.f * z2 - 3.f * x2 - 3.f * y2);
    P[4] = x * (4.f * z2 - x2 - y2);
    P[5] = z * (x2 - y2);
    P[6] = x * (x2 - 3.f * y2);
  }
}

struct Img { int atom, s0, s1, s2; };

struct __align__(16) Smem {
  unsigned long long full_a[kStages], full_b[kStages], empty[kStages], acc_full, acc_empty, done;
  uint32_t tmem_slot;
  int a_ok[2], e_ok;
  int nimg[2];
  int img_off[2][kMaxTcAtoms + 1];
  Img img[2][kMaxImg];
  float2 phase[kNC];
  double colinv[kNC];
};

// ---- the iteration every role walks identically: chunks -> l groups -> stages
struct Walk {
  const unsigned* active;
  const int* chunk_rt;
  int ntile_r, nwords, c0, c1;
  __device__ __forceinline__ const unsigned* act(int tile, int rt) const {
    return active + ((size_t)tile * ntile_r + rt) * nwords;
  }
  __device__ __forceinline__ bool on(int tile, int rt, int l) const {
    return (act(tile, rt)[l >> 5] >> (l & 31)) & 1u;
  }
  // union over the chunk's point tiles of the active l bits, word w
  __device__ __forceinline__ unsigned lmask(const int4& ch, int w) const {
    unsigned m = 0;
    const int n = ch.w & 255;
    for (int j = 0; j < n; ++j) m |= act(ch.x, chunk_rt[ch.z + j])[w];
    return m;
  }
};

// A tile of one stage: rows of the tile's shells at points q0 .. q0+31 shifted by -L_l.
__device__ __forceinline__ void gen_a(const TcParams& p, const Smem& sm, int ib, int tile,
                                      int rt, const int l3[3], unsigned char* a_hi,
                                      unsigned char* a_lo, int t) {
  const int s0 = p.tile_shell0[tile], s1 = p.tile_shell0[tile + 1];
  const int items = (s1 - s0) * 4;
  const int N = p.N;
  const float invN = 1.f / (float)N;
  for (int it = t; it < items; it += 32 * kAWarps) {
    const int e = s0 + (it >> 2), g = it & 3;
    const TcShell sh = p.shells[e];
    float v[7][8];
#pragma unroll
    for (int m = 0; m < 7; ++m)
#pragma unroll
      for (int j = 0; j < 8; ++j) v[m][j] = 0.f;
    int n[8][3];
    bool ok[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long q = (long long)rt * kKP + g * 8 + j;
      ok[j] = q < p.ng;
      const int qq = ok[j] ? (int)q : 0;
      n[j][1] = qq % N;                 // n2 (fields' order q = (n3 N + n1) N + n2)
      const int tq = qq / N;
      n[j][0] = tq % N;                 // n1
      n[j][2] = tq / N;                 // n3
    }
    const int a = sh.atom;
    const int i0 = sm.img_off[ib][a], i1 = sm.img_off[ib][a + 1];
    for (int im = i0; im < i1; ++im) {
      const Img S = sm.img[ib][im];
      const int sd[3] = {S.s0, S.s1, S.s2};
      int base[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) base[d] = N * (l3[d] + sd[d] * p.D[d]) + p.aint[a][d];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float gf[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
          gf[d] = (((float)(n[j][d] - base[d]) - p.arem_hi[a][d]) - p.arem_lo[a][d]) * invN;
        const float x = gf[0] * p.lat[0] + gf[1] * p.lat[3] + gf[2] * p.lat[6];
        const float y = gf[0] * p.lat[1] + gf[1] * p.lat[4] + gf[2] * p.lat[7];
        const float z = gf[0] * p.lat[2] + gf[1] * p.lat[5] + gf[2] * p.lat[8];
        const float r2 = x * x + y * y + z * z;
        if (!ok[j] || r2 > sh.rcut2) continue;
        const float ex = expf(-(sh.alpha * r2 + sh.alpha_lo * r2));
        switch (sh.l) {
          case 0: v[0][j] += ex; break;
          case 1: {
            float P[3]; solid_h<1>(x, y, z, P);
#pragma unroll
            for (int m = 0; m < 3; ++m) v[m][j] += P[m] * ex;
          } break;
          case 2: {
            float P[5]; solid_h<2>(x, y, z, P);
#pragma unroll
            for (int m = 0; m < 5; ++m) v[m][j] += P[m] * ex;
          } break;
          default: {
            float P[7]; solid_h<3>(x, y, z, P);
#pragma unroll
            for (int m = 0; m < 7; ++m) v[m][j] += P[m] * ex;
          } break;
        }
      }
    }
    // rows row0 .. row0 + nm - 1 hold m = m0 .. m0 + nm - 1
    for (int r = 0; r < sh.nm; ++r) {
      const int row = sh.row0 + r;
      const float s = p.rowscale[tile * kM + row];
      __align__(16) __half hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float x = 0.f;
#pragma unroll
        for (int m = 0; m < 7; ++m)
          if (m == sh.m0 + r) x = v[m][j];
        x *= s;
        hi[j] = __float2half_rn(x);
        lo[j] = __float2half_rn(x - __half2float(hi[j]));
      }
      const int off = op_off(row, g * 8, kASlice);
      *reinterpret_cast<uint4*>(a_hi + off) = *reinterpret_cast<const uint4*>(hi);
      *reinterpret_cast<uint4*>(a_lo + off) = *reinterpret_cast<const uint4*>(lo);
    }
  }
}

// Images S of the supercell lattice (per atom) within reach of the point tile shifted by -L_l.
__device__ __forceinline__ bool find_images(const TcParams& p, Smem& sm, int ib, int tile,
                                            int rt, const int l3[3], int lane) {
  const float4 c = p.rtiles[rt];
  const float lx = l3[0] * p.lat[0] + l3[1] * p.lat[3] + l3[2] * p.lat[6];
  const float ly = l3[0] * p.lat[1] + l3[1] * p.lat[4] + l3[2] * p.lat[7];
  const float lz = l3[0] * p.lat[2] + l3[1] * p.lat[5] + l3[2] * p.lat[8];
  const int W0 = 2 * p.w[0] + 1, W1 = 2 * p.w[1] + 1, W2 = 2 * p.w[2] + 1;
  const int ncand = W0 * W1 * W2;
  int count = 0;
  bool ok = true;
  for (int a = 0; a < p.natm; ++a) {
    if (lane == 0) sm.img_off[ib][a] = count;
    const float vx = c.x - lx - p.axyz[a][0], vy = c.y - ly - p.axyz[a][1],
                vz = c.z - lz - p.axyz[a][2];
    int s0[3];
    const float u[3] = {vx * p.scinv[0] + vy * p.scinv[3] + vz * p.scinv[6],
                        vx * p.scinv[1] + vy * p.scinv[4] + vz * p.scinv[7],
                        vx * p.scinv[2] + vy * p.scinv[5] + vz * p.scinv[8]};
#pragma unroll
    for (int d = 0; d < 3; ++d) s0[d] = __float2int_rn(u[d]);
    const float lim = p.reach[tile * p.natm + a] + c.w + 0.01f;
    for (int cb = 0; cb < ncand; cb += 32) {
      const int ci = cb + lane;
      bool in = false;
      int s[3] = {0, 0, 0};
      if (ci < ncand) {
        s[0] = s0[0] + ci / (W1 * W2) - p.w[0];
        s[1] = s0[1] + (ci / W2) % W1 - p.w[1];
        s[2] = s0[2] + ci % W2 - p.w[2];
        const float dx = vx - (s[0] * p.sc[0] + s[1] * p.sc[3] + s[2] * p.sc[6]);
        const float dy = vy - (s[0] * p.sc[1] + s[1] * p.sc[4] + s[2] * p.sc[7]);
        const float dz = vz - (s[0] * p.sc[2] + s[1] * p.sc[5] + s[2] * p.sc[8]);
        in = dx * dx + dy * dy + dz * dz <= lim * lim;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      const int pos = count + __popc(bal & ((1u << lane) - 1u));
      if (in) {
        if (pos < kMaxImg) sm.img[ib][pos] = Img{a, s[0], s[1], s[2]};
        else ok = false;
      }
      count += __popc(bal);
    }
  }
  if (count > kMaxImg) count = kMaxImg;
  if (lane == 0) {
    sm.img_off[ib][p.natm] = count;
    sm.nimg[ib] = count;
  }
  return __all_sync(0xffffffffu, ok);
}

__global__ void __launch_bounds__(kThreads, 1) contract_tc_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* stage0 = smraw;   // kStages x (A hi | A lo | B hi | B lo)
  Smem& sm = *reinterpret_cast<Smem*>(smraw + kStages * kStageBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Walk walk{p.active, p.chunk_rt, p.ntile_r, p.nwords, p.cta_chunk0[blockIdx.x],
                  p.cta_chunk0[blockIdx.x + 1]};

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(tc::smem_u32(&sm.full_a[s]), 32 * kAWarps);
      tc::mbar_init(tc::smem_u32(&sm.full_b[s]), 1);
      tc::mbar_init(tc::smem_u32(&sm.empty[s]), 1);
    }
    tc::mbar_init(tc::smem_u32(&sm.acc_full), 1);
    tc::mbar_init(tc::smem_u32(&sm.acc_empty), 32 * kEWarps);
    tc::mbar_init(tc::smem_u32(&sm.done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // pad rows of A are never written by the generators: zero every stage's A once
  for (int e = tid; e < kStages * 2 * kABytes / 16; e += kThreads) {
    const int s = e / (2 * kABytes / 16), o = e % (2 * kABytes / 16);
    reinterpret_cast<uint4*>(stage0 + (size_t)s * kStageBytes)[o] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&sm.tmem_slot), 512);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sm.tmem_slot;
  const uint32_t t_acc = tmem, t_sum = tmem + kN;   // columns [0, 256) and [256, 512)

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long sidx = 0, group = 0;
      bool good = true;
      for (int ci = walk.c0; ci < walk.c1 && good; ++ci) {
        const int4 ch = p.chunks[ci];
        const int nrt = ch.w & 255;
        for (int w = 0; w < p.nwords && good; ++w) {
          unsigned lm = walk.lmask(ch, w);
          while (lm && good) {
            const int l = w * 32 + __ffs(lm) - 1;
            lm &= lm - 1;
            // the epilogue has read the previous group's P_l
            if (group > 0 &&
                !tc::mbar_wait(tc::smem_u32(&sm.acc_empty), (unsigned)((group - 1) & 1),
                               p.wait_ns)) {
              good = false;
              break;
            }
            bool first = true;
            for (int j = 0; j < nrt; ++j) {
              const int rt = p.chunk_rt[ch.z + j];
              if (!walk.on(ch.x, rt, l)) continue;
              const int s = (int)(sidx % kStages);
              const long long u = sidx / kStages;
              if (!tc::mbar_wait(tc::smem_u32(&sm.full_a[s]), (unsigned)(u & 1), p.wait_ns) ||
                  !tc::mbar_wait(tc::smem_u32(&sm.full_b[s]), (unsigned)(u & 1), p.wait_ns)) {
                good = false;
                break;
              }
              tc::tc_fence_after();
              unsigned char* st = stage0 + (size_t)s * kStageBytes;
              const uint32_t a_hi = tc::smem_u32(st), a_lo = a_hi + kABytes;
              const uint32_t b_hi = a_hi + 2 * kABytes, b_lo = b_hi + kBBytes;
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                const uint64_t ah = tc::smem_desc(a_hi + k * kASlice, kLBO, kSBO);
                const uint64_t al = tc::smem_desc(a_lo + k * kASlice, kLBO, kSBO);
                const uint64_t bh = tc::smem_desc(b_hi + k * kBSlice, kLBO, kSBO);
                const uint64_t bl = tc::smem_desc(b_lo + k * kBSlice, kLBO, kSBO);
                tc::mma_f16(t_acc, ah, bh, kIdesc, (first && k == 0) ? 0u : 1u);
                tc::mma_f16(t_acc, ah, bl, kIdesc, 1u);
                tc::mma_f16(t_acc, al, bh, kIdesc, 1u);
              }
              first = false;
              tc::mma_commit(tc::smem_u32(&sm.empty[s]));
              ++sidx;
            }
            if (!good) break;
            tc::mma_commit(tc::smem_u32(&sm.acc_full));   // P_l complete
            ++group;
          }
        }
      }
      if (!good) fail(p.status);
      // every MMA issued has completed before the tensor memory is released
      tc::mma_commit(tc::smem_u32(&sm.done));
      if (!tc::mbar_wait(tc::smem_u32(&sm.done), 0u, p.wait_ns)) fail(p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ B producer
    if (lane == 0) {
      long long sidx = 0;
      bool good = true;
      for (int ci = walk.c0; ci < walk.c1 && good; ++ci) {
        const int4 ch = p.chunks[ci];
        const int nrt = ch.w & 255;
        for (int w = 0; w < p.nwords && good; ++w) {
          unsigned lm = walk.lmask(ch, w);
          while (lm && good) {
            const int l = w * 32 + __ffs(lm) - 1;
            lm &= lm - 1;
            for (int j = 0; j < nrt; ++j) {
              const int rt = p.chunk_rt[ch.z + j];
              if (!walk.on(ch.x, rt, l)) continue;
              const int s = (int)(sidx % kStages);
              const long long u = sidx / kStages;
              if (u > 0 && !tc::mbar_wait(tc::smem_u32(&sm.empty[s]), (unsigned)((u - 1) & 1),
                                          p.wait_ns)) {
                good = false;
                break;
              }
              const uint32_t fb = tc::smem_u32(&sm.full_b[s]);
              tc::mbar_expect_tx(fb, kBBlock);
              const unsigned char* src = p.yh + ((size_t)ch.y * p.ntile_r + rt) * kBBlock;
              unsigned char* dst = stage0 + (size_t)s * kStageBytes + 2 * kABytes;
              tc::bulk_g2s(tc::smem_u32(dst), src, kBBlock, fb);
              ++sidx;
            }
          }
        }
      }
      // no copy may be in flight when the CTA leaves: wait for the last ones issued
      for (long long last = std::max<long long>(0, sidx - kStages); last < sidx; ++last) {
        const int s = (int)(last % kStages);
        if (!tc::mbar_wait(tc::smem_u32(&sm.full_b[s]), (unsigned)((last / kStages) & 1),
                           p.wait_ns))
          good = false;
      }
      if (!good) fail(p.status);
    }
    __syncwarp();
  } else if (warp < 2 + kAWarps) {
    // ------------------------------------------------------------ A generators
    const int t = tid - 64;
    long long sidx = 0;
    bool good = true;
    for (int ci = walk.c0; ci < walk.c1 && good; ++ci) {
      const int4 ch = p.chunks[ci];
      const int nrt = ch.w & 255;
      for (int w = 0; w < p.nwords && good; ++w) {
        unsigned lm = walk.lmask(ch, w);
        while (lm && good) {
          const int l = w * 32 + __ffs(lm) - 1;
          lm &= lm - 1;
          const int l3[3] = {l / (p.D[1] * p.D[2]), (l / p.D[2]) % p.D[1], l % p.D[2]};
          for (int j = 0; j < nrt; ++j) {
            const int rt = p.chunk_rt[ch.z + j];
            if (!walk.on(ch.x, rt, l)) continue;
            const int s = (int)(sidx % kStages);
            const long long u = sidx / kStages;
            const int ib = (int)(sidx & 1);
            if (warp == 2) {
              const bool fits = find_images(p, sm, ib, ch.x, rt, l3, lane);
              // one thread waits for the stage buffer; every generator then follows its verdict
              bool freed = true;
              if (lane == 0 && u > 0)
                freed = tc::mbar_wait(tc::smem_u32(&sm.empty[s]), (unsigned)((u - 1) & 1),
                                      p.wait_ns);
              if (lane == 0) sm.a_ok[ib] = (freed && fits) ? 1 : 0;
            }
            tc::named_sync(1, 32 * kAWarps);
            if (!sm.a_ok[ib]) {
              good = false;
              break;
            }
            // acquire: the phase is complete already, so this returns at once
            if (u > 0) tc::mbar_try_wait(tc::smem_u32(&sm.empty[s]), (unsigned)((u - 1) & 1));
            unsigned char* st = stage0 + (size_t)s * kStageBytes;
            gen_a(p, sm, ib, ch.x, rt, l3, st, st + kABytes, t);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(tc::smem_u32(&sm.full_a[s]));
            ++sidx;
          }
        }
      }
    }
    if (!good && t == 0) fail(p.status);
  } else {
    // ------------------------------------------------------------ epilogue
    const int et = tid - 32 * (2 + kAWarps);          // 0..127
    const int quarter = warp & 3;                      // TMEM lanes 32 quarter ..
    const int row = 32 * quarter + lane;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    long long group = 0;
    bool good = true;
    for (int ci = walk.c0; ci < walk.c1 && good; ++ci) {
      const int4 ch = p.chunks[ci];
      const int tile = ch.x, ct = ch.y;
      const int flags = ch.w;
      // per-column reciprocal scales of this chunk's columns
      {
        const int c = ct * kNC + et;
        double inv = 0.0;
        if (c < p.ncol) {
          const float mx = __uint_as_float(p.colmax[c]);
          int e2 = 0;
          if (mx > 0.f) frexpf(mx, &e2);
          inv = ldexp(1.0, e2 - 13);
        }
        tc::named_sync(2, 32 * kEWarps);   // previous chunk's readers of colinv are done
        sm.colinv[et] = inv;
      }
      bool first_group = true;
      // how many l groups this chunk has (the last one may end in FP64 atomics)
      int ngroups = 0;
      for (int w = 0; w < p.nwords; ++w) ngroups += __popc(walk.lmask(ch, w));
      int gi = 0;
      for (int w = 0; w < p.nwords && good; ++w) {
        unsigned lm = walk.lmask(ch, w);
        while (lm && good) {
          const int l = w * 32 + __ffs(lm) - 1;
          lm &= lm - 1;
          // phases e^{-ik.L_l} of the chunk's columns
          {
            const int c = ct * kNC + et;
            float2 ph = make_float2(0.f, 0.f);
            if (c < p.ncol) {
              const int k = c / p.nocc;
              const int l3[3] = {l / (p.D[1] * p.D[2]), (l / p.D[2]) % p.D[1], l % p.D[2]};
              const int Dc = p.D[0] * p.D[1] * p.D[2];
              long long num = 0;
              for (int d = 0; d < 3; ++d)
                num += (long long)p.kint[3 * k + d] * l3[d] * (Dc / p.D[d]);
              const float2 v = dev::cis_frac<float>(num, Dc, -1);
              ph = v;
            }
            tc::named_sync(2, 32 * kEWarps);
            sm.phase[et] = ph;
            if (et == 0)
              sm.e_ok = tc::mbar_wait(tc::smem_u32(&sm.acc_full), (unsigned)(group & 1),
                                      p.wait_ns) ? 1 : 0;
            tc::named_sync(2, 32 * kEWarps);
          }
          if (!sm.e_ok) {
            good = false;
            break;
          }
          tc::mbar_try_wait(tc::smem_u32(&sm.acc_full), (unsigned)(group & 1));   // acquire
          tc::tc_fence_after();
          const bool init = first_group && (flags & kFirstSum);
          const bool last = (gi == ngroups - 1);
          const bool to_global = last && (flags & kToGlobal);
          const int mu = p.perm[tile * kM + row];
          const double rf = (mu >= 0) ? p.rowf[tile * kM + row] * p.scale : 0.0;
#pragma unroll 1
          for (int q = 0; q < kN / 16; ++q) {
            uint32_t va[16], vs[16];
            tc::tmem_ld16(t_acc + lane_off + q * 16, va);
            if (!init) tc::tmem_ld16(t_sum + lane_off + q * 16, vs);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float2 ph = sm.phase[q * 8 + j];
              const float ar = __uint_as_float(va[2 * j]), ai = __uint_as_float(va[2 * j + 1]);
              float sr = ph.x * ar - ph.y * ai, si = ph.x * ai + ph.y * ar;
              if (!init) {
                sr += __uint_as_float(vs[2 * j]);
                si += __uint_as_float(vs[2 * j + 1]);
              }
              vs[2 * j] = __float_as_uint(sr);
              vs[2 * j + 1] = __float_as_uint(si);
            }
            if (to_global) {
              if (mu >= 0) {
#pragma unroll 1
                for (int j = 0; j < 8; ++j) {
                  const int cl = q * 8 + j, c = ct * kNC + cl;
                  if (c >= p.ncol) break;
                  const int k = c / p.nocc, i = c - k * p.nocc;
                  const double f = rf * sm.colinv[cl];
                  double* dst = reinterpret_cast<double*>(
                      p.kc + ((size_t)k * p.nao + mu) * p.nocc + i);
                  atomicAdd(dst, f * (double)__uint_as_float(vs[2 * j]));
                  atomicAdd(dst + 1, f * (double)__uint_as_float(vs[2 * j + 1]));
                }
              }
            } else {
              tc::tmem_st16(t_sum + lane_off + q * 16, vs);
            }
          }
          tc::tmem_wait_st();
          tc::tc_fence_before();
          tc::mbar_arrive(tc::smem_u32(&sm.acc_empty));
          ++group;
          ++gi;
          first_group = false;
        }
      }
    }
    if (!good && et == 0) fail(p.status);
  }

  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// max over the points of |Re| + |Im| of every (k, i) field of Y, as float bits
__global__ void colmax_kernel(const float2* __restrict__ Y, unsigned* __restrict__ colmax,
                              long long ng, long long fs) {
  const int c = blockIdx.x;
  float m = 0.f;
  for (long long q = threadIdx.x; q < ng; q += blockDim.x) {
    const float2 v = Y[(size_t)c * fs + q];
    m = fmaxf(m, fabsf(v.x) + fabsf(v.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) colmax[c] = __float_as_uint(m);
  }
}

// Y -> FP16 hi/lo B blocks: block (ct, rt) row 2c + {0: Re, 1: Im} of column c of the tile,
// K index = point q - 32 rt; scaled by 2^(13 - e) with e the column's max exponent.
__global__ void convert_y_kernel(const float2* __restrict__ Y, const unsigned* __restrict__ colmax,
                                 unsigned char* __restrict__ yh, int ncol, int n_ct, int ntile_r,
                                 long long ng, long long fs) {
  const long long total = (long long)n_ct * kNC * ntile_r * 4;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(e & 3);
    long long r = e >> 2;
    const int cl = (int)(r % kNC);
    r /= kNC;
    const int rt = (int)(r % ntile_r);
    const int ct = (int)(r / ntile_r);
    const int c = ct * kNC + cl;
    __align__(16) __half rh[8], rl[8], ih[8], il[8];
    float s = 0.f;
    if (c < ncol) {
      const float mx = __uint_as_float(colmax[c]);
      int e2 = 0;
      if (mx > 0.f) frexpf(mx, &e2);
      s = ldexpf(1.f, 13 - e2);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long q = (long long)rt * kKP + g * 8 + j;
      float2 v = make_float2(0.f, 0.f);
      if (c < ncol && q < ng) v = Y[(size_t)c * fs + q];
      const float xr = v.x * s, xi = v.y * s;
      rh[j] = __float2half_rn(xr);
      rl[j] = __float2half_rn(xr - __half2float(rh[j]));
      ih[j] = __float2half_rn(xi);
      il[j] = __float2half_rn(xi - __half2float(ih[j]));
    }
    unsigned char* blk = yh + ((size_t)ct * ntile_r + rt) * kBBlock;
    const int o_re = op_off(2 * cl, g * 8, kBSlice), o_im = op_off(2 * cl + 1, g * 8, kBSlice);
    *reinterpret_cast<uint4*>(blk + o_re) = *reinterpret_cast<const uint4*>(rh);
    *reinterpret_cast<uint4*>(blk + o_im) = *reinterpret_cast<const uint4*>(ih);
    *reinterpret_cast<uint4*>(blk + kBBytes + o_re) = *reinterpret_cast<const uint4*>(rl);
    *reinterpret_cast<uint4*>(blk + kBBytes + o_im) = *reinterpret_cast<const uint4*>(il);
  }
}

}  // namespace tcc

// ------------------------------------------------------------------ host planning

namespace {

void inv3x3(const double a[3][3], double inv[3][3]) {
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

// Upper bound of |P_lm(d)| e^{-alpha d^2} over d: c_l (l / (2 alpha e))^{l/2}.
double shell_peak(int l, double alpha) {
  static const double cl[4] = {1.0, 1.0, 2.0, 4.0};
  if (l == 0) return 1.0;
  return cl[l] * std::pow(l / (2.0 * alpha * std::exp(1.0)), 0.5 * l);
}

template <typename X>
cudaError_t put(X** d, const std::vector<X>& v, size_t* tot) {
  *tot += v.size() * sizeof(X);
  cudaError_t e = device_malloc((void**)d, std::max<size_t>(1, v.size()) * sizeof(X));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(*d, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice);
}

}  // namespace

struct TcPlan {
  tcc::TcParams prm;
  int ncta = 0;
  size_t smem = 0;
  std::vector<void*> bufs;
  unsigned char* yh = nullptr;
  unsigned* colmax = nullptr;
};

void tc_plan_free(TcPlan* t) {
  if (!t) return;
  for (void* b : t->bufs)
    if (b) cudaFree(b);
  delete t;
}

int tc_plan_create(Plan* p, const std::vector<ShellDev>& sh, const double* xyz,
                   const std::vector<double>& rcut, size_t* total) {
  using namespace tcc;
  if (p->natm > kMaxTcAtoms) return OCCRI_EUNSUPPORTED;
  const int NL = p->D[0] * p->D[1] * p->D[2];
  if (NL > 32 * 16) return OCCRI_EUNSUPPORTED;
  const int N = p->N[0];
  const long long ng = p->ng;
  TcPlan* t = new TcPlan();
  TcParams& q = t->prm;
  std::memset(&q, 0, sizeof(q));
  q.nk = p->nk; q.nao = p->nao; q.nocc = p->nocc; q.natm = p->natm; q.N = N; q.ng = ng;
  q.ncol = p->nk * p->nocc;
  q.n_ct = (q.ncol + kNC - 1) / kNC;
  q.ntile_r = (int)((ng + kKP - 1) / kKP);
  q.nl = NL;
  q.nwords = (NL + 31) / 32;
  for (int d = 0; d < 3; ++d) q.D[d] = p->D[d];
  double sc[3][3], scinv[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      sc[i][j] = p->lat[i][j] * p->D[i];
      q.lat[3 * i + j] = (float)p->lat[i][j];
      q.sc[3 * i + j] = (float)sc[i][j];
    }
  inv3x3(sc, scinv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q.scinv[3 * i + j] = (float)scinv[i][j];
  double linv[3][3];
  inv3x3(p->lat, linv);
  for (int a = 0; a < p->natm; ++a) {
    for (int d = 0; d < 3; ++d) {
      const double f = xyz[3 * a] * linv[0][d] + xyz[3 * a + 1] * linv[1][d] + xyz[3 * a + 2] * linv[2][d];
      const double fn = f * N;
      const double ai = std::nearbyint(fn);
      const double rem = fn - ai;
      q.aint[a][d] = (int)ai;
      q.arem_hi[a][d] = (float)rem;
      q.arem_lo[a][d] = (float)(rem - (double)(float)rem);
      q.axyz[a][d] = (float)xyz[3 * a + d];
    }
  }

  // AO rows sorted by screening radius (descending), shells kept whole
  std::vector<int> order(p->nshell);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rcut[x] > rcut[y]; });
  const int ntile = (p->nao + kM - 1) / kM;
  std::vector<TcShell> shells;
  std::vector<int> tile_shell0(ntile + 1, 0);
  std::vector<float> rowscale((size_t)ntile * kM, 1.f), reach((size_t)ntile * p->natm, 0.f);
  std::vector<double> rowf((size_t)ntile * kM, 0.0);
  std::vector<int> perm((size_t)ntile * kM, -1);
  int row = 0;
  int cur_tile = 0;
  for (int idx = 0; idx < p->nshell; ++idx) {
    const ShellDev& s = sh[order[idx]];
    const int nm = 2 * s.l + 1;
    // rows of this shell, possibly split across two tiles
    int m = 0;
    double bound = shell_peak(s.l, s.alpha);
    // periodic images can add up where the supercell is small: allow for their count
    while (m < nm) {
      const int tile = row / kM, r0 = row % kM;
      while (cur_tile < tile) tile_shell0[++cur_tile] = (int)shells.size();
      const int take = std::min(nm - m, kM - r0);
      TcShell e;
      e.alpha = s.alpha_f; e.alpha_lo = s.alpha_lo; e.rcut2 = s.rcut2_f;
      e.atom = s.atom; e.l = s.l; e.row0 = r0; e.m0 = m; e.nm = take;
      shells.push_back(e);
      for (int j = 0; j < take; ++j) {
        const int gr = tile * kM + r0 + j;
        perm[gr] = s.ao + m + j;
        rowf[gr] = s.norm[m + j];
        rowscale[gr] = (float)bound;   // replaced below by a power of two
      }
      float& rr = reach[(size_t)tile * p->natm + s.atom];
      rr = std::max(rr, (float)rcut[order[idx]]);
      m += take;
      row += take;
    }
  }
  while (cur_tile < ntile) tile_shell0[++cur_tile] = (int)shells.size();

  // point tiles: centre and radius
  std::vector<float4> rtiles(q.ntile_r);
  std::vector<double> pts;
  for (int rt = 0; rt < q.ntile_r; ++rt) {
    double c[3] = {0, 0, 0};
    int cnt = 0;
    pts.clear();
    for (int j = 0; j < kKP; ++j) {
      const long long qq = (long long)rt * kKP + j;
      if (qq >= ng) break;
      const int n2 = (int)(qq % N), tq = (int)(qq / N), n1 = tq % N, n3 = tq / N;
      const double f[3] = {(double)n1 / N, (double)n2 / N, (double)n3 / N};
      double x[3];
      for (int d = 0; d < 3; ++d)
        x[d] = f[0] * p->lat[0][d] + f[1] * p->lat[1][d] + f[2] * p->lat[2][d];
      for (int d = 0; d < 3; ++d) { c[d] += x[d]; pts.push_back(x[d]); }
      ++cnt;
    }
    for (int d = 0; d < 3; ++d) c[d] /= std::max(cnt, 1);
    double rad = 0;
    for (int j = 0; j < cnt; ++j) {
      double e2 = 0;
      for (int d = 0; d < 3; ++d) e2 += (pts[3 * j + d] - c[d]) * (pts[3 * j + d] - c[d]);
      rad = std::max(rad, std::sqrt(e2));
    }
    rtiles[rt] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)(rad + 1e-6));
  }

  // image search widths and the activity of each (tile, point tile, l)
  double rmax = 0;
  for (float r : reach) rmax = std::max(rmax, (double)r);
  double rad_max = 0;
  for (const float4& r : rtiles) rad_max = std::max(rad_max, (double)r.w);
  for (int d = 0; d < 3; ++d) {
    const double bn = std::sqrt(scinv[0][d] * scinv[0][d] + scinv[1][d] * scinv[1][d] +
                                scinv[2][d] * scinv[2][d]);
    // s0 = round(u) is within 1/2 of the fractional position, so every image within r
    // lies within floor(r |b_d| + 1/2) of s0 along axis d
    q.w[d] = (int)std::floor((rmax + rad_max + 0.02) * bn + 0.5);
  }
  std::vector<unsigned> active((size_t)ntile * q.ntile_r * q.nwords, 0u);
  std::vector<long long> cost_tile_rt((size_t)ntile * q.ntile_r, 0);
  int max_img = 0;
  {
    std::vector<double> dmin(p->natm);
    std::vector<int> nimg_a(p->natm);
    for (int rt = 0; rt < q.ntile_r; ++rt) {
      const float4 c = rtiles[rt];
      for (int l = 0; l < NL; ++l) {
        const int l3[3] = {l / (p->D[1] * p->D[2]), (l / p->D[2]) % p->D[1], l % p->D[2]};
        double L[3];
        for (int d = 0; d < 3; ++d)
          L[d] = l3[0] * p->lat[0][d] + l3[1] * p->lat[1][d] + l3[2] * p->lat[2][d];
        int tot_img = 0;
        for (int a = 0; a < p->natm; ++a) {
          const double v[3] = {c.x - L[0] - xyz[3 * a], c.y - L[1] - xyz[3 * a + 1],
                               c.z - L[2] - xyz[3 * a + 2]};
          int s0[3];
          for (int d = 0; d < 3; ++d)
            s0[d] = (int)std::nearbyint(v[0] * scinv[0][d] + v[1] * scinv[1][d] + v[2] * scinv[2][d]);
          double best = 1e300;
          int cnt = 0;
          const double lim0 = reach[a] + c.w + 0.01;   // tile 0 holds the largest radii
          for (int i0 = -q.w[0]; i0 <= q.w[0]; ++i0)
            for (int i1 = -q.w[1]; i1 <= q.w[1]; ++i1)
              for (int i2 = -q.w[2]; i2 <= q.w[2]; ++i2) {
                const int s[3] = {s0[0] + i0, s0[1] + i1, s0[2] + i2};
                double e2 = 0;
                for (int d = 0; d < 3; ++d) {
                  const double x = v[d] - (s[0] * sc[0][d] + s[1] * sc[1][d] + s[2] * sc[2][d]);
                  e2 += x * x;
                }
                const double dist = std::sqrt(e2);
                best = std::min(best, dist);
                if (dist <= lim0) ++cnt;
              }
          dmin[a] = best;
          tot_img += cnt;
        }
        max_img = std::max(max_img, tot_img);
        for (int tl = 0; tl < ntile; ++tl) {
          bool on = false;
          for (int a = 0; a < p->natm && !on; ++a)
            on = dmin[a] <= reach[(size_t)tl * p->natm + a] + c.w;
          if (on) {
            active[((size_t)tl * q.ntile_r + rt) * q.nwords + (l >> 5)] |= 1u << (l & 31);
            ++cost_tile_rt[(size_t)tl * q.ntile_r + rt];
          }
        }
      }
    }
  }
  if (max_img > kMaxImg) {
    delete t;
    return OCCRI_EUNSUPPORTED;
  }
  // row scales: powers of two that keep |A| < 2^13, allowing for overlapping images
  for (size_t gr = 0; gr < rowscale.size(); ++gr) {
    if (perm[gr] < 0) { rowscale[gr] = 1.f; rowf[gr] = 0.0; continue; }
    const double bound = (double)rowscale[gr] * std::max(1, max_img);
    int e2 = 0;
    std::frexp(bound, &e2);
    rowscale[gr] = std::ldexp(1.f, 13 - e2);
    rowf[gr] = rowf[gr] / (double)rowscale[gr];
  }

  // work chunks: per (tile, column tile), the active point tiles in runs of kChunkTiles;
  // CTAs take contiguous runs of chunks of about equal cost
  struct Chunk { int tile, ct, off, n; long long cost; };
  std::vector<Chunk> chunks;
  std::vector<int> chunk_rt;
  for (int tl = 0; tl < ntile; ++tl)
    for (int ct = 0; ct < q.n_ct; ++ct) {
      Chunk cur{tl, ct, (int)chunk_rt.size(), 0, 0};
      std::vector<unsigned> uni(q.nwords, 0u);
      auto close = [&]() {
        if (cur.n == 0) return;
        long long groups = 0;
        for (unsigned u : uni) groups += __builtin_popcount(u);
        cur.cost += groups * 2;      // epilogue of each P_l, in stage units
        chunks.push_back(cur);
        cur = Chunk{tl, ct, (int)chunk_rt.size(), 0, 0};
        std::fill(uni.begin(), uni.end(), 0u);
      };
      for (int rt = 0; rt < q.ntile_r; ++rt) {
        const long long c = cost_tile_rt[(size_t)tl * q.ntile_r + rt];
        if (c == 0) continue;
        chunk_rt.push_back(rt);
        ++cur.n;
        cur.cost += c;
        for (int w = 0; w < q.nwords; ++w)
          uni[w] |= active[((size_t)tl * q.ntile_r + rt) * q.nwords + w];
        if (cur.n == kChunkTiles) close();
      }
      close();
    }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  long long total_cost = 0;
  for (const Chunk& c : chunks) total_cost += c.cost;
  const int ncta = std::max(1, std::min<int>(nsm > 0 ? nsm : 1, (int)chunks.size()));
  std::vector<int> cta_chunk0(ncta + 1, (int)chunks.size());
  {
    long long acc = 0;
    int b = 0;
    cta_chunk0[0] = 0;
    for (size_t i = 0; i < chunks.size(); ++i) {
      while (b + 1 < ncta && acc >= (long long)((double)total_cost * (b + 1) / ncta)) {
        cta_chunk0[++b] = (int)i;
      }
      acc += chunks[i].cost;
    }
    while (b + 1 < ncta) cta_chunk0[++b] = (int)chunks.size();
    cta_chunk0[ncta] = (int)chunks.size();
  }
  std::vector<int4> ch4(chunks.size());
  for (int b = 0; b < ncta; ++b) {
    int since = 0;
    for (int i = cta_chunk0[b]; i < cta_chunk0[b + 1]; ++i) {
      const Chunk& c = chunks[i];
      const bool first = (i == cta_chunk0[b]) || since == 0 ||
                         chunks[i - 1].tile != c.tile || chunks[i - 1].ct != c.ct;
      if (first) since = 0;
      ++since;
      const bool last = (i + 1 == cta_chunk0[b + 1]) || chunks[i + 1].tile != c.tile ||
                        chunks[i + 1].ct != c.ct || since == kFlushChunks;
      if (last) since = 0;
      ch4[i] = make_int4(c.tile, c.ct, c.off, c.n | (first ? kFirstSum : 0) | (last ? kToGlobal : 0));
    }
  }
  t->ncta = ncta;

  // device copies
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess && x != cudaSuccess) e = x; };
  TcShell* d_sh = nullptr; int* d_ts = nullptr; float* d_rs = nullptr; double* d_rf = nullptr;
  int* d_perm = nullptr; float* d_reach = nullptr; float4* d_rt = nullptr; unsigned* d_act = nullptr;
  int4* d_ch = nullptr; int* d_crt = nullptr; int* d_c0 = nullptr;
  chk(put(&d_sh, shells, total)); t->bufs.push_back(d_sh);
  chk(put(&d_ts, tile_shell0, total)); t->bufs.push_back(d_ts);
  chk(put(&d_rs, rowscale, total)); t->bufs.push_back(d_rs);
  chk(put(&d_rf, rowf, total)); t->bufs.push_back(d_rf);
  chk(put(&d_perm, perm, total)); t->bufs.push_back(d_perm);
  chk(put(&d_reach, reach, total)); t->bufs.push_back(d_reach);
  chk(put(&d_rt, rtiles, total)); t->bufs.push_back(d_rt);
  chk(put(&d_act, active, total)); t->bufs.push_back(d_act);
  chk(put(&d_ch, ch4, total)); t->bufs.push_back(d_ch);
  chk(put(&d_crt, chunk_rt, total)); t->bufs.push_back(d_crt);
  chk(put(&d_c0, cta_chunk0, total)); t->bufs.push_back(d_c0);
  {
    void* b = nullptr;
    const size_t yb = (size_t)q.n_ct * q.ntile_r * kBBlock;
    *total += yb;
    chk(device_malloc(&b, yb)); t->bufs.push_back(b); t->yh = (unsigned char*)b;
    b = nullptr;
    *total += (size_t)q.ncol * 4;
    chk(device_malloc(&b, (size_t)q.ncol * 4)); t->bufs.push_back(b); t->colmax = (unsigned*)b;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    tc_plan_free(t);
    return e == cudaErrorMemoryAllocation ? OCCRI_ENOMEM : OCCRI_ECUDA;
  }
  q.yh = t->yh; q.shells = d_sh; q.tile_shell0 = d_ts; q.rowscale = d_rs; q.rowf = d_rf;
  q.perm = d_perm; q.reach = d_reach; q.rtiles = d_rt; q.active = d_act; q.chunks = d_ch;
  q.chunk_rt = d_crt; q.cta_chunk0 = d_c0; q.kint = p->kint; q.colmax = t->colmax;
  t->smem = (size_t)kStages * kStageBytes + sizeof(Smem);
  p->tc = t;
  return OCCRI_OK;
}

cudaError_t launch_contract_tc(const Plan& p, cudaStream_t s) {
  using namespace tcc;
  TcPlan* t = p.tc;
  TcParams q = t->prm;
  q.kc = p.kc;
  q.scale = -p.omega_cell * 4.0 * 3.14159265358979323846 /
            ((double)p.nk * (double)p.ng * (double)p.ng);
  q.status = p.status;
  q.wait_ns = p.wait_ns;
  const float2* Y = (const float2*)p.Y;
  colmax_kernel<<<q.ncol, 256, 0, s>>>(Y, t->colmax, p.ng, p.fs);
  convert_y_kernel<<<8 * 152, 256, 0, s>>>(Y, t->colmax, t->yh, q.ncol, q.n_ct, q.ntile_r, p.ng,
                                           p.fs);
  static DeviceCache attr;
  attr.get(p.device, [&] {
    cudaFuncSetAttribute(contract_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)t->smem);
    return 1;
  });
  contract_tc_kernel<<<t->ncta, kThreads, t->smem, s>>>(q);
  return cudaGetLastError();
}

}  // namespace occri
