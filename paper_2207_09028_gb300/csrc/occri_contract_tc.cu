// occri_contract_tc.cu -- step (e), K_{mu i}(k) = -(Omega/(N_k N_g)) sum_r conj(chi_{mu k}(r))
// Y_ik(r) (Eq. occrik, the last step of Algorithm 3), as one dense GEMM on the tensor cores.
//
// Formulation. Let D_d be the k denominators (kappa_{k,d} = kint_d / D_d), L_l = sum_d l_d a_d
// for l_d in [0, D_d) the cell offsets of the D1 x D2 x D3 supercell, and
// Phi_mu(x) = sum_S phi_mu(x - A_mu - S) the AO periodised over the supercell lattice S
// (e^{ik.S} = 1 there). Then conj(chi_{mu k}(r)) = sum_l e^{-ik.L_l} Phi_mu(r - L_l), and
//   K_{mu i}(k) = scale sum_l e^{-ik.L_l} P_l[mu, (k,i)],   P_l = sum_r Phi_mu(r - L_l) Y_ik(r).
// P_l is a real-by-complex GEMM: rows mu (128 AOs per tile, sorted by screening radius so that
// tight AOs share tiles), columns the (Re, Im) of 96 (k, i) pairs (N = 192), reduction over the
// cell's grid points. A stage is one tile of 32 grid points r at one offset l: A = Phi at the
// points r - L_l, B = Y at the points r. Both operands are split hi + lo in FP16 (power-of-two
// scalings per row and column), and three FP16 MMAs (hi.hi + hi.lo + lo.hi) with FP32
// accumulation give FP32-level products. Stages where no AO of the tile reaches r - L_l are
// skipped: tight AOs are sparse here.
//
// Kernels of one contraction:
//   colmax_kernel, convert_y_kernel  Y -> FP16 hi/lo B blocks (tensor-core layout), once
//   gen_blocks_kernel               the A blocks of a slab of stages (Phi generated from the
//                                   Gaussians; each block serves every column tile)
//   contract_tc_kernel              the GEMM over the slab's stages: one producer thread copies
//                                   each stage's A and B blocks with the bulk-copy engine, one
//                                   thread issues the MMAs into one of two tensor-memory
//                                   accumulators, and 12 epilogue warps take every stage's
//                                   product out at once (times the phases e^{-ik.L_l}) into
//                                   FP32 running sums held in registers, which go to K_{mu i}
//                                   by FP64 atomics. Each product leaves tensor memory after
//                                   one stage because the tensor cores' FP32 accumulation was
//                                   measured to bias long sums by ~1e-6 relative.
// Every mbarrier wait is bounded by the plan's wait limit; on timeout the kernel records
// OCCRI_ETIMEOUT, each role stops issuing and no copy is left in flight.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fft_reg.cuh"
#include "occri_device.cuh"
#include "occri_internal.h"
#include "occri_tc.cuh"

namespace occri {
namespace tcc {

namespace pk = fft::pk;
using pk::u64;

constexpr int kM = 128;             // AO rows per tile (TMEM lanes)
constexpr int kNC = 96;             // complex (k, i) columns per tile (a multiple of 32)
constexpr int kN = 2 * kNC;         // real columns (Re, Im)
constexpr int kKP = 32;             // grid points per stage (MMA K, two slices of 16)
constexpr int kStages = 4;
constexpr int kFlushTiles = 16;     // point tiles summed in FP32 before the FP64 atomics
constexpr int kSlabBlocks = 1 << 18;     // A blocks generated at a time (4 GiB)
constexpr int kMaxImg = 128;        // supercell images of one stage, all atoms
constexpr int kEWarps = kNC / 8;    // epilogue: per 32 complex columns one warp per lane quarter
constexpr int kEThreads = 32 * kEWarps;
constexpr int kThreads = 64 + kEThreads;     // + MMA warp and bulk-copy warp
constexpr int kGenThreads = 256;             // threads of the block-generation kernel
constexpr int kASlice = kM * 16 * 2;          // bytes of one K slice of A (hi or lo)
constexpr int kBSlice = kN * 16 * 2;          // bytes of one K slice of B
constexpr int kABytes = 2 * kASlice;          // A hi (or lo) of a stage
constexpr int kBBytes = 2 * kBSlice;          // B hi (or lo) of a stage
constexpr int kABlock = 2 * kABytes;          // one generated A block (hi then lo): 16 KB
constexpr int kBBlock = 2 * kBBytes;          // one converted Y block (hi then lo): 32 KB
constexpr int kStageBytes = kABlock + kBBlock;
constexpr uint32_t kIdesc = tc::idesc_f16_f32(kM, kN);
constexpr int kPhaseRow = 3 * kNC;      // floats of the phases of one (column tile, l)
constexpr int kAccCols = 256;           // tensor-memory columns between the two accumulators
static_assert(kNC % 32 == 0 && kN <= kAccCols, "column tile");
// Descriptor strides of the no-swizzle K-major layout used below: inside one 16-wide K slice,
// an 8-row group holds its two 8-column core matrices at +0 and +128 bytes and groups follow
// every 256 bytes.
constexpr uint32_t kLBO = 128, kSBO = 256;

// byte offset of element (row, k) inside one operand of a stage (slices of 16 along K)
__host__ __device__ constexpr int op_off(int row, int k, int slice_bytes) {
  return (k >> 4) * slice_bytes + (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 +
         (k & 7) * 2;
}

struct TcShell {        // the rows of one shell inside a tile
  float alpha, alpha_lo, rcut2;
  int atom, l, row0, m0, nm, exact;   // exact: Gaussian argument in double-float
};

constexpr int kMaxTiles = 4;             // AO tiles of a plan (nao <= 512)
constexpr int kMaxEntries = 192;         // shell entries of all tiles

// A stage of the GEMM: x = A slot in the slab | l << 22; y = point tile | column tile << 16
// | flags << 24 | AO tile << 27 (kFirstSum: the running sums start here; kToGlobal: they go
// to K_{mu i} after this stage).
// kChain: this stage and the next one (same column tile and offset l, the next point tile)
// share one accumulator, and the epilogue takes their sum out once.
enum { kFirstSum = 1, kToGlobal = 2, kChain = 4 };

struct TcParams {
  int nk, nao, nocc, natm, N, ncol, n_ct, ntile_r, nl, ntile, nentries;
  int D[3], w[3];
  long long ng;
  const unsigned char* yh;       // converted Y blocks [ct][rt][32 KB]
  unsigned char* ablk;           // generated A blocks of the current slab [slot][16 KB]
  const uint2* blocks;           // the slab's A blocks: (rt | l << 16, tile)
  int nblocks;
  const TcShell* shells;         // entries of all tiles, tile by tile
  const int* tile_shell0;        // entries of tile t: [tile_shell0[t], tile_shell0[t+1])
  const float* rowscale;         // [tile*128 + row]
  const double* rowf;            // N_mu / rowscale, 0 on pad rows
  const int* perm;               // tile row -> AO (or -1)
  const float* reach;            // [tile][natm] largest screening radius of the tile's shells
  const float4* rtiles;          // [ntile_r] centre (x, y, z) and radius of the point tile
  const float* phase;            // [ct][nl][3][128] cos, sin, -sin of the phase e^{-ik.L_l}
                                 // of the tile's columns (0 past ncol)
  const uint2* stages;           // the slab's stages, CTA by CTA
  const long long* cta_stage0;   // stages of CTA b: [cta_stage0[b], cta_stage0[b+1])
  const double* colf;            // [ncol] 2^(e - 13): undoes the column scaling of Y (e as below)
  double2* kc;
  double scale;
  float lat[9], sc[9], scinv[9]; // rows a_d; supercell rows D_d a_d; cart -> supercell frac
  float sclo[9];                 // supercell rows, the remainder sc - (double) sc_f
  const float* pts;              // [ng][6] grid point r_q: x, y, z (hi), x, y, z (lo)
  const float* tbase;            // [natm][nl][6] L_l + A_a (hi, lo)
  int* status;
  long long wait_ns;
};

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

// One supercell image of one atom for a block: T = L_l + S + A_atom (cartesian, hi + lo).
struct Img { float th[3], tl[3]; };

// The tables of one A block: its grid points and the supercell images in reach.
struct StageTab {
  int ok;                          // 0: the images did not fit
  int img_off[kMaxTcAtoms + 1];    // images of atom a: [img_off[a], img_off[a+1])
  float pts[kKP][6];               // the block's grid points r (x, y, z hi; x, y, z lo)
  Img img[kMaxImg];
};

// FP16 hi/lo split of two values, packed as two 32-bit words (x0 in the low half)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 back = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - back.x, x1 - back.y);
  memcpy(&hi, &h, 4);
  memcpy(&lo, &l, 4);
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The rows of one shell entry (angular momentum L) at 4 points of the block.
template <int L>
__device__ __forceinline__ void gen_item(const StageTab& tb, const TcShell& sh, int g,
                                         const float* rowscale, unsigned char* a_hi,
                                         unsigned char* a_lo) {
  constexpr int NM = 2 * L + 1;
  float v[NM][4];
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[m][j] = 0.f;
  const int i0 = tb.img_off[sh.atom], i1 = tb.img_off[sh.atom + 1];
  for (int im = i0; im < i1; ++im) {
    const Img T = tb.img[im];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float* r = tb.pts[g * 4 + j];
      float c[3], cl[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        // r - T as an unevaluated hi + lo sum: exact difference of the hi parts near the atom
        float se, ee;
        two_sum_f(r[d], -T.th[d], se, ee);
        c[d] = se;
        cl[d] = ee + (r[3 + d] - T.tl[d]);
      }
      const float x = c[0] + cl[0], y = c[1] + cl[1], z = c[2] + cl[2];
      float r2, ex;
      if (sh.exact) {
        // r^2 and alpha r^2 as hi + lo pairs (FMA two-products), e^{-a} = e^{-ah} (1 - al)
        float ph[3], pl[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          ph[d] = c[d] * c[d];
          pl[d] = fmaf(c[d], c[d], -ph[d]) + 2.f * c[d] * cl[d];
        }
        float s1, e1, s2, e2;
        two_sum_f(ph[0], ph[1], s1, e1);
        two_sum_f(s1, ph[2], s2, e2);
        const float rl = (e1 + e2) + (pl[0] + pl[1] + pl[2]);
        r2 = s2;
        const float ah = sh.alpha * s2;
        const float al = fmaf(sh.alpha, s2, -ah) + sh.alpha * rl + sh.alpha_lo * s2;
        ex = expf(-ah) * (1.f - al);
      } else {
        r2 = x * x + y * y + z * z;
        ex = expf(-(sh.alpha * r2 + sh.alpha_lo * r2));
      }
      // points past the grid carry a NaN coordinate and fail the test, like those out of reach
      if (!(r2 <= sh.rcut2)) ex = 0.f;
      float P[NM];
      solid_h<L>(x, y, z, P);
#pragma unroll
      for (int m = 0; m < NM; ++m) v[m][j] += (ex != 0.f) ? P[m] * ex : 0.f;
    }
  }
  // rows row0 .. row0 + nm - 1 hold m = m0 .. m0 + nm - 1
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    if (m < sh.m0 || m >= sh.m0 + sh.nm) continue;
    const int row = sh.row0 + (m - sh.m0);
    const float sc = rowscale[row];
    uint2 hi, lo;
    split2(v[m][0] * sc, v[m][1] * sc, hi.x, lo.x);
    split2(v[m][2] * sc, v[m][3] * sc, hi.y, lo.y);
    const int off = op_off(row, g * 4, kASlice);
    *reinterpret_cast<uint2*>(a_hi + off) = hi;
    *reinterpret_cast<uint2*>(a_lo + off) = lo;
  }
}

// The block's table of grid points (hi/lo; NaN past the grid) and, per atom, the images
// T = L_l + A + S of the supercell lattice within reach of the point tile (hi + lo, from the
// plan's table of L_l + A and error-free products S_d x (supercell row d)). One warp.
// tb.ok = 0 if the images do not fit the table.
__device__ __forceinline__ void block_tables(const TcParams& p, StageTab& tb, int tile, int rt,
                                             int l, int lane) {
  const float4 c = p.rtiles[rt];
  {
    const long long q = (long long)rt * kKP + lane;
    float* o = tb.pts[lane];
    if (q < p.ng) {
      const float2* src = reinterpret_cast<const float2*>(p.pts + 6 * (size_t)q);
      const float2 a0 = src[0], a1 = src[1], a2 = src[2];
      o[0] = a0.x; o[1] = a0.y; o[2] = a1.x; o[3] = a1.y; o[4] = a2.x; o[5] = a2.y;
    } else {
#pragma unroll
      for (int d = 0; d < 6; ++d) o[d] = __int_as_float(0x7fc00000);
    }
  }
  const int W0 = 2 * p.w[0] + 1, W1 = 2 * p.w[1] + 1, W2 = 2 * p.w[2] + 1;
  const int ncand = W0 * W1 * W2;
  int count = 0;
  bool ok = true;
  for (int a = 0; a < p.natm; ++a) {
    if (lane == 0) tb.img_off[a] = count;
    const float* base = p.tbase + ((size_t)a * p.nl + l) * 6;
    const float vx = c.x - base[0], vy = c.y - base[1], vz = c.z - base[2];
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
      int sv[3] = {0, 0, 0};
      if (ci < ncand) {
        sv[0] = s0[0] + ci / (W1 * W2) - p.w[0];
        sv[1] = s0[1] + (ci / W2) % W1 - p.w[1];
        sv[2] = s0[2] + ci % W2 - p.w[2];
        const float dx = vx - (sv[0] * p.sc[0] + sv[1] * p.sc[3] + sv[2] * p.sc[6]);
        const float dy = vy - (sv[0] * p.sc[1] + sv[1] * p.sc[4] + sv[2] * p.sc[7]);
        const float dz = vz - (sv[0] * p.sc[2] + sv[1] * p.sc[5] + sv[2] * p.sc[8]);
        in = dx * dx + dy * dy + dz * dz <= lim * lim;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      const int pos = count + __popc(bal & ((1u << lane) - 1u));
      if (in) {
        if (pos < kMaxImg) {
          Img& T = tb.img[pos];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float th = base[d], tl = base[3 + d];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
              const float sf = (float)sv[e];
              const float pr = sf * p.sc[3 * e + d];
              const float pe = fmaf(sf, p.sc[3 * e + d], -pr);   // exact product remainder
              float ss, se;
              two_sum_f(th, pr, ss, se);
              th = ss;
              tl += se + pe + sf * p.sclo[3 * e + d];
            }
            float hh, ll;
            two_sum_f(th, tl, hh, ll);
            T.th[d] = hh;
            T.tl[d] = ll;
          }
        } else {
          ok = false;
        }
      }
      count += __popc(bal);
    }
  }
  if (count > kMaxImg) count = kMaxImg;
  ok = __all_sync(0xffffffffu, ok);
  if (lane == 0) {
    tb.img_off[p.natm] = count;
    tb.ok = ok ? 1 : 0;
  }
}

// The A blocks of the slab: block b (tile, rt, l) holds Phi of the tile's 128 AO rows at the
// 32 points r - L_l of point tile rt, FP16 hi then lo, in the tensor cores' layout. One CTA
// per block at a time; warp 0 builds the tables, every thread generates (shell entry, four
// points) items into shared memory, and the block is stored with 16-byte coalesced stores.
// Three CTAs per SM (80 registers) hide the block barriers a little better than two.
__global__ void __launch_bounds__(kGenThreads, 3) gen_blocks_kernel(TcParams p) {
  __shared__ __align__(16) unsigned char a[kABlock];
  __shared__ StageTab tb;
  __shared__ TcShell shells[kMaxEntries];
  __shared__ int tile_shell0[kMaxTiles + 1];
  __shared__ float rowscale[kMaxTiles * kM];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int e = t; e < p.nentries; e += kGenThreads) shells[e] = p.shells[e];
  for (int e = t; e <= p.ntile; e += kGenThreads) tile_shell0[e] = p.tile_shell0[e];
  for (int e = t; e < p.ntile * kM; e += kGenThreads) rowscale[e] = p.rowscale[e];
  for (int b = blockIdx.x; b < p.nblocks; b += gridDim.x) {
    const uint2 e = p.blocks[b];
    const int rt = (int)(e.x & 0xffffu), l = (int)(e.x >> 16), tile = (int)e.y;
    __syncthreads();   // the previous block is stored (and the tables are free)
    for (int o = t; o < kABlock / 16; o += kGenThreads)
      reinterpret_cast<uint4*>(a)[o] = make_uint4(0, 0, 0, 0);
    if (warp == 0) block_tables(p, tb, tile, rt, l, lane);
    __syncthreads();
    if (!tb.ok) {
      if (t == 0) fail(p.status);
      continue;
    }
    const int s0 = tile_shell0[tile], s1 = tile_shell0[tile + 1];
    const int items = (s1 - s0) * 8;
    for (int it = t; it < items; it += kGenThreads) {
      const TcShell& sh = shells[s0 + (it >> 3)];
      const int g = it & 7;
      const float* rs = rowscale + tile * kM;
      switch (sh.l) {
        case 0: gen_item<0>(tb, sh, g, rs, a, a + kABytes); break;
        case 1: gen_item<1>(tb, sh, g, rs, a, a + kABytes); break;
        case 2: gen_item<2>(tb, sh, g, rs, a, a + kABytes); break;
        default: gen_item<3>(tb, sh, g, rs, a, a + kABytes); break;
      }
    }
    __syncthreads();
    uint4* dst = reinterpret_cast<uint4*>(p.ablk + (size_t)b * kABlock);
    for (int o = t; o < kABlock / 16; o += kGenThreads) dst[o] = reinterpret_cast<const uint4*>(a)[o];
  }
}

// The phases of each stage's (column tile, l) row travel with the stage, in a ring of their
// own: the A/B slot is free once the MMA is done, the phases only once the epilogue is.
constexpr int kPhRing = 8;
constexpr int kPhBytes = kPhaseRow * 4;

struct __align__(16) Smem {
  unsigned long long full[kStages], empty[kStages], acc_full[2], acc_empty[2], done;
  unsigned long long ph_full[kPhRing], ph_empty[kPhRing];
  uint32_t tmem_slot;
};

constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + (size_t)kPhRing * kPhBytes + sizeof(Smem);
static_assert(kSmemBytes <= 227 * 1024, "shared memory of one CTA");
static_assert(kPhBytes % 16 == 0, "bulk copies of whole 16-byte pieces");

__device__ __forceinline__ int st_ablk(uint2 e) { return (int)(e.x & 0x3fffffu); }
__device__ __forceinline__ int st_l(uint2 e) { return (int)(e.x >> 22); }
__device__ __forceinline__ int st_rt(uint2 e) { return (int)(e.y & 0xffffu); }
__device__ __forceinline__ int st_ct(uint2 e) { return (int)((e.y >> 16) & 0xffu); }
__device__ __forceinline__ int st_flags(uint2 e) { return (int)((e.y >> 24) & 7u); }
__device__ __forceinline__ int st_tile(uint2 e) { return (int)((e.y >> 27) & 3u); }

// One lane of the warp waits (bounded) for the mbarrier phase, the warp follows its verdict,
// and the other lanes then observe the completed phase themselves (acquire).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, long long limit_ns,
                                          int lane) {
  int ok = 1;
  if (lane == 0) ok = tc::mbar_wait(bar, parity, limit_ns) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) tc::mbar_try_wait(bar, parity);
  return ok != 0;
}

__global__ void __launch_bounds__(kThreads, 1) contract_tc_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* stage0 = smraw;   // kStages x (A hi | A lo | B hi | B lo)
  float* ph0 = reinterpret_cast<float*>(smraw + kStages * kStageBytes);   // kPhRing phase rows
  Smem& sm = *reinterpret_cast<Smem*>(smraw + kStages * kStageBytes + kPhRing * kPhBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long s_begin = p.cta_stage0[blockIdx.x];
  const long long nst = p.cta_stage0[blockIdx.x + 1] - s_begin;
  const uint2* stages = p.stages + s_begin;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(tc::smem_u32(&sm.full[s]), 1);
      tc::mbar_init(tc::smem_u32(&sm.empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tc::smem_u32(&sm.acc_full[b]), 1);
      tc::mbar_init(tc::smem_u32(&sm.acc_empty[b]), kEThreads);
    }
    tc::mbar_init(tc::smem_u32(&sm.done), 1);
    for (int j = 0; j < kPhRing; ++j) {
      tc::mbar_init(tc::smem_u32(&sm.ph_full[j]), 1);
      tc::mbar_init(tc::smem_u32(&sm.ph_empty[j]), kEWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&sm.tmem_slot), 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sm.tmem_slot;   // accumulators: columns [0, kN) and [256, 256 + kN)

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool good = true;
      long long g = 0;   // accumulator groups: one stage, or a chained pair of stages
      for (long long sidx = 0; sidx < nst && good; ++g) {
        const int ab = (int)(g & 1);
        const int n = ((st_flags(stages[sidx]) & kChain) && sidx + 1 < nst) ? 2 : 1;
        // the epilogue has taken group g - 2 out of this accumulator
        if (g >= 2 && !tc::mbar_wait(tc::smem_u32(&sm.acc_empty[ab]),
                                     (unsigned)(((g >> 1) - 1) & 1), p.wait_ns)) {
          good = false;
          break;
        }
        uint64_t ah[2][2], al[2][2], bh[2][2], bl[2][2];
        int slot[2] = {0, 0};
        for (int q = 0; q < n && good; ++q) {
          const long long si = sidx + q;
          slot[q] = (int)(si % kStages);
          if (!tc::mbar_wait(tc::smem_u32(&sm.full[slot[q]]), (unsigned)((si / kStages) & 1),
                             p.wait_ns))
            good = false;
        }
        if (!good) break;
        tc::tc_fence_after();
        for (int q = 0; q < n; ++q) {
          const uint32_t a_hi = tc::smem_u32(stage0 + (size_t)slot[q] * kStageBytes);
          const uint32_t a_lo = a_hi + kABytes, b_hi = a_hi + kABlock, b_lo = b_hi + kBBytes;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            ah[q][k] = tc::smem_desc(a_hi + k * kASlice, kLBO, kSBO);
            al[q][k] = tc::smem_desc(a_lo + k * kASlice, kLBO, kSBO);
            bh[q][k] = tc::smem_desc(b_hi + k * kBSlice, kLBO, kSBO);
            bl[q][k] = tc::smem_desc(b_lo + k * kBSlice, kLBO, kSBO);
          }
        }
        const uint32_t t_acc = tmem + (uint32_t)(ab * kAccCols);
        // the small cross terms of every K slice of the group first, the hi x hi products
        // last: each accumulation into tensor memory rounds toward zero at the running sum's
        // magnitude, so only the hi x hi additions happen at full magnitude (two per stage)
        uint32_t acc = 0u;
        for (int q = 0; q < n; ++q)
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            tc::mma_f16(t_acc, ah[q][k], bl[q][k], kIdesc, acc);
            tc::mma_f16(t_acc, al[q][k], bh[q][k], kIdesc, 1u);
            acc = 1u;
          }
        for (int q = 0; q < n; ++q)
#pragma unroll
          for (int k = 0; k < 2; ++k) tc::mma_f16(t_acc, ah[q][k], bh[q][k], kIdesc, 1u);
        for (int q = 0; q < n; ++q) tc::mma_commit(tc::smem_u32(&sm.empty[slot[q]]));
        tc::mma_commit(tc::smem_u32(&sm.acc_full[ab]));
        sidx += n;
      }
      if (!good) fail(p.status);
      // every MMA issued has completed before the tensor memory is released
      tc::mma_commit(tc::smem_u32(&sm.done));
      if (!tc::mbar_wait(tc::smem_u32(&sm.done), 0u, p.wait_ns)) fail(p.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ bulk copies of A and B
    if (lane == 0) {
      bool good = true;
      long long sidx = 0;
      for (; sidx < nst; ++sidx) {
        const int s = (int)(sidx % kStages);
        const long long u = sidx / kStages;
        if (u > 0 && !tc::mbar_wait(tc::smem_u32(&sm.empty[s]), (unsigned)((u - 1) & 1),
                                    p.wait_ns)) {
          good = false;
          break;
        }
        const int j = (int)(sidx % kPhRing);
        const long long v = sidx / kPhRing;
        if (v > 0 && !tc::mbar_wait(tc::smem_u32(&sm.ph_empty[j]), (unsigned)((v - 1) & 1),
                                    p.wait_ns)) {
          good = false;
          break;
        }
        const uint2 e = stages[sidx];
        const uint32_t pb = tc::smem_u32(&sm.ph_full[j]);
        tc::mbar_expect_tx(pb, kPhBytes);
        tc::bulk_g2s(tc::smem_u32(ph0 + (size_t)j * kPhaseRow),
                     p.phase + ((size_t)st_ct(e) * p.nl + st_l(e)) * kPhaseRow, kPhBytes, pb);
        const uint32_t fb = tc::smem_u32(&sm.full[s]);
        tc::mbar_expect_tx(fb, kStageBytes);
        const uint32_t dst = tc::smem_u32(stage0 + (size_t)s * kStageBytes);
        tc::bulk_g2s(dst, p.ablk + (size_t)st_ablk(e) * kABlock, kABlock, fb);
        tc::bulk_g2s(dst + kABlock, p.yh + ((size_t)st_ct(e) * p.ntile_r + st_rt(e)) * kBBlock,
                     kBBlock, fb);
      }
      // no copy may be in flight when the CTA leaves: wait for the last ones issued (a stage
      // whose phase copy was issued also had its A/B copies issued, and the other way round,
      // except when the loop stopped between the two waits above)
      for (long long last = std::max<long long>(0, sidx - kStages); last < sidx; ++last) {
        const int s = (int)(last % kStages);
        if (!tc::mbar_wait(tc::smem_u32(&sm.full[s]), (unsigned)((last / kStages) & 1),
                           p.wait_ns))
          good = false;
      }
      for (long long last = std::max<long long>(0, sidx - kPhRing); last < sidx; ++last) {
        const int j = (int)(last % kPhRing);
        if (!tc::mbar_wait(tc::smem_u32(&sm.ph_full[j]), (unsigned)((last / kPhRing) & 1),
                           p.wait_ns))
          good = false;
      }
      if (!good) fail(p.status);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;                    // 0 .. 15
    const int quarter = warp & 3;               // TMEM lanes 32 quarter ..
    const int cs = ew >> 2;                     // complex columns [32 cs, 32 cs + 32)
    const int row = 32 * quarter + lane;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    // running sums of the warp's 32 complex columns as packed pairs of columns:
    // SR[p] = (Re c_2p, Re c_2p+1), SI[p] = (Im c_2p, Im c_2p+1)
    u64 SR[16], SI[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) { SR[j] = 0ull; SI[j] = 0ull; }
    bool good = true;
    int g = 0;             // accumulator groups taken out
    int carry_first = 0;   // kFirstSum of the first stage of a chained pair
    for (int sidx = 0; sidx < (int)nst; ++sidx) {
      const uint2 e = stages[sidx];
      const int jp = sidx % kPhRing;
      const int flags = st_flags(e) | carry_first, ct = st_ct(e);
      if ((flags & kChain) && sidx + 1 < (int)nst) {
        // the first stage of a chained pair: its product comes out with the next stage's;
        // only its phase-ring slot is handed back (once its copy has landed)
        if (!warp_wait(tc::smem_u32(&sm.ph_full[jp]), (unsigned)((sidx / kPhRing) & 1),
                       p.wait_ns, lane)) {
          good = false;
          break;
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tc::smem_u32(&sm.ph_empty[jp]));
        carry_first = flags & kFirstSum;
        continue;
      }
      carry_first = 0;
      const int ab = g & 1;
      if (!warp_wait(tc::smem_u32(&sm.acc_full[ab]), (unsigned)((g >> 1) & 1), p.wait_ns,
                     lane)) {
        good = false;
        break;
      }
      ++g;
      tc::tc_fence_after();
      if (flags & kFirstSum) {
#pragma unroll
        for (int j = 0; j < 16; ++j) { SR[j] = 0ull; SI[j] = 0ull; }
      }
      // cos, sin and -sin of the phases of the warp's columns, from the stage's slot of the
      // phase ring (copied in by the producer with the stage's operands)
      if (!warp_wait(tc::smem_u32(&sm.ph_full[jp]), (unsigned)((sidx / kPhRing) & 1), p.wait_ns,
                     lane)) {
        good = false;
        break;
      }
      const u64* wc = reinterpret_cast<const u64*>(ph0 + (size_t)jp * kPhaseRow) + 16 * cs;
      const u64* ws = wc + kNC / 2;
      const u64* wn = wc + kNC;
      const uint32_t ta = tmem + (uint32_t)(ab * kAccCols) + lane_off + (uint32_t)(64 * cs);
      // eight groups of 4 complex columns (Re at ta + 32 (q/4) + 4 (q%4), Im 16 columns on),
      // software-pipelined: the tensor-memory and phase loads of group q + 1 are in flight
      // while group q is added in
      uint32_t vr[2][4], vi[2][4];
      auto load = [&](int q, int b) {
        const uint32_t tq = ta + 32 * (q >> 2) + 4 * (q & 3);
        tc::tmem_ld4(tq, vr[b]);
        tc::tmem_ld4(tq + 16, vi[b]);
      };
      load(0, 0);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int b = q & 1;
        if (q + 1 < 8) load(q + 1, b ^ 1);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int pi = 2 * q + u;
          const u64 ar = pk::pack(__uint_as_float(vr[b][2 * u]), __uint_as_float(vr[b][2 * u + 1]));
          const u64 ai = pk::pack(__uint_as_float(vi[b][2 * u]), __uint_as_float(vi[b][2 * u + 1]));
          const u64 c = wc[pi], sn = ws[pi], ns = wn[pi];
          SR[pi] = pk::fma(ns, ai, pk::fma(c, ar, SR[pi]));
          SI[pi] = pk::fma(sn, ar, pk::fma(c, ai, SI[pi]));
        }
        if (q + 1 < 8) tc::tmem_wait_ld();
      }
      tc::tc_fence_before();
      tc::mbar_arrive(tc::smem_u32(&sm.acc_empty[ab]));
      __syncwarp();   // every lane has read the phase slot
      if (lane == 0) tc::mbar_arrive(tc::smem_u32(&sm.ph_empty[jp]));
      if (flags & kToGlobal) {
        const int tl = st_tile(e);
        const int mu = p.perm[tl * kM + row];
        if (mu >= 0) {
          const double rf = p.rowf[tl * kM + row] * p.scale;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = ct * kNC + 32 * cs + j;
            if (c >= p.ncol) continue;
            const double f = rf * p.colf[c];
            const int k = c / p.nocc, i = c - k * p.nocc;
            float r0, r1, i0, i1;
            pk::unpack(SR[j >> 1], r0, r1);
            pk::unpack(SI[j >> 1], i0, i1);
            double* dst = reinterpret_cast<double*>(p.kc + ((size_t)k * p.nao + mu) * p.nocc + i);
            atomicAdd(dst, f * (double)((j & 1) ? r1 : r0));
            atomicAdd(dst + 1, f * (double)((j & 1) ? i1 : i0));
          }
        }
      }
    }
    if (!good && lane == 0) fail(p.status);
  }

  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// max over the points of |Re| + |Im| of every (k, i) field of Y, as float bits
// and colf = 2^(e - 13), e the exponent of that max (frexp)
__global__ void colmax_kernel(const float2* __restrict__ Y, unsigned* __restrict__ colmax,
                              double* __restrict__ colf, long long ng, long long fs) {
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
    if (threadIdx.x == 0) {
      colmax[c] = __float_as_uint(m);
      int e2 = 0;
      if (m > 0.f) frexpf(m, &e2);
      colf[c] = ldexp(1.0, e2 - 13);
    }
  }
}

// Y -> FP16 hi/lo B blocks: in block (ct, rt), column c of the tile is row 32 (c / 16) + c % 16
// (Re) and that row + 16 (Im), so that a tensor-memory load of 8 consecutive columns gives
// the real (or imaginary) parts of 8 consecutive columns;
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
    uint4 rh, rl, ih, il;
    float s = 0.f;
    if (c < ncol) {
      const float mx = __uint_as_float(colmax[c]);
      int e2 = 0;
      if (mx > 0.f) frexpf(mx, &e2);
      s = ldexpf(1.f, 13 - e2);
    }
    float xr[8], xi[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long q = (long long)rt * kKP + g * 8 + j;
      float2 v = make_float2(0.f, 0.f);
      if (c < ncol && q < ng) v = Y[(size_t)c * fs + q];
      xr[j] = v.x * s;
      xi[j] = v.y * s;
    }
    split2(xr[0], xr[1], rh.x, rl.x); split2(xr[2], xr[3], rh.y, rl.y);
    split2(xr[4], xr[5], rh.z, rl.z); split2(xr[6], xr[7], rh.w, rl.w);
    split2(xi[0], xi[1], ih.x, il.x); split2(xi[2], xi[3], ih.y, il.y);
    split2(xi[4], xi[5], ih.z, il.z); split2(xi[6], xi[7], ih.w, il.w);
    unsigned char* blk = yh + ((size_t)ct * ntile_r + rt) * kBBlock;
    // rows of the 16-column group of cl: Re of its columns, then Im
    const int r_re = 32 * (cl >> 4) + (cl & 15);
    const int o_re = op_off(r_re, g * 8, kBSlice), o_im = op_off(r_re + 16, g * 8, kBSlice);
    *reinterpret_cast<uint4*>(blk + o_re) = rh;
    *reinterpret_cast<uint4*>(blk + o_im) = ih;
    *reinterpret_cast<uint4*>(blk + kBBytes + o_re) = rl;
    *reinterpret_cast<uint4*>(blk + kBBytes + o_im) = il;
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

// One slab: a run of A blocks generated together, and the CTAs of its stages.
struct TcSlab {
  long long block0 = 0, stage0 = 0;
  int nblocks = 0, cta0 = 0, ncta = 0;
};

struct TcPlan {
  tcc::TcParams prm;
  long long stages = 0;
  size_t smem = 0;
  std::vector<TcSlab> slabs;
  std::vector<void*> bufs;
  unsigned char* yh = nullptr;
  unsigned char* ablk = nullptr;
  uint2* blocks = nullptr;
  unsigned* colmax = nullptr;
  double* colf = nullptr;
};

long long tc_plan_stages(const TcPlan* t) { return t ? t->stages : 0; }
int tc_plan_launches(const TcPlan* t) { return t ? 2 + 2 * (int)t->slabs.size() : 0; }
double tc_flops_per_stage() { return 6.0 * tcc::kM * tcc::kN * tcc::kKP; }

void tc_plan_free(TcPlan* t) {
  if (!t) return;
  for (void* b : t->bufs)
    if (b) cudaFree(b);
  delete t;
}

int tc_plan_create(Plan* p, const std::vector<ShellDev>& sh, const double* xyz,
                   const std::vector<double>& rcut, size_t* total) {
  using namespace tcc;
  // outside these limits the plan keeps the CUDA-core contraction
  if (p->natm > kMaxTcAtoms) return OCCRI_OK;
  const int NL = p->D[0] * p->D[1] * p->D[2];
  if (NL > 32 * 16) return OCCRI_OK;
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
  const int nwords = (NL + 31) / 32;
  for (int d = 0; d < 3; ++d) q.D[d] = p->D[d];
  double sc[3][3], scinv[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      sc[i][j] = p->lat[i][j] * p->D[i];
      q.lat[3 * i + j] = (float)p->lat[i][j];
      q.sc[3 * i + j] = (float)sc[i][j];
      q.sclo[3 * i + j] = (float)(sc[i][j] - (double)q.sc[3 * i + j]);
    }
  inv3x3(sc, scinv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q.scinv[3 * i + j] = (float)scinv[i][j];
  // grid points r_q (fields' order q = (n3 N + n1) N + n2) and L_l + A_a, as hi/lo floats
  std::vector<float> pts((size_t)ng * 6), tbase((size_t)p->natm * NL * 6);
  auto split = [](double x, float* hi, float* lo) {
    *hi = (float)x;
    *lo = (float)(x - (double)*hi);
  };
  for (long long qq = 0; qq < ng; ++qq) {
    const int n2 = (int)(qq % N), tq = (int)(qq / N), n1 = tq % N, n3 = tq / N;
    const double f[3] = {(double)n1 / N, (double)n2 / N, (double)n3 / N};
    for (int d = 0; d < 3; ++d)
      split(f[0] * p->lat[0][d] + f[1] * p->lat[1][d] + f[2] * p->lat[2][d], &pts[6 * qq + d],
            &pts[6 * qq + 3 + d]);
  }
  for (int a = 0; a < p->natm; ++a)
    for (int l = 0; l < NL; ++l) {
      const int l3[3] = {l / (p->D[1] * p->D[2]), (l / p->D[2]) % p->D[1], l % p->D[2]};
      float* o = &tbase[((size_t)a * NL + l) * 6];
      for (int d = 0; d < 3; ++d)
        split(l3[0] * p->lat[0][d] + l3[1] * p->lat[1][d] + l3[2] * p->lat[2][d] + xyz[3 * a + d],
              &o[d], &o[3 + d]);
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
      e.atom = s.atom; e.l = s.l; e.row0 = r0; e.m0 = m; e.nm = take; e.exact = s.exact_arg;
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
  std::vector<double> tpts;
  for (int rt = 0; rt < q.ntile_r; ++rt) {
    double c[3] = {0, 0, 0};
    int cnt = 0;
    tpts.clear();
    for (int j = 0; j < kKP; ++j) {
      const long long qq = (long long)rt * kKP + j;
      if (qq >= ng) break;
      const int n2 = (int)(qq % N), tq = (int)(qq / N), n1 = tq % N, n3 = tq / N;
      const double f[3] = {(double)n1 / N, (double)n2 / N, (double)n3 / N};
      double x[3];
      for (int d = 0; d < 3; ++d)
        x[d] = f[0] * p->lat[0][d] + f[1] * p->lat[1][d] + f[2] * p->lat[2][d];
      for (int d = 0; d < 3; ++d) { c[d] += x[d]; tpts.push_back(x[d]); }
      ++cnt;
    }
    for (int d = 0; d < 3; ++d) c[d] /= std::max(cnt, 1);
    double rad = 0;
    for (int j = 0; j < cnt; ++j) {
      double e2 = 0;
      for (int d = 0; d < 3; ++d) e2 += (tpts[3 * j + d] - c[d]) * (tpts[3 * j + d] - c[d]);
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
  std::vector<unsigned> active((size_t)ntile * q.ntile_r * nwords, 0u);
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
            active[((size_t)tl * q.ntile_r + rt) * nwords + (l >> 5)] |= 1u << (l & 31);
            ++cost_tile_rt[(size_t)tl * q.ntile_r + rt];
          }
        }
      }
    }
  }
  if (max_img > kMaxImg) {
    // a supercell this small puts too many images in reach of a point tile: the plan keeps
    // the CUDA-core contraction (small cells, where it is cheap anyway)
    delete t;
    return OCCRI_OK;
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

  // The A blocks are the (tile, point tile, l) at which the tile reaches r - L_l; they are
  // generated slab by slab (at most kSlabBlocks, one tile and a range of point tiles per
  // slab) into one buffer. A slab's stages are its blocks times the column tiles: per column
  // tile, runs of kFlushTiles point tiles share FP32 running sums, which then go to K_{mu i}.
  // CTAs take contiguous runs of stages of equal count.
  if (ntile > kMaxTiles || (int)shells.size() > kMaxEntries || q.ntile_r > 65536 ||
      q.n_ct > 255) {
    delete t;
    return OCCRI_OK;
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  nsm = std::max(nsm, 1);
  std::vector<uint2> blocks;
  std::vector<uint2> stages;
  std::vector<long long> cta_stage0;
  long long total_st = 0;
  size_t max_slab = 0;
  for (int tl = 0; tl < ntile; ++tl) {
    int rt = 0;
    while (rt < q.ntile_r) {
      // one slab: point tiles [rt0, rt1) of tile tl
      TcSlab slab;
      slab.block0 = (long long)blocks.size();
      const int rt0 = rt;
      while (rt < q.ntile_r) {
        const long long c = cost_tile_rt[(size_t)tl * q.ntile_r + rt];
        if ((long long)blocks.size() - slab.block0 + c > kSlabBlocks && rt > rt0) break;
        ++rt;
      }
      const int rt1 = rt;
      for (int r = rt0; r < rt1; ++r) {
        const unsigned* act = &active[((size_t)tl * q.ntile_r + r) * nwords];
        for (int l = 0; l < NL; ++l)
          if ((act[l >> 5] >> (l & 31)) & 1u)
            blocks.push_back(make_uint2((unsigned)r | ((unsigned)l << 16), (unsigned)tl));
      }
      slab.nblocks = (int)((long long)blocks.size() - slab.block0);
      if (slab.nblocks == 0) continue;
      max_slab = std::max(max_slab, (size_t)slab.nblocks);
      // stages: column tile by column tile, runs of kFlushTiles active point tiles. Inside a
      // run, point tiles go in pairs, and for each offset l active in both tiles of a pair
      // the two stages are chained (one accumulator, one epilogue pass).
      std::vector<int> slot_of((size_t)(rt1 - rt0) * NL, -1);   // A block slot of (r, l)
      {
        int sl = 0;
        for (int r = rt0; r < rt1; ++r) {
          const unsigned* act = &active[((size_t)tl * q.ntile_r + r) * nwords];
          for (int l = 0; l < NL; ++l)
            if ((act[l >> 5] >> (l & 31)) & 1u) slot_of[(size_t)(r - rt0) * NL + l] = sl++;
        }
      }
      std::vector<uint2> st;
      std::vector<size_t> ct_begin(q.n_ct + 1, 0);   // stages of column tile ct in st
      for (int ct = 0; ct < q.n_ct; ++ct) {
        ct_begin[ct] = st.size();
        std::vector<int> run;   // the run's active point tiles
        auto push = [&](int r, int l, unsigned flags) {
          st.push_back(make_uint2((unsigned)slot_of[(size_t)(r - rt0) * NL + l] | ((unsigned)l << 22),
                                  (unsigned)r | ((unsigned)ct << 16) | (flags << 24) |
                                      ((unsigned)tl << 27)));
        };
        auto close_run = [&]() {
          if (run.empty()) return;
          const size_t first = st.size();
          for (size_t i = 0; i < run.size(); i += 2) {
            const int ra = run[i], rb = i + 1 < run.size() ? run[i + 1] : -1;
            for (int l = 0; l < NL; ++l) {
              const bool in_a = slot_of[(size_t)(ra - rt0) * NL + l] >= 0;
              const bool in_b = rb >= 0 && slot_of[(size_t)(rb - rt0) * NL + l] >= 0;
              if (in_a) push(ra, l, in_b ? (unsigned)kChain : 0u);
              if (in_b) push(rb, l, 0u);
            }
          }
          st[first].y |= (unsigned)kFirstSum << 24;
          st.back().y |= (unsigned)kToGlobal << 24;   // never a chained first stage
          run.clear();
        };
        for (int r = rt0; r < rt1; ++r) {
          bool any = false;
          for (int l = 0; l < NL && !any; ++l) any = slot_of[(size_t)(r - rt0) * NL + l] >= 0;
          if (!any) continue;
          run.push_back(r);
          if ((int)run.size() == kFlushTiles) close_run();
        }
        close_run();
      }
      ct_begin[q.n_ct] = st.size();
      // CTAs: every column tile's stages are cut (at run ends) into `parts` ranges of about
      // equal length, one CTA each, with parts = SMs / column tiles (one more for the first
      // SMs % column tiles tiles, so that every SM has a CTA). The CTAs of one part but
      // different column tiles then read the same A blocks in about the same order at about
      // the same time, so an A block comes from DRAM once and from L2 for the others.
      slab.stage0 = (long long)stages.size();
      slab.cta0 = (int)cta_stage0.size();
      int b = 0;
      for (int ct = 0; ct < q.n_ct; ++ct) {
        const size_t b0 = ct_begin[ct], b1 = ct_begin[ct + 1];
        if (b1 == b0) continue;
        const int parts = std::max(1, nsm / q.n_ct + (ct < nsm % q.n_ct ? 1 : 0));
        cta_stage0.push_back(slab.stage0 + (long long)b0);
        ++b;
        int part = 1;
        for (size_t i = b0; i + 1 < b1 && part < parts; ++i) {
          const bool run_end = (st[i].y >> 24) & kToGlobal;
          if (run_end && (double)(i + 1 - b0) >= (double)(b1 - b0) * part / parts) {
            cta_stage0.push_back(slab.stage0 + (long long)i + 1);
            ++b;
            ++part;
          }
        }
      }
      slab.ncta = b;
      stages.insert(stages.end(), st.begin(), st.end());
      total_st += (long long)st.size();
      t->slabs.push_back(slab);
    }
  }
  cta_stage0.push_back((long long)stages.size());
  // per (column tile, l): the phases e^{-ik.L_l} of the tile's 128 columns
  std::vector<float> phase((size_t)q.n_ct * NL * kPhaseRow, 0.f);
  {
    const int Dc = NL;
    for (int ct = 0; ct < q.n_ct; ++ct)
      for (int l = 0; l < NL; ++l) {
        const int l3[3] = {l / (p->D[1] * p->D[2]), (l / p->D[2]) % p->D[1], l % p->D[2]};
        for (int j = 0; j < kNC; ++j) {
          const int c = ct * kNC + j;
          if (c >= q.ncol) break;
          const int k = c / p->nocc;
          long long num = 0;
          for (int d = 0; d < 3; ++d)
            num += (long long)p->kint_h[3 * k + d] * l3[d] * (Dc / p->D[d]);
          num %= Dc;
          const double ang = -2.0 * 3.14159265358979323846 * (double)num / (double)Dc;
          float* row = &phase[((size_t)ct * NL + l) * kPhaseRow];
          row[j] = (float)std::cos(ang);
          row[kNC + j] = (float)std::sin(ang);
          row[2 * kNC + j] = -(float)std::sin(ang);
        }
      }
  }

  // device copies
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess && x != cudaSuccess) e = x; };
  TcShell* d_sh = nullptr; int* d_ts = nullptr; float* d_rs = nullptr; double* d_rf = nullptr;
  int* d_perm = nullptr; float* d_reach = nullptr; float4* d_rt = nullptr;
  uint2* d_st = nullptr; long long* d_s0 = nullptr; uint2* d_bl = nullptr;
  float* d_pts = nullptr; float* d_tb = nullptr; float* d_ph = nullptr;
  chk(put(&d_pts, pts, total)); t->bufs.push_back(d_pts);
  chk(put(&d_tb, tbase, total)); t->bufs.push_back(d_tb);
  chk(put(&d_sh, shells, total)); t->bufs.push_back(d_sh);
  chk(put(&d_ts, tile_shell0, total)); t->bufs.push_back(d_ts);
  chk(put(&d_rs, rowscale, total)); t->bufs.push_back(d_rs);
  chk(put(&d_rf, rowf, total)); t->bufs.push_back(d_rf);
  chk(put(&d_perm, perm, total)); t->bufs.push_back(d_perm);
  chk(put(&d_reach, reach, total)); t->bufs.push_back(d_reach);
  chk(put(&d_rt, rtiles, total)); t->bufs.push_back(d_rt);
  chk(put(&d_st, stages, total)); t->bufs.push_back(d_st);
  chk(put(&d_s0, cta_stage0, total)); t->bufs.push_back(d_s0);
  chk(put(&d_bl, blocks, total)); t->bufs.push_back(d_bl);
  chk(put(&d_ph, phase, total)); t->bufs.push_back(d_ph);
  {
    void* b = nullptr;
    const size_t yb = (size_t)q.n_ct * q.ntile_r * kBBlock;
    *total += yb;
    chk(device_malloc(&b, yb)); t->bufs.push_back(b); t->yh = (unsigned char*)b;
    b = nullptr;
    const size_t ab = std::max<size_t>(1, max_slab) * kABlock;
    *total += ab;
    chk(device_malloc(&b, ab)); t->bufs.push_back(b); t->ablk = (unsigned char*)b;
    b = nullptr;
    *total += (size_t)q.ncol * 4;
    const size_t cm = ((size_t)q.ncol * 4 + 15) / 16 * 16;
    *total += (size_t)q.ncol * 8;
    chk(device_malloc(&b, cm + (size_t)q.ncol * 8)); t->bufs.push_back(b);
    t->colmax = (unsigned*)b;
    t->colf = b ? (double*)((unsigned char*)b + cm) : nullptr;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    tc_plan_free(t);
    return e == cudaErrorMemoryAllocation ? OCCRI_ENOMEM : OCCRI_ECUDA;
  }
  q.yh = t->yh; q.ablk = t->ablk; q.shells = d_sh; q.tile_shell0 = d_ts; q.rowscale = d_rs;
  q.rowf = d_rf; q.perm = d_perm; q.reach = d_reach; q.rtiles = d_rt; q.stages = d_st;
  q.cta_stage0 = d_s0; q.colf = t->colf; q.pts = d_pts; q.tbase = d_tb; q.phase = d_ph;
  q.ntile = ntile;
  q.nentries = (int)shells.size();
  t->blocks = d_bl;
  t->stages = total_st;
  t->smem = kSmemBytes;
  p->tc = t;
  return OCCRI_OK;
}

cudaError_t launch_contract_tc(const Plan& p, cudaStream_t s, LaunchHook* hook) {
  using namespace tcc;
  TcPlan* t = p.tc;
  TcParams q = t->prm;
  q.kc = p.kc;
  q.scale = -p.omega_cell * 4.0 * 3.14159265358979323846 /
            ((double)p.nk * (double)p.ng * (double)p.ng);
  q.status = p.status;
  q.wait_ns = p.wait_ns;
  const float2* Y = (const float2*)p.Y;
  colmax_kernel<<<q.ncol, 256, 0, s>>>(Y, t->colmax, t->colf, p.ng, p.fs);
  convert_y_kernel<<<8 * 152, 256, 0, s>>>(Y, t->colmax, t->yh, q.ncol, q.n_ct, q.ntile_r, p.ng,
                                           p.fs);
  static DeviceCache attr;
  attr.get(p.device, [&] {
    cudaFuncSetAttribute(contract_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)t->smem);
    return 1;
  });
  for (const TcSlab& sl : t->slabs) {
    TcParams qs = q;
    qs.blocks = t->blocks + sl.block0;
    qs.nblocks = sl.nblocks;
    qs.cta_stage0 = q.cta_stage0 + sl.cta0;
    gen_blocks_kernel<<<std::min(sl.nblocks, 152 * 8), kGenThreads, 0, s>>>(qs);
    if (hook) hook->before();
    contract_tc_kernel<<<sl.ncta, kThreads, t->smem, s>>>(qs);
    if (hook) hook->after();
  }
  return cudaGetLastError();
}

}  // namespace occri
