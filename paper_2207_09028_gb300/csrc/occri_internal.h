// occri_internal.h -- plan layout and kernel launchers shared by the CUDA sources.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "occri.h"

namespace occri {

// Cubic grid edges with a compiled transform (each {2,3,5}-smooth, <= 64).
#define OCCRI_FOR_EACH_N(X) \
  X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(36) X(40) \
  X(45) X(48) X(50) X(54) X(60) X(64)

bool grid_edge_supported(int n);

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using cplx_t = typename Vec2<T>::type;

// One shell of primitives on the device.
struct ShellDev {
  double alpha;
  double rcut2;      // squared screening radius
  double norm[7];    // N_lm, m = -l..l
  float alpha_f, alpha_lo, rcut2_f;   // alpha = alpha_f + alpha_lo
  float norm_f[7];
  int l, atom, ao, nimg;   // nimg: prefix of the sorted image list that can reach the cell
  int exact_arg;           // FP32: form r - A - T, r^2 and alpha r^2 in double-float
};

// Geometry / AO tables for the AO kernels (steps a, b, e).
struct AOParams {
  int nk, nao, nocc, natm, nshell;
  long long ng;
  long long fs;      // stride of the orbital-shaped fields: ng rounded up to 64
  int N[3];
  int D[3];          // per-axis k denominators: kappa_{k,d} = kint[k][d] / D[d]
  int Dc;            // D[0]*D[1]*D[2]
  const ShellDev* shells;
  const int* atom_shell0;    // [natm+1] shell range per atom (shells are atom-major)
  int nimg;                  // master image count
  const double* img_d;       // [3][nimg] Cartesian image offsets T'
  const float* img_hi;       // [3][nimg] float hi part
  const float* img_lo;       // [3][nimg] float residual
  const void* img_phase;     // [nk][nimg] e^{i k.T'} in the plan's precision
  const double* d0_d;        // [natm][3][ng] r_n - A - T0 (bohr)
  const float* d0_hi;        // [natm][3][ng]
  const float* d0_lo;        // [natm][3][ng]
  const int* t0;             // [natm][nblk] packed T0 of each point block (3 x 10 bits)
  const int* kint;           // [nk][3]
  // point blocks of 2 x 4 x 4 grid points (one warp each) sharing one Wigner-Seitz
  // shift T0; per (atom, block) the master images sorted by distance from the block
  // centre, and per shell the prefix of that list that reaches every point of the block
  int nb[3], nblk, lmax, nsa;
  const unsigned short* blist;   // [natm][nblk][lmax] master-list indices
  const unsigned short* bpre;    // [natm][nblk][nsa] per-shell prefix lengths
  const void* cs;            // [nk][nao][nocc] N_mu C^k_{mu i}: double2 (FP64) or float4 hi/lo (FP32)
};

// Atoms a plan may have for the tensor-core contraction.
constexpr int kMaxTcAtoms = 8;
struct TcPlan;   // tables and buffers of the tensor-core contraction (occri_contract_tc.cu)

// Parameters of one wave of pair fields (steps c, d): output k, a block of k'.
constexpr int kFadN = 40;   // terms of the Faddeeva approximation (OCCRI_ERF_TRUNC)

struct PairParams {
  int nk, nocc, N1;          // N1: cubic grid edge
  long long ng;
  long long fs;              // field stride in points (orbital, accumulator and scratch
                             // fields): ng rounded up to 64, every field 512-byte aligned
  int k, kp0, nkp;
  int diag;                  // 1: the wave is (k, k) and holds the fields i <= j only
  long long vt_off;          // bytes from a scratch buffer's start to its kernel tables
  const void* vq;            // the plan's kernel tables of every k - k' (qtab_index order), or
                             // null: each wave forms its own behind its scratch (vt_off)
  int* status;               // plan status word (first device error, k), for bounded waits
  long long wait_ns;         // limit of every bounded device wait (nanoseconds)
  int fault;                 // test-only fault injection (OCCRI_FAULT_*), 0 in normal use
  int device;                // CUDA device the plan lives on
  int D[3];
  const int* kint;           // [nk][3]
  double g[6];               // reciprocal metric b_i.b_j: 11, 22, 33, 12, 13, 23
  int kind;                  // occri_kernel_kind
  double inv4w2;             // 1 / (4 omega^2)
  double omega;
  double g0;                 // value at G+q = 0, in units of 4 pi
  double dg0;                // d g0 / d omega, in units of 4 pi
  double rc;                 // truncation radius of OCCRI_COULOMB_TRUNC
  // OCCRI_ERF_TRUNC: Weideman's coefficients of the Faddeeva function w(z) (Im z > 0),
  // w = 2 P(Z)/(L - i z)^2 + 1/(sqrt(pi) (L - i z)), Z = (L + i z)/(L - i z),
  // P(Z) = sum_n fad_a[n] Z^n; erf(omega R_c) and e^{-omega^2 R_c^2}
  double fad_a[kFadN];
  double fad_L, lr_erf, lr_exp;
  int b_div;                 // pass-B CTAs = resident slots / b_div (set by the autotuner)
  int split_cd;              // 1: passes C and D even where the fused pass CD applies
  // FP32 copies (hi/lo for the metric) made on the host, so FP32 kernels never
  // convert from double on the device (FP64 issue is 1/64 rate)
  float gh[6], gl[6];
  float inv4w2_f, omega_f, g0_f, dg0_f;
};
// The transforms apply v/(4 pi) between unnormalised forward and inverse FFTs, so
// Y carries a factor N_g/(4 pi); the contraction restores it in FP64.

struct Plan {
  // problem
  int nk, nao, nocc, natm, nshell, precision;
  int N[3];
  long long ng;
  double lat[3][3];
  double omega_cell;
  occri_kernel kernel;
  cudaStream_t stream;
  double g0_4pi = 0.0, dg0_4pi = 0.0;   // the G+q = 0 value and its omega-derivative / (4 pi)
  double rc = 0.0;                       // truncation radius (OCCRI_COULOMB_TRUNC, _ERF_TRUNC)
  double fad_a[kFadN] = {}, fad_L = 0.0, lr_erf = 0.0, lr_exp = 0.0;   // OCCRI_ERF_TRUNC
  int device = 0;            // the CUDA device current at plan creation; every call runs on it
  int fault = 0;             // test-only fault injection (occri_plan_inject_fault)
  long long wait_ns = 2000000000LL;   // limit of the bounded device waits
  int D[3];
  std::vector<int> kint_h;
  int fields_cap;            // pair fields held by the transform scratch
  long long fs;              // scratch field stride in points (ng rounded up to 64)
  int nkp_wave;              // k' per wave
  int nkp_cap = 1;           // k' per wave the scratch buffers hold
  // launch configuration of the pair loop (occri_plan_autotune may change it)
  int nstreams = 3;          // consecutive waves go round-robin over 1, 2 or 3 streams
  int b_div = 1;             // pass-B CTAs = resident slots / b_div
  int split_cd = 0;          // 1: passes C and D instead of the fused pass CD
  int wave_tables = 0;       // 1: each wave forms its kernel tables even where vq is held
  int tuned = 0;             // 1: the configuration came from the autotuner (or its cache)
  std::vector<int> shells_by_l[4];

  // device tables
  ShellDev* shells = nullptr;
  int* atom_shell0 = nullptr;
  int* shell_list_l[4] = {nullptr, nullptr, nullptr, nullptr};
  double* img_d = nullptr;
  float* img_hi = nullptr;
  float* img_lo = nullptr;
  void* img_phase = nullptr;
  double* d0_d = nullptr;
  float* d0_hi = nullptr;
  float* d0_lo = nullptr;
  int* t0 = nullptr;
  int* kint = nullptr;
  int nimg = 0;
  int nb[3] = {0, 0, 0}, nblk = 0, lmax = 0, nsa = 0;
  unsigned short* blist = nullptr;
  unsigned short* bpre = nullptr;

  // device workspaces. The orbital and accumulator fields store each grid function
  // with the third axis outermost, point (n1, n2, n3) at (n3 N + n1) N + n2: the
  // transform passes then read a plane n1 as N rows of N contiguous points, and the
  // inverse pass along the third axis leaves the potentials of a wave in this same
  // order, so the accumulation streams every array coalesced.
  // Every field (orbital, accumulator or scratch) is fs = ng rounded up to 64 points
  // long, so each starts 512-byte aligned (whole-tile bulk copies).
  void* psi = nullptr;       // [nk][nocc][fs] cplx_t<T>
  void* Y = nullptr;         // [nk][nocc][fs] cplx_t<T>
  // private accumulators of the second and third streams (same layout), added into Y after
  // the wave loop, so that waves on different streams never wait for each other's updates;
  // null when they would take too much memory (the streams' updates of Y are then chained)
  void* Yx[2] = {nullptr, nullptr};
  void* scratch = nullptr;   // [fields_cap][fs] cplx_t<T>, waves on the plan's stream, then
                             // the wave's kernel tables [nkp_wave][m3][m1][m2] T
  void* scratch2 = nullptr;  // the same for the waves on the second stream
  // kernel tables v/(4 pi) of every integer difference kint[k] - kint[k'] ((2 D_d - 1) per
  // axis, each [m3][m1][m2] T), formed once at creation where they take at most
  // kQTabMaxBytes; null otherwise
  void* vq = nullptr;
  // Consecutive waves alternate between the plan's stream and `aux`, each with its own
  // scratch, so one wave's passes overlap the next one's; only the accumulation passes,
  // which both update Y_k, are ordered across the two streams (event ev_y).
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_y = nullptr, ev_iso = nullptr;
  cudaEvent_t ev_iso2 = nullptr;
  // the third stream and scratch (three waves in flight)
  cudaStream_t aux2 = nullptr;
  void* scratch3 = nullptr;
  size_t scratch_bytes = 0;  // bytes of each scratch buffer
  cudaEvent_t ev_join2 = nullptr, ev_iso3 = nullptr;
  // adjoint workspaces, allocated by the first occri_vjp_full call
  void* gam = nullptr;       // [nk][nocc][fs] adjoint orbital field (periodic parts)
  void* gpsi = nullptr;      // [nk][nocc][fs] accumulated dL/dpsi (periodic parts)
  void* cs_g = nullptr;      // scaled coefficients of -dL/dKC (like cs)
  double2* gkc = nullptr;    // [nk][nao][nocc] dL/dKC after the assembly's adjoint
  double2* gcf = nullptr;    // [nk][nao][nocc] dL/dC through the assembly alone
  double2* gacc = nullptr;   // [nk][nao][nocc] dL/dC through the orbitals
  double2* kc = nullptr;     // [nk][nao][nocc]
  double2* xi = nullptr;     // [nk][nao][nocc]
  double2* mmat = nullptr;   // [nk][nocc][nocc]
  double* ek = nullptr;      // [nk]
  double* dacc = nullptr;    // [2] scratch accumulators (d E/d omega)
  int* status = nullptr;     // [2]: first device error code, k index
  bool have_kc = false;
  TcPlan* tc = nullptr;      // OCCRI_MIXED_TC: the tensor-core contraction's tables
  void* asm_scratch = nullptr;   // paper-form assembly: M, T, D (grown on demand)
  size_t asm_bytes = 0;
  double* ao_norm = nullptr; // [nao] N_lm per AO
  void* cs = nullptr;        // scaled coefficients (see AOParams::cs)

  // host-call staging (allocated on first occri_k_build_host)
  double2* h_c = nullptr;
  double2* h_kc = nullptr;
  double2* h_k = nullptr;
  double* h_ex = nullptr;

  size_t workspace_bytes = 0;
  long long launches_per_build = 0;

  // sampled stage timing
  struct TimedSpan { cudaEvent_t a, b; int stage; double units; };
  int timing_every = 0;
  std::vector<cudaEvent_t> ev_free;
  std::vector<TimedSpan> ev_pending;
  std::vector<cudaEvent_t> ev_used;
  double stage_ms[OCCRI_NSTAGES] = {};
  long long stage_n[OCCRI_NSTAGES] = {};
  double stage_units[OCCRI_NSTAGES] = {};

  AOParams ao_params() const;
  PairParams pair_params() const;
};

// orbitals per launch of the orbital kernel, and per launch of the contraction kernel
constexpr int kOrbChunk = 8;
// k-points per thread in the orbital kernel (the image geometry is shared by them);
// the phase table e^{i k.T'} has its k rows padded with zeros to a multiple of 4.
template <typename T> constexpr int orbital_kbatch() { return sizeof(T) == 4 ? 4 : 2; }
constexpr int kPhasePadK = 4;
template <typename T> constexpr int contract_chunk() { return sizeof(T) == 4 ? 8 : 4; }

// ---- launchers (return cudaError_t of the launch) ----
template <typename T>
cudaError_t launch_scale_c(const Plan& p, const double2* C, cudaStream_t s);
template <typename T>
cudaError_t launch_orbitals(const Plan& p, cudaStream_t s);
// k-points [k0, k0 + nkk) (nkk < 0: all from k0)
template <typename T>
cudaError_t launch_contract(const Plan& p, cudaStream_t s, int k0 = 0, int nkk = -1);
// The same stages on other buffers (the adjoint): orbitals of the scaled coefficients cs
// into out; scaled coefficients factor N_mu X of X into out; scale N_mu sum_r conj(chi) F
// added into out.
template <typename T>
cudaError_t launch_orbitals_to(const Plan& p, const void* cs, void* out, cudaStream_t s,
                               int k0 = 0, int nkk = -1);
template <typename T>
cudaError_t launch_scale_to(const Plan& p, const double2* X, void* out, double factor,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_contract_field(const Plan& p, const void* F, double2* out, double scale,
                                  cudaStream_t s, int k0 = 0, int nkk = -1);
// F[k][i][.] *= e^{sign i k.r} over the orbital-shaped field F (psi -> periodic parts
// with sign -1 before the pair passes, accumulated periodic parts -> Y with +1 after).
template <typename T>
cudaError_t launch_phase_fields(const Plan& p, void* F, int sign, cudaStream_t s, int k0 = 0,
                                int nkk = -1);
// Pair-wave launches over unordered pairs: diag = 1 is the wave (k, k) with fields
// i <= j; diag = 0 covers k' in [kp0, kp0 + nkp), all kp0 > k, with every (i, j).
// S is the wave's scratch and Y the accumulator the wave adds into (the plan's Y, or the
// private one of the wave's stream). When ev != nullptr, ev[0..3] are recorded before pass
// A, before pass B, before pass C and after pass D. When ev_y != nullptr, pass D first
// waits for it and then records it (orders the updates of one Y by waves on several streams).
template <typename T>
cudaError_t launch_pair_wave(const Plan& p, int k, int kp0, int nkp, int diag, cudaStream_t s,
                             void* S, void* Y, cudaEvent_t* ev = nullptr,
                             cudaEvent_t ev_y = nullptr);
template <typename T>
cudaError_t launch_domega_wave(const Plan& p, int k, int kp0, int nkp, int diag, cudaStream_t s);
// The plan's kernel tables of every k - k' into p.vq (allocated by the caller), on stream s.
template <typename T>
cudaError_t launch_qtables(const Plan& p, cudaStream_t s);
// Most device memory the plan's kernel tables may take; beyond it every wave forms its own.
constexpr size_t kQTabMaxBytes = (size_t)4 << 30;
// One wave of the adjoint build: forward potentials in scratch, adjoint potentials in
// scratch2, their contributions added to gpsi (uses psi and gam); with dacc != nullptr
// also the omega term sum (dv/d omega)/(4 pi) Re(conj(sigma^) rho^) added to *dacc.
template <typename T>
cudaError_t launch_vjp_wave(const Plan& p, int k, int kp0, int nkp, int diag, double* dacc,
                            cudaStream_t s);

// Largest nocc whose FP32 waves run the inverse along m3 and the Y accumulation as one
// fused pass. A wave launches passes A (with the wave's kernel tables where the plan holds
// none) and B, then the fused pass or passes C and D.
constexpr int kFusedCdNoc = 8;
template <typename T> constexpr int pair_wave_launches(int nocc, int split_cd = 0) {
  return (std::is_same<T, float>::value && nocc <= kFusedCdNoc && !split_cd) ? 3 : 4;
}

// scratch per wave (MB): how many k' one wave takes when nocc^2 fields of a k' fit
constexpr int kWaveBudgetMB = 96;

// fields and pass-C targets of a wave
__host__ __device__ inline int wave_fields(int nocc, int nkp, int diag) {
  return diag ? nocc * (nocc + 1) / 2 : nkp * nocc * nocc;
}
inline int wave_targets(int nocc, int nkp, int diag) { return diag ? nocc : nocc + nkp * nocc; }
template <typename T>
cudaError_t launch_widen(const Plan& p, void* out, cudaStream_t s);

// The tensor-core contraction (OCCRI_MIXED_TC): tables built at plan creation from the shells
// (with their screening radii) and atom positions, freed with the plan; the launch turns the
// Bloch-phased Y into FP16 hi/lo blocks and adds K_{mu i} into p.kc.
int tc_plan_create(Plan* p, const std::vector<ShellDev>& shells, const double* xyz,
                   const std::vector<double>& rcut, size_t* total);
void tc_plan_free(TcPlan* t);
long long tc_plan_stages(const TcPlan* t);
int tc_plan_launches(const TcPlan* t);      // kernels one tensor-core contraction launches
double tc_flops_per_stage();
// Paper-form assembly and conduction-band helpers (occri_assemble.cu), on the plan's stream.
cudaError_t launch_assemble_paper(Plan& p, int ncol, const double2* S, const double2* C,
                                  const double2* KC, double2* K);
cudaError_t launch_gather_cols(const double2* all, double2* cr, long long rows, int nocc, int nr,
                               cudaStream_t s);
cudaError_t launch_band_diff(const double2* all, const double2* rr, double2* out, long long rows,
                             int nocc, int nr, cudaStream_t s);   // MMA flops of one stage of the tensor-core contraction   // stages of one contraction (0 without a plan)
// Called around every GEMM launch of the tensor-core contraction (stage timing).
struct LaunchHook {
  virtual void before() = 0;
  virtual void after() = 0;
  virtual ~LaunchHook() = default;
};
cudaError_t launch_contract_tc(const Plan& p, cudaStream_t s, LaunchHook* hook = nullptr);

// Launch settings derived once per kernel instantiation and device (function attributes,
// resident-slot counts): each entry is filled under a lock the first time a plan on that
// device launches the kernel.
constexpr int kMaxDevices = 64;
struct DeviceCache {
  std::mutex mu;
  bool set[kMaxDevices] = {};
  int val[kMaxDevices] = {};
  template <typename F>
  int get(int device, F&& init) {
    if (device < 0 || device >= kMaxDevices) device = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!set[device]) {
      val[device] = init();
      set[device] = true;
    }
    return val[device];
  }
};

// Makes the plan's device current for the duration of an entry-point call and restores
// the caller's current device afterwards (ok = false if either could not be queried or set).
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return;
    }
    if (cur != dev) {
      if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
        return;
      }
      prev = cur;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Allocation with the test-only failure injection of occri_debug_fail_allocation: when
// armed, the chosen allocation reports cudaErrorMemoryAllocation without allocating.
cudaError_t device_malloc(void** ptr, size_t bytes);

}  // namespace occri

// The opaque handle behind occri_plan*.
struct occri_plan {
  occri::Plan* p;
};
