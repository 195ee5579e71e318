/*
 * occri.h -- C ABI of the GB300 occ-RI-K exact-exchange library (liboccri.so).
 *
 * The library builds the exact-exchange matrix of a periodic solid in a
 * Gaussian basis by the occ-RI-K algorithm of Lee, Rettig, Feng, Epifanovsky
 * and Head-Gordon, arXiv:2207.09028 (Sec. II.D, Algorithm 3, with the
 * integral-direct AO treatment of Algorithm 4):
 *   (a) Bloch-summed Gaussian AOs on the real-space grid (Sec. II.A),
 *   (b) occupied orbitals on the grid (Eq. occmo),
 *   (c) pair densities conj(psi_jk') psi_ik e^{-iq.r}, q = k - k' (Eq. aodf),
 *   (d) forward FFT x kernel v(|G+q|) x inverse FFT (Eqs. Vrao, VGao,
 *       recipcoul), accumulated into Y_ik = sum_{k'j} psi_jk' W (Eq. occrikinterm),
 *   (e) K_{mu i}(k) = -(Omega/(N_k N_g)) sum_r conj(chi_mu k) Y_ik (Eq. occrik),
 *   (f) occ-RI assembly in ACE form K_k = KC (C^H KC)^{-1} KC^H, and
 *       E_x = (1/N_k) sum_k Re Tr(C_k^H KC_k) in Ha per cell (closed shell).
 *
 * Conventions.
 *   Lengths in bohr, exponents in bohr^-2, omega in bohr^-1.
 *   Lattice rows a_1, a_2, a_3. Grid points r_n = sum_i (n_i/N_i) a_i,
 *   n = (n1*N2 + n2)*N3 + n3 (n3 fastest).
 *   Bloch AO chi_{mu k}(r) = sum_T e^{i k.T} phi_mu(r - A_mu - T), without the
 *   1/sqrt(N_k) of Sec. II.A; the 1/N_k sits in K instead.
 *   Primitives phi = N_lm P_lm(r) e^{-alpha r^2}, real solid harmonics, unit
 *   norm. AO order: shell order as given (callers use atom -> l -> exponent),
 *   m ascending: p = (x, y, z); d = (xy, yz, 3z^2-r^2, xz, x^2-y^2);
 *   f = (y(3x^2-y^2), xyz, y(4z^2-x^2-y^2), z(2z^2-3x^2-3y^2),
 *        x(4z^2-x^2-y^2), z(x^2-y^2), x(x^2-3y^2)).
 *   Kernel per FFT bin m: x_i = m_i + q_i reduced to [-N_i/2, N_i/2); at an
 *   exact tie x_i = -N_i/2 the two aliases are averaged; the bin G+q = 0
 *   takes g0 (0, or pi/omega^2 for erfc with g0_mode = 1).
 *   Complex numbers are interleaved (re, im) doubles ("c128") unless stated.
 *
 * Ownership. The caller owns every buffer passed in; the plan owns its
 * workspaces (orbitals, Y accumulator, transform scratch, tables). Host
 * structs are copied at plan creation.
 *
 * Streams. Every call is asynchronous on the plan's stream except
 * occri_plan_create (which uploads tables and synchronises), occri_plan_sync,
 * and the *_host entry points (which synchronise before returning).
 *
 * Errors. Every entry point returns an occri_status; none aborts or throws.
 * Device-side failures (a non-positive-definite C^H K C) are recorded in the
 * plan and returned by the next occri_plan_sync.
 */
#ifndef OCCRI_H
#define OCCRI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OCCRI_OK = 0,
  OCCRI_EINVAL = 1,        /* bad argument: shapes, nocc > nao, grid not {2,3,5}-smooth,
                              l > 3, omega <= 0 for erfc/erf, NULL required pointer */
  OCCRI_ENOMEM = 2,        /* a workspace allocation failed */
  OCCRI_ENOTPD = 3,        /* -C^H K C was not positive definite at some k: a Cholesky pivot
                              fell to <= tol * (largest diagonal), tol = 1e-10 (FP64) or
                              1e-5 (mixed) */
  OCCRI_ECUDA = 4,         /* a CUDA runtime call failed */
  OCCRI_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  OCCRI_EUNSUPPORTED = 6   /* valid input outside what this build implements */
} occri_status;

/* Kernels v(r) of the exchange operator (Eq. recipcoul, and the truncations of Sec. II.A):
 * OCCRI_COULOMB 1/r, OCCRI_ERFC erfc(omega r)/r, OCCRI_ERF erf(omega r)/r,
 * OCCRI_COULOMB_TRUNC 1/r cut at R_c (Spencer-Alavi), (4 pi/3) R_c^3 = the volume of the
 * k-mesh's supercell D_1 a_1 x D_2 a_2 x D_3 a_3 (D_d: the k denominators, see occri_kmesh),
 * whose transform is (4 pi/x^2)(1 - cos(x R_c)), and
 * OCCRI_ERF_TRUNC erf(omega r)/r cut at the same R_c (Eq. lrtrunc, Appendix A), whose transform
 * (4 pi/x^2)[e^{-x^2/(4 omega^2)} - e^{-omega^2 R_c^2} Re(e^{-i x R_c} w(z)) - erf(omega R_c)
 * cos(x R_c)], z = -x/(2 omega) + i omega R_c, uses the Faddeeva function w (bounded in the
 * upper half plane, so the cancellation of the appendix does not arise), evaluated in FP64 by
 * Weideman's rational approximation with 40 terms (1994; ~1e-14 relative there). Its
 * omega-derivative is not implemented: occri_vjp and occri_vjp_full return
 * OCCRI_EUNSUPPORTED when asked for d/d omega with this kernel. */
typedef enum {
  OCCRI_COULOMB = 0, OCCRI_ERFC = 1, OCCRI_ERF = 2, OCCRI_COULOMB_TRUNC = 3, OCCRI_ERF_TRUNC = 4
} occri_kernel_kind;

/* OCCRI_FP64: every step in double precision.
 * OCCRI_MIXED: AO evaluation, orbitals, pair densities, FFTs, the kernel multiply
 *   and the Y accumulation in FP32; the contraction (e) accumulates per thread in
 *   FP32 and across threads in FP64; assembly (f) and E_x in FP64.
 * OCCRI_MIXED_TC: as OCCRI_MIXED, but the contraction (e) runs on the tensor cores as
 *   one GEMM over the grid points of the k-mesh's supercell: the AOs periodised over the
 *   supercell (generated on the fly) times Y, both split into FP16 hi + lo parts with
 *   power-of-two scalings, three FP16 products with FP32 accumulation per term; each
 *   32-point product leaves tensor memory at once, times the phase of its supercell offset,
 *   into FP32 running sums over at most 16 point tiles, and FP64 sums beyond.
 *   Where the supercell has more than 512 cells, the cell more than 8 atoms, or a tile of 32
 *   grid points more than 128 supercell images in reach (small supercells), the plan keeps
 *   the CUDA-core contraction of OCCRI_MIXED; occri_plan_info reports which one it uses. */
typedef enum { OCCRI_FP64 = 0, OCCRI_MIXED = 1, OCCRI_MIXED_TC = 2 } occri_precision;

typedef struct {
  double a[3][3];          /* lattice rows a_1, a_2, a_3 (bohr) */
  int natm;
  const double *xyz;       /* host, natm x 3 atom positions (bohr) */
} occri_cell;

typedef struct {
  int nshell;
  const int *atom;         /* host, nshell atom indices in [0, natm) */
  const int *l;            /* host, nshell angular momenta in [0, 3] */
  const double *alpha;     /* host, nshell exponents (bohr^-2), > 0 */
} occri_basis;

typedef struct {
  int nk;
  const double *kfrac;     /* host, nk x 3 fractional k-points; every coordinate must be a
                              rational j/D with D <= 64 on its axis (all Monkhorst-Pack
                              meshes qualify), else OCCRI_EUNSUPPORTED */
} occri_kmesh;

typedef struct {
  int kind;                /* occri_kernel_kind (Eq. recipcoul) */
  double omega;            /* range-separation parameter (bohr^-1), > 0 for erfc / erf */
  int g0_mode;             /* the G+q = 0 term (Eq. VGao's chi):
                              0: dropped;
                              1: f(x -> 0): pi/omega^2 (erfc), 2 pi R_c^2 (truncated Coulomb),
                                 4 pi [(R_c^2/2 - 1/(4 omega^2)) erf(omega R_c) + R_c
                                 e^{-omega^2 R_c^2}/(2 omega sqrt(pi))] (truncated erf);
                              2: the Madelung correction of the supercell of volume V
                                 (Coulomb: chi = -V v_M, v_M the Ewald potential at a unit
                                 point charge from its images in a neutralising background;
                                 erf: chi = V 2 omega/sqrt(pi) - sum_{G != 0} 4 pi
                                 e^{-G^2/(4 omega^2)}/G^2 over the supercell's reciprocal
                                 lattice, the kernel's integral minus its lattice sum) */
} occri_kernel;

typedef struct {
  int nk, nao, nocc, natm, nshell;
  int grid[3];
  long long ng;
  int precision;
  size_t workspace_bytes;  /* device bytes owned by the plan */
  int fields_per_wave;     /* pair fields transformed per launch group */
  long long launches_per_build;  /* kernels one occri_k_build launches */
  int contraction_tc;      /* 1: step (e) runs on the tensor cores (OCCRI_MIXED_TC where the
                              supercell admits it), 0: on the CUDA cores */
  long long tc_stages;     /* tensor-core contraction: stages per build, else 0 */
  double tc_flops_per_stage;  /* MMA flops one stage issues: 3 products (FP16 hi/lo) of
                                 M = 128 AO rows, N = 192 (Re, Im of 96 (k, i) columns),
                                 K = 32 grid points, i.e. 3 x 2 M N K */
} occri_plan_info_t;

/* Stages reported by occri_plan_stage_times. */
enum {
  OCCRI_STAGE_ORBITALS = 0,  /* (a)+(b) */
  OCCRI_STAGE_PAIR_A = 1,    /* (c)+(d) pass A: pair density, FFT along n3 and n2; where the
                                plan holds no kernel tables (occri_tune_t.wave_tables), also
                                the wave's, filled by extra CTAs of the same launch */
  OCCRI_STAGE_PAIR_B = 2,    /* (d) pass B: FFT along n1, kernel, inverse along m2, m1 */
  OCCRI_STAGE_PAIR_C = 3,    /* (d) inverse along m3 and the Y accumulation (one fused pass
                                for FP32 waves of nocc <= 8, else passes C and D) */
  OCCRI_STAGE_CONTRACT = 4,  /* (e) */
  OCCRI_STAGE_ASSEMBLE = 5,  /* (f) */
  OCCRI_STAGE_PAIRS = 6,     /* (c)+(d): the whole loop over pair waves, wall time */
  OCCRI_STAGE_CONTRACT_GEMM = 7,  /* (e) on the tensor cores: the GEMM kernels alone (inside
                                     OCCRI_STAGE_CONTRACT, which also holds the Y conversion
                                     and the A-block generation) */
  OCCRI_NSTAGES = 8
};

typedef struct occri_plan occri_plan;

/* Validate the problem, build image lists and tables, allocate workspaces.
 * Problem statement: Sec. II.A (cell, Bloch AOs), Eq. recipcoul (kernel).
 * grid: N1, N2, N3, each {2,3,5}-smooth in [4, 64]; this build requires
 * N1 = N2 = N3 with an edge in {8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40,
 * 45, 48, 50, 54, 60, 64} and nocc <= 32 (else OCCRI_EUNSUPPORTED): every 1-D transform is
 * compiled for its length, and the pair passes are compiled per cubic edge. cuda_stream: a
 * cudaStream_t or NULL (legacy default stream). The plan lives on the device current at
 * this call: every later call on it makes that device current for its duration and then
 * restores the caller's. Among its workspaces are the kernel tables v/(4 pi) of every integer
 * k - k' on the mesh, formed here where they take at most 4 GiB (occri_tune_t.wave_tables).
 * On success *out owns a plan to be destroyed with occri_plan_destroy; on failure *out is
 * NULL. */
int occri_plan_create(occri_plan **out, const occri_cell *cell, const occri_kmesh *kmesh,
                      const occri_basis *basis, int nocc, const int grid[3],
                      const occri_kernel *kernel, int precision, void *cuda_stream);

int occri_plan_destroy(occri_plan *plan);
int occri_plan_info(const occri_plan *plan, occri_plan_info_t *info);
int occri_plan_set_stream(occri_plan *plan, void *cuda_stream);

/* Synchronise the plan's stream and return the first device-side status
 * recorded since the previous sync (OCCRI_ENOTPD, ...). *bad_k (may be NULL)
 * receives the k index of an OCCRI_ENOTPD failure, else -1. */
int occri_plan_sync(occri_plan *plan, int *bad_k);

/* One exchange build, steps (a)-(f) (Algorithm 3 + ACE assembly).
 * C_dev : device, c128 [nk][nao][nocc] row-major, read only.
 * KC_dev: device, c128 [nk][nao][nocc] = K_{mu i}(k) (Eq. occrik), or NULL.
 * K_dev : device, c128 [nk][nao][nao] ACE-form exchange matrix, or NULL.
 * Ex_dev: device, 1 double, E_x in Ha per cell, or NULL.
 * Asynchronous; call occri_plan_sync to observe OCCRI_ENOTPD. */
int occri_k_build(occri_plan *plan, const void *C_dev, void *KC_dev, void *K_dev,
                  double *Ex_dev);

/* Launch configuration of the pair loop (Algorithm 3's loops over (k, k') and orbital
 * pairs, scheduled as waves of fields). None of it changes what is computed; the choice of
 * wave width and of fused or separate passes C and D changes the order of the FP32/FP64
 * accumulations, i.e. the rounding. */
typedef struct {
  int k_per_wave;       /* k' per wave (1 .. the plan's scratch capacity) */
  int streams;          /* 1, 2 or 3: consecutive waves go round-robin over that many streams,
                           each with its own scratch (default 3) */
  int pass_b_div;       /* pass-B CTAs = resident CTA slots / pass_b_div (1 or 2) */
  int split_cd;         /* 1: separate passes C and D where the fused pass CD applies */
  int wave_tables;      /* 1: every wave forms its own kernel tables v/(4 pi); 0 (default): the
                           waves read the plan's tables, one per integer k - k' on the mesh,
                           formed once at plan creation where they take at most 4 GiB
                           ((2 D_1 - 1)(2 D_2 - 1)(2 D_3 - 1) N_g values of the plan's real
                           type, D_d the mesh's k denominators). occri_plan_tuning reports 1
                           when the plan holds no tables. Same values either way */
  double us_per_field;  /* autotuner: measured microseconds per pair field of this choice */
  double us_default;    /* autotuner: the same for the default (widest wave, 3 streams, 1, 0) */
  int candidates;       /* autotuner: configurations timed; 0: taken from the cache;
                           occri_plan_tuning: -1 if the autotuner set it, else 0 */
} occri_tune_t;

enum { OCCRI_TUNE_FORCE = 1 };   /* time again even if the cache holds this shape */

/* Autotuner (not in the paper): times every candidate launch configuration of the pair loop
 * (k' per wave in powers of two up to the scratch capacity, one to three streams, pass-B CTAs
 * per resident slot 1 or 1/2, fused or separate passes C and D) on the plan's own buffers,
 * with CUDA events on the plan's stream, over the same number of pair fields each, and
 * keeps the fastest. The choice is cached per (device, grid edge, nocc, precision, N_k,
 * scratch capacity) for the life of the process: later calls, and plans created later with
 * the same shape, take it from the cache unless flags has OCCRI_TUNE_FORCE.
 * Synchronises the plan's stream. Leaves the plan's accumulators in an undefined state
 * (every build overwrites them). chosen (may be NULL) receives the configuration.
 * OCCRI_EINVAL for a NULL plan or unknown flags. */
int occri_plan_autotune(occri_plan *plan, int flags, occri_tune_t *chosen);

/* The plan's current launch configuration (us_* fields 0). */
int occri_plan_tuning(const occri_plan *plan, occri_tune_t *current);

/* Set the launch configuration by hand (k_per_wave >= 1, clamped to the scratch capacity;
 * streams 1, 2 or 3; pass_b_div 1 or 2; split_cd 0 or 1; wave_tables 0 or 1; other fields
 * ignored), else OCCRI_EINVAL. Takes effect at the next build. The autotuner and its cache
 * leave wave_tables as it is. */
int occri_plan_set_tuning(occri_plan *plan, const occri_tune_t *cfg);

/* The paper's form of the assembly (Sec. II.C, Eq. occrikop): K ~ PKP + PKQ + QKP, where
 * P = C C^H S projects on the orbitals C (S-orthonormal: C^H S C = 1) and Q = 1 - P; the QKQ
 * block is dropped. Per k, in FP64:
 *   K = KC (S C)^H + (S C) KC^H - (S C) M (S C)^H,   M = (C^H KC + KC^H C) / 2.
 * It agrees with the ACE form of occri_k_build on the occupied space (K C = KC) and keeps the
 * occupied-virtual blocks exactly.
 * ncol  : columns of C and KC, 1 <= ncol <= nao: the plan's nocc, or nocc plus chosen
 *         conduction bands (with KC from occri_k_build_conduction, Sec. II.D; P then projects
 *         on all ncol orbitals and only the block of the remaining bands is dropped).
 * S_dev : device c128 [nk][nao][nao], the AO overlap S^k of the Bloch AOs (Hermitian).
 * C_dev : device c128 [nk][nao][ncol]. KC_dev: device c128 [nk][nao][ncol] = <mu|K|p>.
 * K_dev : device c128 [nk][nao][nao], written. All buffers are the caller's; read only
 *         except K_dev. Asynchronous on the plan's stream; the plan keeps a scratch of
 *         16 (nk ncol^2 + 2 nk nao ncol) bytes, grown on demand (OCCRI_ENOMEM if that fails).
 * OCCRI_EINVAL for a NULL buffer or ncol outside [1, nao]. */
int occri_k_assemble_paper(occri_plan *plan, int ncol, const void *S_dev, const void *C_dev,
                           const void *KC_dev, void *K_dev);

/* Exchange columns of chosen conduction bands (Sec. II.D, conduction-band paragraph):
 * KCr[k][mu][r] = K_{mu p}(k) = -sum_{k'} sum_{i in occ} (mu_k i_k' | i_k' p_k), p the r-th
 * conduction band, i.e. the exchange operator of the occupied density applied to band p.
 * plan_all: a plan whose orbitals are the nocc occupied ones followed by the nr bands
 *           (its nocc = nocc + nr); plan_r: the same cell, k-mesh, basis, grid, kernel and
 *           precision with nocc = nr (the bands alone).
 * The result is KC of plan_all's build (every orbital summed over) minus KC of plan_r's
 * build (the bands' own terms), so it costs one build of each.
 * C_all_dev: device c128 [nk][nao][nocc + nr], occupied columns first.
 * KCr_dev  : device c128 [nk][nao][nr], written.
 * Both builds run on plan_all's stream; the call synchronises it, allocates and frees a
 * temporary of 16 nk nao (nocc + 3 nr) bytes (OCCRI_ENOMEM), and returns the first device
 * error of either build (as occri_plan_sync). OCCRI_EINVAL if the plans differ in anything
 * but nocc, or plan_r's nocc is not below plan_all's. */
int occri_k_build_conduction(occri_plan *plan_all, occri_plan *plan_r, const void *C_all_dev,
                             void *KCr_dev);

/* One-shot build with the signature of the problem statement (Sec. II.A and Eq. occrik):
 * creates a plan for (cell, kmesh, basis, nocc, grid, kernel, precision) on the current
 * device, runs occri_k_build(C_dev -> K_dev, Ex_dev) on cuda_stream, synchronises, and
 * destroys the plan. C_dev, K_dev, Ex_dev: device buffers as in occri_k_build (K_dev or
 * Ex_dev may be NULL). Returns the first failure of the three steps (creation errors as
 * occri_plan_create, then build and device-side errors such as OCCRI_ENOTPD as
 * occri_plan_sync). Every call pays the plan's set-up (tables, workspaces); repeated
 * builds of one cell should keep a plan instead. */
int occri_k_build_once(const occri_cell *cell, const occri_kmesh *kmesh,
                       const occri_basis *basis, const void *C_dev, int nocc, const int grid[3],
                       const occri_kernel *kernel, int precision, void *K_dev, double *Ex_dev,
                       void *cuda_stream);

/* The same build with HOST buffers (same layouts; NULL outputs skipped): copies
 * C to the device, builds, copies the outputs back, synchronises. */
int occri_k_build_host(occri_plan *plan, const void *C_host, void *KC_host, void *K_host,
                       double *Ex_host);

/* Steps (a)+(b) only (Sec. II.A Bloch sums, Eq. occmo): psi_dev receives
 * c128 [nk][nocc][N_g] occupied orbitals on the grid (computed in the plan's
 * precision, widened to c128). Asynchronous. */
int occri_orbitals(occri_plan *plan, const void *C_dev, void *psi_dev);

/* Adjoint of E_x (hand-written, pair densities recomputed, W never stored).
 * gEx: the incoming gradient dL/dE_x.
 * gC_dev: device c128 [nk][nao][nocc] receives gEx * 2 dE_x/dC* =
 *   gEx * (4/N_k) K_{mu i}(k) (PyTorch's conjugate-Wirtinger convention), or NULL.
 * gomega_dev: device double receives gEx * dE_x/d omega
 *   = -gEx (Omega/N_k^2) sum_{kk'ij} sum_m (dv_q(m)/d omega) |rho^_{ij}^{kk'}(m)|^2, or NULL
 *   (zero for the Coulomb kernel).
 * Requires a preceding occri_k_build with the same C (its K_{mu i} is reused). */
int occri_vjp(occri_plan *plan, const void *C_dev, double gEx, void *gC_dev,
              double *gomega_dev);

/* Adjoint of the whole build for any seed: dL/dE_x, dL/dK_{mu i} and dL/dK (the energy
 * of Sec. II.A, Eq. occrik and the ACE assembly, differentiated; not in the paper).
 * gEx      : dL/dE_x.
 * gKC_dev  : device c128 [nk][nao][nocc], the gradient of L with respect to K_{mu i}(k) in
 *            PyTorch's convention (2 dL/dKC*), or NULL.
 * gK_dev   : device c128 [nk][nao][nao], the same for K (any matrix; K is Hermitian, so
 *            only the Hermitian part of the seed matters), or NULL.
 * gC_dev   : device c128 [nk][nao][nocc] receives 2 dL/dC* (every C entry free).
 * gomega_dev: device double receives dL/d omega through the kernel (zero for Coulomb), or
 *            NULL; it adds, per unordered pair, sum_m (dv_q(m)/d omega) Re(conj(sigma^) rho^)
 *            with sigma the adjoint density below.
 * The assembly is differentiated in FP64. The rest recomputes, per unordered pair, the
 * forward potential W and the potential Z of the adjoint density conj(psi_jk') g_ik +
 * conj(g_jk') psi_ik, g_ik = sum_mu chi_mu dL/dK_{mu i}: two pair round trips per pair.
 * With gKC_dev = gK_dev = NULL it equals occri_vjp's gC and gomega. Requires a preceding
 * occri_k_build with the same C; the first call allocates two more orbital-sized fields.
 * Asynchronous on the plan's stream. */
int occri_vjp_full(occri_plan *plan, const void *C_dev, double gEx, const void *gKC_dev,
                   const void *gK_dev, void *gC_dev, double *gomega_dev);

/* Stage timing with CUDA events on the plan's stream. every > 0 brackets every
 * `every`-th pair wave (run alone: the other stream waits around it) and every orbital,
 * contraction and assembly stage and the whole pair loop with events; every = -1 records
 * the stage and pair-loop spans only (no wave is sampled or run alone, so the build runs
 * as it does untimed); every = 0 turns timing off and discards pending samples. */
int occri_plan_set_timing(occri_plan *plan, int every);

/* Synchronise, resolve pending events and return, per stage, the accumulated
 * device milliseconds, the number of timed launches and the number of pair
 * fields (stages 1-3) or k-points (stages 0, 4, 5) those launches covered.
 * Arrays have OCCRI_NSTAGES entries; the accumulators are then reset. */
int occri_plan_stage_times(occri_plan *plan, double *ms, long long *launches, double *units);

/* Bytes of device memory behind occri_orbitals_noalloc (one array per GPU that loads
 * the library, held until the process exits). */
#define OCCRI_STATIC_SCRATCH_BYTES (32u << 20)

/* occri_orbitals for callers that cannot allocate device memory at call time -- for
 * example hosts whose device memory is owned by another allocator. No counterpart in the
 * paper.
 * Same inputs, output and result as occri_orbitals, but the call's scratch (the
 * normalised coefficients and the orbitals before widening) lives in one static
 * device array of OCCRI_STATIC_SCRATCH_BYTES instead of the plan's workspaces; the
 * call makes no cudaMalloc, cudaFree or other allocating call.
 * A call needs 16*nk*nao*nocc bytes (rounded up to 256) plus 16*nk*nocc*F (FP64)
 * or 8*nk*nocc*F (mixed) bytes of it, F being N_g rounded up to a multiple of 64;
 * larger problems return OCCRI_EINVAL before anything is launched.
 * The first call on each device looks up the array's device address (with that device
 * current). All calls share the one
 * array and it keeps the previous call's contents (every byte a call reads it has
 * written first, so nothing needs clearing); calls whose work overlaps on the GPU --
 * on different streams, or from different host threads -- race on it and must be
 * serialised by the caller. */
int occri_orbitals_noalloc(const occri_plan *plan, const void *C_dev, void *psi_dev);

/* ---- Batches of cells: several uneven cells built by one graph launch ----
 * A batch builds several plans together: cells that may differ in size, k-mesh, basis,
 * kernel or precision, such as the five cells of a lattice-constant scan. On the first
 * occri_batch_build (and again whenever the caller's buffers change) the builds of all
 * cells are captured into one CUDA graph, each cell on its own branch, so that the cells
 * run concurrently; every call then launches that graph once on the batch's stream. No
 * counterpart in the paper, whose parallel loops run one cell at a time.
 * plans: nplans (>= 1) distinct plans, owned by the caller and alive while the batch
 *   exists; a batch build does not use their own streams, and their stage timing is off
 *   while the graph is captured.
 * cuda_stream: the stream the graph is launched on (a cudaStream_t, or NULL for the
 *   legacy default stream).
 * On success *out owns the batch (occri_batch_destroy); on failure *out is NULL. */
typedef struct occri_batch occri_batch;
int occri_batch_create(occri_batch **out, occri_plan *const *plans, int nplans,
                       void *cuda_stream);

/* One build of every cell of the batch. Each argument is an array of nplans device
 * pointers with the meaning and layout of the same argument of occri_k_build (entries of
 * KC_dev, K_dev and Ex_dev may be NULL; the arrays themselves may be NULL for "all
 * NULL"). Asynchronous on the batch's stream; the captured graph is reused while the
 * pointers stay the same. Returns OCCRI_EINVAL for a NULL C entry and OCCRI_ECUDA when the
 * capture or the launch fails. */
int occri_batch_build(occri_batch *batch, const void *const *C_dev, void *const *KC_dev,
                      void *const *K_dev, double *const *Ex_dev);

/* Synchronise the batch's stream and return the first device-side status of any cell
 * since the previous sync (as occri_plan_sync); *bad_cell and *bad_k (may be NULL)
 * receive the cell and the k index of an OCCRI_ENOTPD failure, else -1. */
int occri_batch_sync(occri_batch *batch, int *bad_cell, int *bad_k);

int occri_batch_destroy(occri_batch *batch);

/* ---- Fault injection, for tests of the error paths (no counterpart in the paper) ----
 * occri_plan_inject_fault(plan, OCCRI_FAULT_WAIT, ms): in the plan's following builds the
 *   producer warp of every bulk-copy accumulation pass (FP64 waves, and FP32 waves of
 *   nocc > 8, where shared memory allows) issues no copy, so each consumer's bounded
 *   wait runs out after ms milliseconds; the build then completes with a meaningless Y,
 *   and occri_plan_sync returns OCCRI_ETIMEOUT. No copy is in flight when a CTA leaves.
 *   occri_plan_inject_fault(plan, OCCRI_FAULT_NONE, ms) restores normal builds with
 *   wait limit ms (the default limit is 2000 ms). ms must lie in (0, 60000].
 * occri_debug_fail_allocation(n): the n-th device allocation made by the library from
 *   now on (n >= 1, any plan, any thread) fails as if the device were out of memory, so
 *   that the entry point making it returns OCCRI_ENOMEM after freeing what it took;
 *   n <= 0 disarms. */
enum { OCCRI_FAULT_NONE = 0, OCCRI_FAULT_WAIT = 1 };
int occri_plan_inject_fault(occri_plan *plan, int fault, double wait_limit_ms);
int occri_debug_fail_allocation(int nth);

/* Measured arithmetic peak of the current device (no counterpart in the paper; the
 * denominator of the roofline fraction of ALU-bound stages): kind 0 = FP64 FMA, 1 = FP32 FMA,
 * 2 = packed FP32 FMA (fma.rn.f32x2). Eight independent FMA chains per thread on every SM,
 * the best of three timed runs after one warm-up, CUDA events on the legacy default stream;
 * *tflops receives 2 x FMAs / time in TFLOP/s. Synchronises the device. */
int occri_measure_fma_peak(int kind, double *tflops);

const char *occri_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* OCCRI_H */
