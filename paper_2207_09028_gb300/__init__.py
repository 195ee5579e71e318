"""GB300-native occ-RI-K exact-exchange build (arXiv:2207.09028).

Thin Python binding over the C ABI in ``include/occri.h`` (``liboccri.so``).
Every step of the exchange build runs in the library's CUDA kernels; this
module only marshals arguments (torch tensors -> device pointers, the current
CUDA stream). There is no CPU fallback: if the library is missing, importing
the entry points raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboccri.so")

OCCRI_OK = 0
OCCRI_EINVAL = 1
OCCRI_ENOMEM = 2
OCCRI_ENOTPD = 3
OCCRI_ECUDA = 4
OCCRI_ETIMEOUT = 5
OCCRI_EUNSUPPORTED = 6

OCCRI_COULOMB, OCCRI_ERFC, OCCRI_ERF = 0, 1, 2
OCCRI_FP64, OCCRI_MIXED, OCCRI_MIXED_TC = 0, 1, 2
OCCRI_COULOMB_TRUNC, OCCRI_ERF_TRUNC = 3, 4
KERNELS = {"coulomb": OCCRI_COULOMB, "erfc": OCCRI_ERFC, "erf": OCCRI_ERF,
           "coulomb_trunc": OCCRI_COULOMB_TRUNC, "erf_trunc": OCCRI_ERF_TRUNC}
PRECISIONS = {"fp64": OCCRI_FP64, "mixed": OCCRI_MIXED, "mixed_tc": OCCRI_MIXED_TC}


class occri_cell(ctypes.Structure):
    _fields_ = [("a", (ctypes.c_double * 3) * 3), ("natm", ctypes.c_int),
                ("xyz", ctypes.POINTER(ctypes.c_double))]


class occri_basis(ctypes.Structure):
    _fields_ = [("nshell", ctypes.c_int), ("atom", ctypes.POINTER(ctypes.c_int)),
                ("l", ctypes.POINTER(ctypes.c_int)), ("alpha", ctypes.POINTER(ctypes.c_double))]


class occri_kmesh(ctypes.Structure):
    _fields_ = [("nk", ctypes.c_int), ("kfrac", ctypes.POINTER(ctypes.c_double))]


class occri_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("omega", ctypes.c_double), ("g0_mode", ctypes.c_int)]


class occri_tune_t(ctypes.Structure):
    _fields_ = [("k_per_wave", ctypes.c_int), ("streams", ctypes.c_int),
                ("pass_b_div", ctypes.c_int), ("split_cd", ctypes.c_int),
                ("wave_tables", ctypes.c_int), ("us_per_field", ctypes.c_double),
                ("us_default", ctypes.c_double), ("candidates", ctypes.c_int)]


OCCRI_TUNE_FORCE = 1


class occri_plan_info_t(ctypes.Structure):
    _fields_ = [("nk", ctypes.c_int), ("nao", ctypes.c_int), ("nocc", ctypes.c_int),
                ("natm", ctypes.c_int), ("nshell", ctypes.c_int), ("grid", ctypes.c_int * 3),
                ("ng", ctypes.c_longlong), ("precision", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("fields_per_wave", ctypes.c_int),
                ("launches_per_build", ctypes.c_longlong), ("contraction_tc", ctypes.c_int),
                ("tc_stages", ctypes.c_longlong), ("tc_flops_per_stage", ctypes.c_double)]


EXPORTED = ["occri_plan_create", "occri_plan_destroy", "occri_plan_info", "occri_plan_set_stream",
            "occri_plan_sync", "occri_k_build", "occri_k_build_host", "occri_orbitals",
            "occri_vjp", "occri_plan_set_timing", "occri_plan_stage_times", "occri_orbitals_noalloc",
            "occri_vjp_full", "occri_batch_create", "occri_batch_build", "occri_batch_sync",
            "occri_batch_destroy", "occri_k_build_once", "occri_plan_inject_fault",
            "occri_debug_fail_allocation", "occri_measure_fma_peak",
            "occri_k_assemble_paper", "occri_k_build_conduction", "occri_plan_autotune",
            "occri_plan_tuning", "occri_plan_set_tuning", "occri_status_string"]

OCCRI_FAULT_NONE, OCCRI_FAULT_WAIT = 0, 1

STAGES = ["orbitals", "pair_a", "pair_b", "pair_c", "contract", "assemble", "pairs",
          "contract_gemm"]

_lib_handle = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liboccri.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           "g.build()'` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.occri_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(occri_cell),
                                      ctypes.POINTER(occri_kmesh), ctypes.POINTER(occri_basis), ip,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(occri_kernel),
                                      ip, vp]
    lib.occri_plan_destroy.argtypes = [vp]
    lib.occri_plan_info.argtypes = [vp, ctypes.POINTER(occri_plan_info_t)]
    lib.occri_plan_set_stream.argtypes = [vp, vp]
    lib.occri_plan_sync.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.occri_k_build.argtypes = [vp, vp, vp, vp, vp]
    lib.occri_k_build_host.argtypes = [vp, vp, vp, vp, vp]
    lib.occri_orbitals.argtypes = [vp, vp, vp]
    lib.occri_vjp.argtypes = [vp, vp, ctypes.c_double, vp, vp]
    lib.occri_vjp_full.argtypes = [vp, vp, ctypes.c_double, vp, vp, vp, vp]
    lib.occri_plan_set_timing.argtypes = [vp, ip]
    lib.occri_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_double)]
    lib.occri_orbitals_noalloc.argtypes = [vp, vp, vp]
    lib.occri_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ip, vp]
    lib.occri_batch_build.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.occri_batch_sync.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.occri_batch_destroy.argtypes = [vp]
    lib.occri_k_build_once.argtypes = [ctypes.POINTER(occri_cell), ctypes.POINTER(occri_kmesh),
                                       ctypes.POINTER(occri_basis), vp, ip,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(occri_kernel),
                                       ip, vp, vp, vp]
    lib.occri_plan_inject_fault.argtypes = [vp, ip, ctypes.c_double]
    lib.occri_debug_fail_allocation.argtypes = [ip]
    lib.occri_measure_fma_peak.argtypes = [ip, dp]
    lib.occri_k_assemble_paper.argtypes = [vp, ip, vp, vp, vp, vp]
    lib.occri_plan_autotune.argtypes = [vp, ip, ctypes.POINTER(occri_tune_t)]
    lib.occri_plan_tuning.argtypes = [vp, ctypes.POINTER(occri_tune_t)]
    lib.occri_plan_set_tuning.argtypes = [vp, ctypes.POINTER(occri_tune_t)]
    lib.occri_k_build_conduction.argtypes = [vp, vp, vp, vp]
    lib.occri_status_string.argtypes = [ip]
    lib.occri_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "occri_status_string":
            getattr(lib, name).restype = ctypes.c_int
    _lib_handle = lib
    return lib


class OccriError(RuntimeError):
    def __init__(self, status: int, what: str, bad_k: int = -1):
        msg = load_library().occri_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status}" + (f", k={bad_k})" if bad_k >= 0 else ")"))
        self.status = status
        self.bad_k = bad_k


def _check(status: int, what: str):
    if status != OCCRI_OK:
        raise OccriError(status, what)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _problem_structs(lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac, grid, kernel,
                     omega, g0_mode, precision) -> dict:
    """The C structs of occri_plan_create / occri_k_build_once (with the numpy arrays they
    point into, which must outlive the call)."""
    lattice = np.ascontiguousarray(lattice, dtype=np.float64)
    keep = dict(xyz=np.ascontiguousarray(xyz, dtype=np.float64),
                atom=np.ascontiguousarray(shell_atom, dtype=np.int32),
                l=np.ascontiguousarray(shell_l, dtype=np.int32),
                alpha=np.ascontiguousarray(shell_alpha, dtype=np.float64),
                kfrac=np.ascontiguousarray(kfrac, dtype=np.float64).reshape(-1, 3))
    cell = occri_cell()
    for i in range(3):
        for j in range(3):
            cell.a[i][j] = float(lattice[i, j])
    cell.natm = keep["xyz"].shape[0]
    cell.xyz = keep["xyz"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    basis = occri_basis(len(keep["l"]), keep["atom"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        keep["l"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        keep["alpha"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    kmesh = occri_kmesh(keep["kfrac"].shape[0],
                        keep["kfrac"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    kern = occri_kernel(KERNELS[kernel] if isinstance(kernel, str) else int(kernel),
                        float(omega), int(g0_mode))
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return dict(keep, cell=cell, basis=basis, kmesh=kmesh, kernel=kern, grid=g, prec=prec)


def build_once(lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac, C, nocc: int, grid,
               kernel: str = "coulomb", omega: float = 0.0, g0_mode: int = 0,
               precision: str = "mixed", want_k: bool = True):
    """occri_k_build_once: plan, build and tear-down in one call. C is a complex128 CUDA
    tensor [nk, nao, nocc]; returns (K [nk, nao, nao] or None, E_x[1]) on C's device."""
    import torch
    lib = load_library()
    a = _problem_structs(lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac, grid, kernel,
                         omega, g0_mode, precision)
    if C.dtype != torch.complex128 or not C.is_cuda or not C.is_contiguous() or C.dim() != 3:
        raise ValueError("C must be a contiguous complex128 CUDA tensor [nk, nao, nocc]")
    nk, nao = C.shape[0], C.shape[1]
    K = torch.empty((nk, nao, nao), dtype=torch.complex128, device=C.device) if want_k else None
    Ex = torch.zeros(1, dtype=torch.float64, device=C.device)
    _check(lib.occri_k_build_once(ctypes.byref(a["cell"]), ctypes.byref(a["kmesh"]),
                                  ctypes.byref(a["basis"]), _ptr(C), int(nocc), a["grid"],
                                  ctypes.byref(a["kernel"]), a["prec"], _ptr(K), _ptr(Ex),
                                  _current_stream()), "occri_k_build_once")
    return K, Ex


FMA_KINDS = {"fp64": 0, "fp32": 1, "fp32x2": 2}


def measure_fma_peak(kind: str) -> float:
    """occri_measure_fma_peak: the device's measured FMA rate (TFLOP/s) for fp64, fp32 or
    packed fp32x2."""
    out = ctypes.c_double(0.0)
    _check(load_library().occri_measure_fma_peak(FMA_KINDS[kind], ctypes.byref(out)),
           "occri_measure_fma_peak")
    return out.value


def fail_allocation(nth: int):
    """occri_debug_fail_allocation: the nth device allocation from now fails (test hook)."""
    _check(load_library().occri_debug_fail_allocation(int(nth)), "occri_debug_fail_allocation")


class Plan:
    """An exchange-build plan (owns device workspaces; see occri_plan_create)."""

    def __init__(self, lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac, nocc: int, grid,
                 kernel: str = "coulomb", omega: float = 0.0, g0_mode: int = 0,
                 precision: str = "mixed", stream=None):
        lib = load_library()
        self._lib = lib
        self._args = _problem_structs(lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac,
                                      grid, kernel, omega, g0_mode, precision)
        cell, kmesh, basis, kern, g, prec = (self._args[k] for k in
                                             ("cell", "kmesh", "basis", "kernel", "grid", "prec"))
        handle = ctypes.c_void_p()
        st = lib.occri_plan_create(ctypes.byref(handle), ctypes.byref(cell), ctypes.byref(kmesh),
                                   ctypes.byref(basis), int(nocc), g, ctypes.byref(kern), prec,
                                   stream if stream is not None else _current_stream())
        _check(st, "occri_plan_create")
        self._h = handle
        info = occri_plan_info_t()
        _check(lib.occri_plan_info(self._h, ctypes.byref(info)), "occri_plan_info")
        self.nk, self.nao, self.nocc = info.nk, info.nao, info.nocc
        self.grid = tuple(info.grid)
        self.ng = info.ng
        self.precision = info.precision
        self.workspace_bytes = info.workspace_bytes
        self.fields_per_wave = info.fields_per_wave
        self.contraction_tc = bool(info.contraction_tc)
        self.kernel_kind = kern.kind

    @classmethod
    def from_workload(cls, w, precision: str = "mixed", **kw) -> "Plan":
        return cls(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac, w.nocc,
                   w.grid, w.kernel, w.omega, w.g0_mode, precision, **kw)

    # -- raw entry points -------------------------------------------------------
    def set_stream(self, stream=None):
        _check(self._lib.occri_plan_set_stream(self._h, stream or _current_stream()),
               "occri_plan_set_stream")

    def info(self) -> dict:
        info = occri_plan_info_t()
        _check(self._lib.occri_plan_info(self._h, ctypes.byref(info)), "occri_plan_info")
        return {f: (tuple(getattr(info, f)) if f == "grid" else getattr(info, f))
                for f, _ in occri_plan_info_t._fields_}

    def inject_fault(self, fault: int, wait_limit_ms: float = 2000.0):
        """occri_plan_inject_fault (test hook for the bounded-wait error path)."""
        _check(self._lib.occri_plan_inject_fault(self._h, int(fault), float(wait_limit_ms)),
               "occri_plan_inject_fault")

    def set_timing(self, every: int):
        _check(self._lib.occri_plan_set_timing(self._h, int(every)), "occri_plan_set_timing")

    def stage_times(self) -> dict:
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        units = (ctypes.c_double * n)()
        _check(self._lib.occri_plan_stage_times(self._h, ms, cnt, units), "occri_plan_stage_times")
        return {STAGES[i]: dict(ms=ms[i], launches=cnt[i], units=units[i]) for i in range(n)}

    def sync(self):
        bad = ctypes.c_int(-1)
        st = self._lib.occri_plan_sync(self._h, ctypes.byref(bad))
        if st != OCCRI_OK:
            raise OccriError(st, "occri_plan_sync", bad.value)

    def k_build(self, C, KC=None, K=None, Ex=None, sync: bool = True):
        """occri_k_build on device tensors (complex128 C [nk,nao,nocc]); returns (KC, K, Ex)."""
        import torch
        self._check_c(C)
        self.set_stream()
        _check(self._lib.occri_k_build(self._h, _ptr(C), _ptr(KC), _ptr(K), _ptr(Ex)),
               "occri_k_build")
        if sync:
            self.sync()
        return KC, K, Ex

    def autotune(self, force: bool = False) -> dict:
        """occri_plan_autotune: time the pair loop's launch configurations, keep the fastest."""
        t = occri_tune_t()
        self.set_stream()
        _check(self._lib.occri_plan_autotune(self._h, OCCRI_TUNE_FORCE if force else 0,
                                             ctypes.byref(t)), "occri_plan_autotune")
        return {f: getattr(t, f) for f, _ in occri_tune_t._fields_}

    def tuning(self) -> dict:
        """occri_plan_tuning: the current launch configuration of the pair loop."""
        t = occri_tune_t()
        _check(self._lib.occri_plan_tuning(self._h, ctypes.byref(t)), "occri_plan_tuning")
        return {f: getattr(t, f) for f, _ in occri_tune_t._fields_}

    def force_tuning(self, k_per_wave: int, streams: int, pass_b_div: int, split_cd: int,
                     wave_tables: int = 0):
        """occri_plan_set_tuning: set the pair loop's launch configuration by hand."""
        t = occri_tune_t(k_per_wave=k_per_wave, streams=streams, pass_b_div=pass_b_div,
                         split_cd=split_cd, wave_tables=wave_tables)
        _check(self._lib.occri_plan_set_tuning(self._h, ctypes.byref(t)), "occri_plan_set_tuning")

    def assemble_paper(self, S, C, KC, K=None):
        """occri_k_assemble_paper: K ~ PKP + PKQ + QKP from device tensors S [nk,nao,nao],
        C and KC [nk,nao,ncol] (complex128); returns K [nk,nao,nao]."""
        import torch
        ncol = int(C.shape[2])
        for t, shape in ((S, (self.nk, self.nao, self.nao)), (C, (self.nk, self.nao, ncol)),
                         (KC, (self.nk, self.nao, ncol))):
            if tuple(t.shape) != shape or t.dtype != torch.complex128 or not t.is_contiguous():
                raise ValueError(f"expected a contiguous complex128 tensor of shape {shape}")
        if K is None:
            K = torch.empty((self.nk, self.nao, self.nao), dtype=torch.complex128,
                            device=C.device)
        self.set_stream()
        _check(self._lib.occri_k_assemble_paper(self._h, ncol, _ptr(S), _ptr(C), _ptr(KC),
                                                _ptr(K)), "occri_k_assemble_paper")
        return K

    def k_build_conduction(self, plan_r: "Plan", C_all):
        """occri_k_build_conduction: the exchange columns K_{mu p} of the conduction bands
        that follow the occupied orbitals in C_all [nk,nao,nocc+nr] (this plan's orbitals),
        with plan_r the same cell with nocc = nr. Returns KCr [nk,nao,nr] (synchronised)."""
        import torch
        self._check_c(C_all)
        KCr = torch.empty((self.nk, self.nao, plan_r.nocc), dtype=torch.complex128,
                          device=C_all.device)
        self.set_stream()
        _check(self._lib.occri_k_build_conduction(self._h, plan_r._h, _ptr(C_all), _ptr(KCr)),
               "occri_k_build_conduction")
        return KCr

    def k_build_host(self, C_host: np.ndarray, want_k: bool = True):
        """occri_k_build_host: host (numpy or pinned torch) buffers in and out."""
        C_host = np.ascontiguousarray(C_host, dtype=np.complex128)
        kc = np.empty((self.nk, self.nao, self.nocc), dtype=np.complex128)
        k = np.empty((self.nk, self.nao, self.nao), dtype=np.complex128) if want_k else None
        ex = np.zeros(1, dtype=np.float64)
        _check(self._lib.occri_k_build_host(self._h, C_host.ctypes.data, kc.ctypes.data,
                                            None if k is None else k.ctypes.data, ex.ctypes.data),
               "occri_k_build_host")
        return kc, k, float(ex[0])

    def orbitals(self, C):
        import torch
        self._check_c(C)
        self.set_stream()
        psi = torch.empty((self.nk, self.nocc) + self.grid, dtype=torch.complex128, device=C.device)
        _check(self._lib.occri_orbitals(self._h, _ptr(C), _ptr(psi)), "occri_orbitals")
        self.sync()
        return psi

    def orbitals_noalloc(self, C, psi=None):
        """occri_orbitals_noalloc: as orbitals(), with the call's scratch in the library's
        static device array instead of the plan's workspaces (no allocation in the call)."""
        import torch
        self._check_c(C)
        self.set_stream()
        if psi is None:
            psi = torch.empty((self.nk, self.nocc) + self.grid, dtype=torch.complex128,
                              device=C.device)
        _check(self._lib.occri_orbitals_noalloc(self._h, _ptr(C), _ptr(psi)),
               "occri_orbitals_noalloc")
        self.sync()
        return psi

    def vjp(self, C, gEx: float, want_c: bool = True, want_omega: bool = True):
        import torch
        self.set_stream()
        gC = torch.empty_like(C) if want_c else None
        gw = torch.zeros(1, dtype=torch.float64, device=C.device) if want_omega else None
        _check(self._lib.occri_vjp(self._h, _ptr(C), float(gEx), _ptr(gC), _ptr(gw)), "occri_vjp")
        self.sync()
        return gC, gw

    def vjp_full(self, C, gEx: float = 0.0, gKC=None, gK=None, want_omega: bool = False):
        """occri_vjp_full: 2 dL/dC* (and dL/d omega) for the seeds dL/dE_x, dL/dKC, dL/dK
        (after a build). Returns gC, or (gC, d omega) with want_omega."""
        import torch
        self.set_stream()
        gC = torch.empty_like(C)
        gw = torch.zeros(1, dtype=torch.float64, device=C.device) if want_omega else None
        _check(self._lib.occri_vjp_full(self._h, _ptr(C), float(gEx), _ptr(gKC), _ptr(gK),
                                        _ptr(gC), _ptr(gw)), "occri_vjp_full")
        self.sync()
        return (gC, float(gw.cpu()[0])) if want_omega else gC

    def build(self, C, want_k: bool = True, sync: bool = True):
        """Allocate outputs and run one build: returns (KC, K or None, Ex[1])."""
        import torch
        self.generation = getattr(self, "generation", 0) + 1
        dev = C.device
        KC = torch.empty((self.nk, self.nao, self.nocc), dtype=torch.complex128, device=dev)
        K = torch.empty((self.nk, self.nao, self.nao), dtype=torch.complex128, device=dev) if want_k else None
        Ex = torch.zeros(1, dtype=torch.float64, device=dev)
        return self.k_build(C, KC, K, Ex, sync=sync)

    def _check_c(self, C):
        import torch
        if C.dtype != torch.complex128 or not C.is_cuda or not C.is_contiguous():
            raise ValueError("C must be a contiguous complex128 CUDA tensor")
        if tuple(C.shape) != (self.nk, self.nao, self.nocc):
            raise ValueError(f"C must have shape {(self.nk, self.nao, self.nocc)}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.occri_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several plans (cells) built by one CUDA-graph launch (see occri_batch_create)."""

    def __init__(self, plans: Sequence[Plan], stream=None):
        lib = load_library()
        self._lib = lib
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[pl._h.value for pl in self.plans])
        handle = ctypes.c_void_p()
        _check(lib.occri_batch_create(ctypes.byref(handle), arr, len(self.plans),
                                      stream if stream is not None else _current_stream()),
               "occri_batch_create")
        self._h = handle

    def build(self, Cs, KCs=None, Ks=None, Exs=None, sync: bool = True):
        """One build of every cell; Cs etc. are lists of device tensors (or None)."""
        n = len(self.plans)
        for pl, C in zip(self.plans, Cs):
            pl._check_c(C)

        def arr(ts):
            if ts is None:
                return None
            return (ctypes.c_void_p * n)(*[None if t is None else t.data_ptr() for t in ts])

        _check(self._lib.occri_batch_build(self._h, arr(Cs), arr(KCs), arr(Ks), arr(Exs)),
               "occri_batch_build")
        if sync:
            self.sync()
        return KCs, Ks, Exs

    def sync(self):
        cell, k = ctypes.c_int(-1), ctypes.c_int(-1)
        st = self._lib.occri_batch_sync(self._h, ctypes.byref(cell), ctypes.byref(k))
        if st != OCCRI_OK:
            raise OccriError(st, f"occri_batch_sync (cell {cell.value})", k.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.occri_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exchange_energy(plan: Plan, C, omega=None):
    """E_x(C[, omega]) as a differentiable torch scalar (backward = occri_vjp).

    Gradients: C in the conjugate-Wirtinger convention, (4/N_k) K_{mu i}(k) times
    the incoming gradient; omega via the hand-written d v/d omega pass. omega
    must equal the plan's omega (it is an input only so that autograd can
    route d E_x/d omega).
    """
    import torch

    class _ExchangeEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, Cin, w):
            KC, _, Ex = plan.build(Cin.detach().contiguous(), want_k=False)
            ctx.save_for_backward(Cin)
            ctx.has_w = w is not None
            ctx.w_device = w.device if w is not None else None
            return Ex[0].clone()

        @staticmethod
        def backward(ctx, g):
            (Cin,) = ctx.saved_tensors
            gC, gw = plan.vjp(Cin.detach().contiguous(), float(g),
                              want_c=ctx.needs_input_grad[0],
                              want_omega=ctx.has_w and ctx.needs_input_grad[1])
            gw_out = gw[0].to(device=ctx.w_device) if gw is not None else None
            return gC, gw_out

    return _ExchangeEnergy.apply(C, omega)


def exchange_build(plan: Plan, C, omega=None):
    """(K, E_x) of one build as differentiable torch tensors; backward = occri_vjp_full.

    K is the ACE-form exchange matrix [nk, nao, nao] and E_x a scalar. Any loss of K and
    E_x can be differentiated: gradients reach C (conjugate-Wirtinger convention, as
    PyTorch's complex autograd) and, when omega is given (a tensor equal to the plan's
    omega), omega through the kernel. backward recomputes the pair potentials (two round
    trips per unordered pair) and reuses the plan's K_{mu i}; if another build ran on the
    plan since this forward, it rebuilds first.
    """
    import torch

    class _ExchangeBuild(torch.autograd.Function):
        @staticmethod
        def forward(ctx, Cin, w):
            Cd = Cin.detach().contiguous()
            _, K, Ex = plan.build(Cd, want_k=True)
            ctx.save_for_backward(Cd)
            ctx.generation = plan.generation
            ctx.has_w = w is not None
            ctx.w_device = w.device if w is not None else None
            return K, Ex[0].clone()

        @staticmethod
        def backward(ctx, gK, gEx):
            (Cd,) = ctx.saved_tensors
            if plan.generation != ctx.generation:
                plan.build(Cd, want_k=False)
            want_w = ctx.has_w and ctx.needs_input_grad[1]
            g_e = 0.0 if gEx is None else float(gEx)
            gKc = None if gK is None else gK.contiguous()
            out = plan.vjp_full(Cd, g_e, None, gKc, want_omega=want_w)
            gC, gw = (out if want_w else (out, None))
            gw_out = (torch.tensor(gw, dtype=torch.float64, device=ctx.w_device)
                      if gw is not None else None)
            return (gC if ctx.needs_input_grad[0] else None), gw_out

    return _ExchangeBuild.apply(C, omega)


__all__ = ["Plan", "Batch", "OccriError", "load_library", "exchange_energy", "exchange_build",
           "build_once", "fail_allocation", "EXPORTED", "LIB_PATH"] + [
    n for n in globals() if n.startswith("OCCRI_")]
