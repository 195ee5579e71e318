#!/usr/bin/env python
"""Throughput of the occ-RI-K exchange build: K-builds/s at 6x6x6 k, 350 AO.

One step = one full exchange build (steps a-f: AO/orbital evaluation, every
(k,k',i,j) pair-density FFT round trip with the Coulomb kernel, the contraction
and the FP64 ACE assembly) on the paper-scale synthetic cell: fcc a = 5.43 A,
2 atoms, 6x6x6 Gamma-centred k-mesh (216 k), 350 uncontracted s/p/d/f AOs,
nocc = 8, 60^3 grid, mixed precision with the tensor-core contraction. Inputs
(C, plan tables) are resident in HBM before the timed region; the orbital and
accumulator fields (3 GB each) exceed L2, so no flush is needed between steps.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle instead
(bounded sample on every host core, extrapolated to a full build).

Other modes (one JSON line per point; none is the headline):

    python bench.py --case 60 8 2 2 2 [--builds 2] [--precision mixed] [--timing]
        builds of a small fixed profiling cell (fcc a = 5.43 A, 2 atoms, 6/4/3/2 s/p/d/f
        shells per atom, exponents 0.1-20) with the given grid edge, nocc and Gamma-centred
        k-mesh: the unit that ncu captures. A 1x1x1 mesh gives one wave of each pass; a
        2x2x2 mesh adds waves with q = 1/2 on every axis, like most waves of a 6x6x6 mesh.
    python bench.py --batch cfg4 [--builds 5]
        the five lattice-constant cells one after another against one batch (graph) build.
    python bench.py --sweep nk|nao [--steps 1]
        K-builds/s of the bench cell at N_k = 1^3..6^3 (the N_k^2 scaling of Sec. III), or
        at nao 26..350 on the 6x6x6 mesh (basis-size dependence of Sec. III), with the
        fitted log-log slope.
    python bench.py --configs all|cfg1,cfg2,... [--steps 3]
        every config cell in FP64, mixed and mixed_tc: K-builds/s and the error against the
        stored oracle goldens (or, for the bench cell, against the FP64 GPU build).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one full mixed-precision wave (pass_a, pass_b reading the plan's
# kernel tables, and pass_cd), keyed by ("round_trip", grid edge, fields per wave, precision),
# from one ncu --set full capture per pass of the same launch shape (an off-diagonal 64-field
# wave at 60^3 of the 2x2x2-k profiling cell of `--case 60 8 2 2 2`; cold cache, each launch
# replayed alone).
TRAFFIC = {("round_trip", 60, 64, "mixed"): 425.0e6}

METRIC = "K-builds/s at 6x6x6 k, 350 AO; mixed vs FP64 GPU at |dE_x|<=1e-6 Ha/cell"
UNIT = "K-builds/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _tensor_peak():
    """Dense bf16 TFLOP/s (FP16 runs at the same tensor-core rate): the sustained figure of
    MEASURED_PEAKS.json, since the contraction is timed inside a multi-second build, else
    the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops_sustained" in d:
            return float(d["bf16_tflops_sustained"]), "measured bf16 sustained"
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured bf16 burst"
    return 1700.0, "fallback (sustained)"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle sample

def cpu_model() -> str:
    """The host CPU's model name (x86 'model name', Arm 'Model name' from lscpu)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _oracle_worker(job):
    """One worker's share of the oracle sample (runs in a spawned process, one BLAS thread).

    pairs: the Algorithm-3 loop over one k-point (its (k, k) block of nocc^2 FFT round trips
    on the full grid) with seeded random orbitals; aos: Bloch AOs for every k at two point
    counts; contract: the contraction of one k over `cpts` points. Returns wall seconds."""
    import oracle as O
    (lattice, xyz, sa, sl, sx, kfrac, grid, kind, omega, g0, nocc, nao, k, seed, npts,
     cpts) = job
    rng = np.random.default_rng(seed)
    ng = int(np.prod(grid))
    out = {}
    psi = rng.standard_normal((1, nocc, ng)) + 1j * rng.standard_normal((1, nocc, ng))
    t0 = time.perf_counter()
    O.occri_kc(lattice, grid, kfrac[k:k + 1], psi, None, kind, omega, g0)
    out["pairs"] = time.perf_counter() - t0
    allpts = O.grid_points(lattice, grid)
    out["aos"] = []
    for n in npts:
        sel = allpts[rng.choice(ng, n, replace=False)]
        t0 = time.perf_counter()
        O.bloch_aos(lattice, xyz, sa, sl, sx, kfrac, points=sel)
        out["aos"].append(time.perf_counter() - t0)
    chi = rng.standard_normal((1, nao, cpts)) + 1j * rng.standard_normal((1, nao, cpts))
    y = rng.standard_normal((1, nocc, cpts)) + 1j * rng.standard_normal((1, nocc, cpts))
    t0 = time.perf_counter()
    O.contract_kc(lattice, chi, y)
    out["contract"] = time.perf_counter() - t0
    return out


class OracleSampler:
    """The FP64 oracle as it stands, timed on every host core on a bounded sample of one
    build and extrapolated to the whole build.

    Each of `workers` spawned processes (one BLAS thread each) runs, at the same time:
    the oracle's Algorithm-3 loop for one k-point of the workload (one (k, k) block of
    nocc^2 FFT round trips of the full grid; every block costs the same), the oracle's
    Bloch AOs of all k at npts[0] and npts[1] grid points (fitted as a + b n per worker),
    and its contraction of one k over cpts points. A build is N_k^2 blocks, N_g AO points
    and N_k contractions of N_g points, spread over the same workers.
    """

    def __init__(self, w, workers=None, npts=(32, 96), cpts=16384):
        import multiprocessing as mp
        self.w = w
        self.workers = workers or os.cpu_count() or 1
        self.npts, self.cpts = npts, cpts
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.pool = mp.get_context("spawn").Pool(self.workers)
        self.calls = 0

    def sample(self):
        """(seconds per full build, sample description, wall seconds of the sample)."""
        import oracle as O
        w = self.w
        g0 = O.g0_value(w.kernel, w.omega, w.g0_mode)
        jobs = [(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac, w.grid,
                 w.kernel, w.omega, g0, w.nocc, w.nao, (self.calls * self.workers + i) % w.nk,
                 1000 * self.calls + i, self.npts, self.cpts) for i in range(self.workers)]
        self.calls += 1
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        nw = self.workers
        t_block = statistics.mean(r["pairs"] for r in res)        # one block on one core
        n0, n1 = self.npts
        slope = statistics.mean(max(0.0, (r["aos"][1] - r["aos"][0]) / (n1 - n0)) for r in res)
        icpt = statistics.mean(max(0.0, r["aos"][0] - slope * n0) for r in res)
        t_contract = statistics.mean(r["contract"] for r in res) * w.ng / self.cpts
        # the build's work spread over nw cores
        total = (w.nk ** 2 * t_block + (nw * icpt + slope * w.ng) + w.nk * t_contract) / nw
        desc = (f"extrapolated: {nw} processes on {nw} cores ({cpu_model()}), each timing the "
                f"oracle's Algorithm-3 loop over one k-point (1 of {w.nk ** 2} (k,k') blocks, "
                f"{w.nocc ** 2} FFT round trips of {w.grid[0]}^3), its Bloch AOs of all {w.nk} k "
                f"at {n0} and {n1} points (a + b n) and its contraction of one k over "
                f"{self.cpts} points; scaled to {w.nk ** 2} blocks, {w.ng} points and {w.nk} "
                "contractions, divided over the cores")
        return total, desc, wall

    def close(self):
        self.pool.close()
        self.pool.join()


# ---------------------------------------------------------------- ranks

L2_BYTES = 129e6   # GB300 L2


def l2_note(nk: int, nocc: int, ng: int) -> str:
    """Whether the timed builds need an L2 flush: every build streams the orbital and
    accumulator fields (FP32 complex, fields padded to 64 points); when each is larger than
    L2, no data survives from one build to the next."""
    gb = nk * nocc * ((ng + 63) // 64 * 64) * 8
    if gb > L2_BYTES:
        return (f"no flush: orbital and accumulator fields (2 x {gb / 1e9:.2g} GB) exceed L2 "
                f"({L2_BYTES / 1e6:.0f} MB)")
    return (f"fields fit L2 (2 x {gb / 1e6:.2g} MB of {L2_BYTES / 1e6:.0f} MB): repeated builds "
            "run warm; small-cell rate, not a bandwidth figure")


def pair_waves(nk: int, nocc: int, fields_per_wave: int) -> int:
    """Waves of one build: (k, k) once per k, then blocks of up to nkp k' > k."""
    nkp = max(1, fields_per_wave // (nocc * nocc))
    return nk + sum((nk - 1 - k + nkp - 1) // nkp for k in range(nk))


def stage_ms_per_build(stages: dict, waves: int, steps: int) -> dict:
    """Per-build stage times. Pair-transform passes are timed on every `timing_every`-th
    wave only, so their sampled sums are scaled by (waves per build / sampled waves)."""
    out = {}
    for name, st in stages.items():
        if name.startswith("pair_"):
            out[name] = st["ms"] * waves / max(1, st["launches"])
        else:
            out[name] = st["ms"] / steps
    return out


def roofline(stages: dict, info: dict, edge: int, ng: int, nocc: int, hbm: float,
             peak_kind: str, tuning: dict = None):
    """Roofline of the dominant work, the pair round trip (steps c, d).

    Its unit is one transformed field; each of the two 3-D transforms reads and writes the
    field once, so the streaming model is 2 x 2 x 8 B x N_g = 32 N_g bytes per field in
    FP32 (c64). A round trip runs as three launches over a wave of fields (pass_a, whose extra
    CTAs fill the kernel tables, pass_b and the fused pass_cd; FP64 or nocc > 8: pass_c and
    pass_d instead);
    waves go round-robin over the plan's streams, so the achieved rate is taken over the wall time
    of the whole wave loop (the `pairs` stage: CUDA events on the plan's stream around the
    loop, every timed build). The per-pass split comes from the sampled waves, run alone.
    """
    loop = stages.get("pairs", {})
    if not loop.get("launches") or loop.get("ms", 0) <= 0:
        return None
    pair = [s_ for s_ in ("pair_a", "pair_b", "pair_c") if s_ in stages]
    rt_ms = sum(stages[s_]["ms"] for s_ in pair)
    fields = loop["units"]
    achieved = 32.0 * ng * fields / (loop["ms"] / 1e3) / 1e9
    fpw = int(info["fields_per_wave"])
    mixed = int(info.get("precision", 1)) in (1, 2)   # OCCRI_MIXED, OCCRI_MIXED_TC
    tuning = tuning or {}
    # FP32 waves of nocc <= 8 fuse passes C and D unless the tuning splits them
    fused = mixed and nocc <= 8 and not tuning.get("split_cd", 0)
    passes = ("pass_a (with the kernel tables) + pass_b + pass_cd" if fused
              else "pass_a (with the kernel tables) + pass_b + pass_c + pass_d")
    nstreams = int(tuning.get("streams", 3))
    return {"kernel": f"pair round trip: {passes} over waves of {fpw} fields of {edge}^3 "
                      f"({nstreams} streams)",
            "bound": "hbm", "achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / hbm,
            "traffic": (TRAFFIC.get(("round_trip", edge, fpw, "mixed")) if fused else None),
            "bytes_per_launch": 32.0 * ng * fpw,
            "ms_per_launch": loop["ms"] * fpw / fields,
            "pass_ms_share": ({s_: stages[s_]["ms"] / rt_ms for s_ in pair} if rt_ms > 0
                              else None)}


def pair_field_flops(ng: int) -> float:
    """Nominal arithmetic of one pair field: two 3-D transforms at the radix-2 count
    5 N_g log2 N_g each, plus pair formation (a complex product), the kernel multiply (real
    times complex) and the two accumulations (two complex multiply-adds): 24 N_g."""
    return (10.0 * np.log2(ng) + 24.0) * ng


def alu_roofline(fields: float, ng: int, ms: float, peak_tflops: float, kind: str):
    """Roofline of a pair loop bound by arithmetic (the FP64 path): nominal flops of the
    build's fields over its time, against the measured FMA rate of that precision."""
    if not peak_tflops or ms <= 0:
        return None
    achieved = pair_field_flops(ng) * fields / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "peak_kind": f"measured {kind} FMA loop",
            "flops_per_field": pair_field_flops(ng)}


# one stage of the tensor-core contraction: three FP16 MMAs (hi.hi, hi.lo, lo.hi) of
# M = 128 AO rows, N = 192 real columns (96 complex), K = 32 grid points


def tensor_roofline(info: dict, contract_ms: float, peak_tflops: float, peak_kind: str,
                    stage_ms: float = 0.0):
    """Roofline of the tensor-core contraction: the MMA flops of its stages over the time of
    its GEMM kernels (CUDA events around each launch), against the measured dense bf16 rate
    (FP16 runs at the same rate on these tensor cores). `stage_ms`, the whole contraction
    stage (with the Y conversion and the A-block generation), is reported beside it."""
    st = int(info.get("tc_stages", 0))
    fps = float(info.get("tc_flops_per_stage", 0.0))
    if not info.get("contraction_tc") or st <= 0 or contract_ms <= 0 or fps <= 0:
        return None
    achieved = fps * st / (contract_ms / 1e3) / 1e12
    return {"kernel": "contract_tc_kernel (tcgen05.mma kind::f16, FP16 hi/lo x3, FP32 accumulate)",
            "bound": "tensor", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "peak_kind": peak_kind, "stages": st,
            "flops_per_stage": fps, "gemm_ms": contract_ms, "stage_ms": stage_ms,
            "frac_of_stage": (fps * st / (stage_ms / 1e3) / 1e12 / peak_tflops
                              if stage_ms > 0 else None),
            "useful_frac": achieved / 3.0 / peak_tflops}


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The slowest rank's time (replicas: every rank runs the whole build on its GPU)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, ms: float) -> float:
    """Builds per second of the whole job: every rank completes `steps` builds in `ms`."""
    return world * steps / (ms / 1e3)


# ---------------------------------------------------------------- other modes

def profiling_cell(edge: int, nocc: int, mesh, seed: int = 77):
    """The small fixed cell that ncu captures (see the module docstring)."""
    from workloads import small_workload
    return small_workload(a_ang=5.43, mesh=tuple(mesh), counts=(6, 4, 3, 2), lo=0.1, hi=20.0,
                          nocc=nocc, grid=(edge,) * 3, seed=seed)


def run_case(args):
    import torch
    import paper_2207_09028_gb300 as occri
    edge, nocc, m1, m2, m3 = args.case
    w = profiling_cell(edge, nocc, (m1, m2, m3))
    plan = occri.Plan.from_workload(w, precision=args.precision)
    C = torch.from_numpy(w.C).cuda()
    if args.timing:
        plan.set_timing(1)
    for _ in range(args.builds):
        KC, K, Ex = plan.build(C)
    out = {"mode": "case", "E_x": float(Ex.cpu()[0]), "info": plan.info()}
    if args.timing:
        out["stages"] = plan.stage_times()
    print(json.dumps(out), flush=True)


def run_batch(args):
    import torch
    import paper_2207_09028_gb300 as occri
    from workloads import config

    cells = config(args.batch)
    plans = [occri.Plan.from_workload(w, precision=args.precision) for w in cells]
    Cs = [torch.from_numpy(w.C).cuda() for w in cells]
    Exs = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in cells]
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()                                    # warm-up (and graph capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.builds):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.builds

    def one_by_one():
        for pl, C, E in zip(plans, Cs, Exs):
            pl.k_build(C, None, None, E, sync=False)

    ms_seq = timed(one_by_one)
    ex_seq = [float(e.cpu()[0]) for e in Exs]
    batch = occri.Batch(plans)
    ms_batch = timed(lambda: batch.build(Cs, None, None, Exs, sync=False))
    batch.sync()
    ex_batch = [float(e.cpu()[0]) for e in Exs]
    print(json.dumps({"mode": "batch", "config": args.batch, "cells": len(cells),
                      "precision": args.precision, "ms_per_build_one_by_one": ms_seq,
                      "ms_per_build_batch": ms_batch, "speedup": ms_seq / ms_batch,
                      "max_abs_dE_x_batch_vs_one_by_one": max(abs(a - b) for a, b in
                                                              zip(ex_seq, ex_batch))}),
          flush=True)


# nao sweep: shells per atom (s, p, d, f) growing to the bench cell's 20/14/10/9 (nao 350)
NAO_SWEEP = [(7, 2, 0, 0), (9, 6, 5, 0), (15, 10, 11, 0), (20, 14, 10, 3), (20, 14, 10, 9)]


def loglog_slope(xs, ys) -> float:
    """Least-squares slope of log y against log x."""
    lx, ly = np.log(np.asarray(xs, float)), np.log(np.asarray(ys, float))
    return float(np.polyfit(lx, ly, 1)[0])


def run_sweep(args):
    """K-builds/s of the bench cell across N_k (1^3..6^3) or nao (26..350 at 6x6x6 k)."""
    import torch
    import paper_2207_09028_gb300 as occri
    from workloads import synthetic as syn

    stream = torch.cuda.current_stream()
    pts = []
    if args.sweep == "nk":
        cases = [dict(mesh=(n, n, n), counts=(20, 14, 10, 9)) for n in range(1, 7)]
    else:
        cases = [dict(mesh=(6, 6, 6), counts=c) for c in NAO_SWEEP]
    for c in cases:
        w = syn._build("sweep", 5.43, c["mesh"], c["counts"], 0.06, 40.0, 8, (60, 60, 60),
                       "coulomb", 0.0, 0, 1050)
        plan = occri.Plan.from_workload(w, precision=args.precision)
        C = torch.from_numpy(w.C).cuda()
        Ex = torch.zeros(1, dtype=torch.float64, device=C.device)
        for _ in range(max(1, args.warmup)):
            plan.k_build(C, None, None, Ex, sync=False)
        plan.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.k_build(C, None, None, Ex, sync=False)
        e1.record(stream)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        pt = {"mode": "sweep", "sweep": args.sweep, "nk": w.nk, "nao": w.nao, "nocc": w.nocc,
              "grid": list(w.grid), "precision": args.precision, "ms_per_build": ms,
              "K_builds_per_s": 1e3 / ms, "E_x": float(Ex.cpu()[0])}
        print(json.dumps(pt), flush=True)
        pts.append(pt)
        plan.close()
        del plan, C
        torch.cuda.empty_cache()
    key = "nk" if args.sweep == "nk" else "nao"
    sel = [p_ for p_ in pts if p_["nk"] > 1] if key == "nk" else pts
    print(json.dumps({"mode": "sweep", "sweep": args.sweep,
                      "loglog_slope_ms_vs_" + key: loglog_slope([p_[key] for p_ in sel],
                                                                [p_["ms_per_build"] for p_ in sel]),
                      "points": len(sel)}), flush=True)


def run_configs(args):
    """Every config cell in every precision: K-builds/s (CUDA events, after warm-up) and the
    error against the stored oracle goldens (tests/golden, written by make_golden.py from the
    oracle) -- |dE_x| and max|dK_{mu i}| -- or, for the bench cell (no golden), against the
    FP64 GPU build. One JSON line per (config, precision)."""
    import numpy as np
    import torch
    import paper_2207_09028_gb300 as occri
    from workloads import config

    stream = torch.cuda.current_stream()
    names = ["cfg1", "cfg2", "cfg3_erfc", "cfg3_erf", "cfg4", "cfg5"]
    if args.configs != "all":
        names = args.configs.split(",")
    for name in names:
        cells = config(name)
        cells = cells if isinstance(cells, list) else [cells]
        for w in cells:
            gpath = os.path.join(ROOT, "tests", "golden", f"{w.name}.npz")
            gold = dict(np.load(gpath)) if os.path.exists(gpath) else None
            C = torch.from_numpy(w.C).cuda()
            ref = None
            for prec in ("fp64", "mixed", "mixed_tc"):
                plan = occri.Plan.from_workload(w, precision=prec)
                steps = 1 if (prec == "fp64" and w.nk * w.grid[0] ** 3 > 2e7) else args.steps
                KC, _, Ex = plan.build(C, want_k=False)        # warm-up
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    plan.k_build(C, KC, None, Ex, sync=False)
                e1.record(stream)
                plan.sync()
                ms = e0.elapsed_time(e1) / steps
                kc = KC.cpu().numpy()
                ex = float(Ex.cpu()[0])
                if prec == "fp64":
                    ref = (kc, ex)
                pt = {"mode": "configs", "config": w.name, "precision": prec, "nk": w.nk,
                      "nao": w.nao, "nocc": w.nocc, "grid": w.grid[0], "kernel": w.kernel,
                      "ms_per_build": ms, "K_builds_per_s": 1e3 / ms, "E_x": ex,
                      "contraction_tc": bool(plan.contraction_tc)}
                if gold is not None:
                    pt["vs"] = "oracle golden"
                    pt["abs_dE_x"] = abs(ex - float(gold["ex"]))
                    pt["max_abs_dK"] = float(np.abs(kc - gold["kc"]).max())
                    pt["max_rel_dK"] = pt["max_abs_dK"] / float(np.abs(gold["kc"]).max())
                elif prec != "fp64":
                    pt["vs"] = "FP64 GPU build"
                    pt["abs_dE_x"] = abs(ex - ref[1])
                    pt["max_abs_dK"] = float(np.abs(kc - ref[0]).max())
                print(json.dumps(pt), flush=True)
                plan.close()
                del plan, KC, Ex
                torch.cuda.empty_cache()


# ---------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="occri", choices=["occri", "reference"])
    ap.add_argument("--workload", default="cfg5")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--timing-every", type=int, default=61)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", type=int, nargs=5, default=None,
                    metavar=("EDGE", "NOCC", "M1", "M2", "M3"))
    ap.add_argument("--batch", default=None)
    ap.add_argument("--sweep", default=None, choices=["nk", "nao"])
    ap.add_argument("--builds", type=int, default=2)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--bench-precision", default="mixed_tc",
                    help="precision of the headline builds (mixed_tc: tensor-core contraction)")
    ap.add_argument("--timing", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="time plain launches instead of the build's CUDA graph")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default launch configuration of the pair loop")
    ap.add_argument("--configs", default=None,
                    help="'all' or a comma list: every precision of those config cells")
    args = ap.parse_args()
    if args.configs:
        return run_configs(args)
    if args.case:
        return run_case(args)
    if args.batch:
        return run_batch(args)
    if args.sweep:
        return run_sweep(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from workloads import config
    w = config(args.workload)
    if isinstance(w, list):
        raise SystemExit("bench workloads are single cells")
    cfg = {"workload": (f"{args.workload}: fcc a=5.43 A, 2 atoms, {w.nk} k ({round(w.nk ** (1 / 3))}^3 "
                        f"Gamma-centred), nao {w.nao}, nocc {w.nocc}, grid {w.grid[0]}^3, "
                        f"{w.kernel} kernel"),
           "nk": w.nk, "nao": w.nao, "nocc": w.nocc, "grid": list(w.grid), "kernel": w.kernel,
           "precision": ("mixed_tc: FP32 AO/orbitals/FFTs/Y; contraction on the tensor cores "
                         "(FP16 hi/lo x3, FP32 accumulate, FP64 sums); FP64 assembly, E_x"
                         if args.bench_precision == "mixed_tc" else
                         "mixed: FP32 AO/orbitals/FFTs/Y, FP64 contraction sum, assembly, E_x"),
           "l2": l2_note(w.nk, w.nocc, w.ng),
           "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        sampler = OracleSampler(w)
        cfg = dict(cfg, precision=f"FP64 CPU oracle (numpy), {sampler.workers} cores")
        samples = []
        for _ in range(args.warmup + args.steps):
            t, desc, wall = sampler.sample()
            samples.append(t)
        sampler.close()
        t = statistics.median(samples[args.warmup:]) if args.steps else samples[-1]
        val = 1.0 / t
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                          "extrapolated": True,
                          "step": "one bounded sample of a build on every host core, "
                                  "extrapolated to the whole build (see cpu_baseline.sample)",
                          "cpu_baseline": {"value": val, "unit": UNIT, "cores": sampler.workers,
                                           "kind": "oracle", "sample": desc,
                                           "cpu": cpu_model()},
                          "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return

    import torch

    import paper_2207_09028_gb300 as occri

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    plan = occri.Plan.from_workload(w, precision=args.bench_precision)
    # the pair loop's launch configuration, timed once per shape before the timed region
    tuning = None if args.no_autotune else plan.autotune()
    C = torch.from_numpy(w.C).to(dev)
    KC = torch.empty((w.nk, w.nao, w.nocc), dtype=torch.complex128, device=dev)
    K = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device=dev)
    Ex = torch.zeros(1, dtype=torch.float64, device=dev)
    # the whole build as one CUDA graph (occri_batch_* with this one cell: the first call
    # captures it, every later call is one graph launch), unless --no-graph
    batch = None if args.no_graph else occri.Batch([plan], stream=stream.cuda_stream)

    def one_build():
        if batch is not None:
            batch.build([C], [KC], [K], [Ex], sync=False)
        else:
            plan.k_build(C, KC, K, Ex, sync=False)

    def sync_builds():
        if batch is not None:
            batch.sync()
        plan.sync()

    for _ in range(args.warmup):
        one_build()
    sync_builds()
    ex_mixed = float(Ex.cpu()[0])

    torch.cuda.synchronize()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            one_build()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    sync_builds()
    # stage spans (events around the stages and the whole pair loop, no wave sampled or
    # isolated) from one more build with plain launches, untimed for the headline
    plan.set_timing(-1)
    plan.k_build(C, KC, K, Ex, sync=False)
    plan.sync()
    stages = plan.stage_times()
    # one more build, untimed for the headline, with every timing_every-th wave run alone
    # and timed pass by pass: the split of the round trip between the passes
    if args.timing_every > 0:
        plan.set_timing(args.timing_every)
        plan.k_build(C, KC, K, Ex, sync=False)
        plan.sync()
        sampled = plan.stage_times()
        for name in ("pair_a", "pair_b", "pair_c"):
            stages[name] = sampled[name]
    plan.set_timing(0)
    ms = max_over_ranks(ms, dist, dev)
    ms_per_step = ms / args.steps
    value = job_throughput(world, args.steps, ms)
    info = plan.info()

    waves = pair_waves(w.nk, w.nocc, int(info["fields_per_wave"]))
    stage_share = stage_ms_per_build(stages, waves, 1)
    for name in ("pair_a", "pair_b", "pair_c"):   # from the one sampled build
        if name in stages:
            stage_share[name] = stages[name]["ms"] * waves / max(1, stages[name]["launches"])
    hbm, peak_kind = _peaks()
    roof = roofline(stages, info, w.grid[0], w.ng, w.nocc, hbm, peak_kind,
                    tuning if tuning is not None else plan.tuning())
    tpeak, tpeak_kind = _tensor_peak()
    contraction_roof = tensor_roofline(info, stage_share.get("contract_gemm", 0.0), tpeak,
                                       tpeak_kind, stage_share.get("contract", 0.0))

    out = {"impl": "occri", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": cfg, "roofline": roof,
           "gpu_launches": int(info["launches_per_build"]) * args.steps,
           "tuning": tuning if tuning is not None else plan.tuning(),
           "launch": ("one CUDA graph per build (occri_batch_* with this cell)" if batch is not None
                      else "plain launches (occri_k_build)"),
           "stage_ms_per_build": stage_share, "E_x_mixed": ex_mixed,
           "roofline_contraction": contraction_roof}
    clocks = clk.summary()
    out["clocks"] = clocks

    # end to end through the host entry point (pinned host buffers, copies timed)
    if args.e2e_steps > 0:
        import ctypes
        Ch = torch.from_numpy(w.C).pin_memory()
        KCh = torch.empty((w.nk, w.nao, w.nocc), dtype=torch.complex128).pin_memory()
        Kh = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128).pin_memory()
        Exh = torch.zeros(1, dtype=torch.float64).pin_memory()
        lib = occri.load_library()
        plan.set_stream()
        call = lambda: lib.occri_k_build_host(plan._h, ctypes.c_void_p(Ch.data_ptr()),
                                              ctypes.c_void_p(KCh.data_ptr()),
                                              ctypes.c_void_p(Kh.data_ptr()),
                                              ctypes.c_void_p(Exh.data_ptr()))
        assert call() == 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            assert call() == 0
        t1 = time.perf_counter()
        out["e2e"] = {"value": world * args.e2e_steps / (t1 - t0), "unit": UNIT,
                      "h2d_bytes_per_step": Ch.numel() * 16,
                      "d2h_bytes_per_step": (KCh.numel() + Kh.numel()) * 16 + 8,
                      "steps": args.e2e_steps}

    # the plain FP64 GPU path on the same workload
    if args.fp64_steps > 0:
        del K
        torch.cuda.empty_cache()
        p64 = occri.Plan.from_workload(w, precision="fp64")
        Ex64 = torch.zeros(1, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            p64.k_build(C, None, None, Ex64, sync=False)
        e1.record(stream)
        p64.sync()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        ex64 = float(Ex64.cpu()[0])
        peaks = {k: occri.measure_fma_peak(k) for k in ("fp64", "fp32", "fp32x2")}
        fields = stages.get("pairs", {}).get("units", 0.0)   # one build with stage spans
        out["fp64_gpu"] = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64,
                           "steps": args.fp64_steps, "E_x": ex64,
                           "mixed_speedup": ms64 / ms_per_step,
                           "abs_dE_x_mixed_vs_fp64": abs(ex_mixed - ex64),
                           "roofline_whole_build": alu_roofline(fields, w.ng, ms64,
                                                                peaks["fp64"], "fp64")}
        out["alu_peaks_tflops"] = peaks
        p64.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sampler = OracleSampler(w)
        t, desc, wall = sampler.sample()
        sampler.close()
        out["cpu_baseline"] = {"value": 1.0 / t, "unit": UNIT, "cores": sampler.workers,
                               "kind": "oracle", "sample": desc, "sample_wall_s": wall,
                               "cpu": cpu_model()}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
