"""Small fixed workloads for kernel profiling (ncu) and stage timing.

    python -m paper_2207_09028_gb300.prof --grid 60 --nocc 8 --mesh 1 1 1 --builds 2

builds a synthetic 2-atom cell with the given grid edge, Gamma-centred k-mesh
and occupied count, and runs `--builds` full exchange builds. With a 1x1x1 mesh
one build issues exactly one wave of each pair-transform pass, which is the unit
ncu captures; a 2x2x2 mesh adds waves with q = 1/2 on every axis (no tied bins),
like most waves of a 6x6x6 mesh. --timing prints per-stage CUDA-event times.

    python -m paper_2207_09028_gb300.prof --batch cfg4 --builds 5

times the five cells of the lattice-constant scan built one after the other on one
stream against the same cells built as one batch (one CUDA-graph launch per build).
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=60)
    ap.add_argument("--nocc", type=int, default=8)
    ap.add_argument("--mesh", type=int, nargs=3, default=[1, 1, 1])
    ap.add_argument("--builds", type=int, default=2)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--timing", action="store_true")
    ap.add_argument("--batch", default=None, help="time a multi-cell config as a batch")
    args = ap.parse_args()
    if args.batch:
        return batch_timing(args)
    import torch
    import paper_2207_09028_gb300 as occri
    from workloads import small_workload

    w = small_workload(a_ang=5.43, mesh=tuple(args.mesh), counts=(6, 4, 3, 2), lo=0.1, hi=20.0,
                       nocc=args.nocc, grid=(args.grid,) * 3, seed=77)
    plan = occri.Plan.from_workload(w, precision=args.precision)
    C = torch.from_numpy(w.C).cuda()
    if args.timing:
        plan.set_timing(1)
    for _ in range(args.builds):
        KC, K, Ex = plan.build(C)
    out = {"E_x": float(Ex.cpu()[0]), "info": plan.info()}
    if args.timing:
        out["stages"] = plan.stage_times()
    print(json.dumps(out))


def batch_timing(args):
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
    print(json.dumps({"config": args.batch, "cells": len(cells), "precision": args.precision,
                      "ms_per_build_one_by_one": ms_seq, "ms_per_build_batch": ms_batch,
                      "speedup": ms_seq / ms_batch,
                      "max_abs_dE_x_batch_vs_one_by_one": max(abs(a - b) for a, b in
                                                              zip(ex_seq, ex_batch))}))


if __name__ == "__main__":
    main()
