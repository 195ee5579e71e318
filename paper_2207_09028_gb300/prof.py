"""Small fixed workloads for kernel profiling (ncu) and stage timing.

    python -m paper_2207_09028_gb300.prof --grid 60 --nocc 8 --mesh 1 1 1 --builds 2

builds a synthetic 2-atom cell with the given grid edge, Gamma-centred k-mesh
and occupied count, and runs `--builds` full exchange builds. With a 1x1x1 mesh
one build issues exactly one wave of each pair-transform pass, which is the unit
ncu captures; a 2x2x2 mesh adds waves with q = 1/2 on every axis (no tied bins),
like most waves of a 6x6x6 mesh. --timing prints per-stage CUDA-event times.
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
    args = ap.parse_args()
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


if __name__ == "__main__":
    main()
