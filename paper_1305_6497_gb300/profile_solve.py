"""Run refined solves of one workload under an NVTX range, for profilers.

    python -m paper_1305_6497_gb300.profile_solve --workload sphere256 --solves 1

Builds the target, tunes the launch schedule for its batch, runs `--warmup`
untimed solves and then `--solves` solves inside the NVTX range "timed" (a
profiler can restrict its capture to that range, e.g. ncu --nvtx
--nvtx-include "timed/").  Prints one JSON line with each solve's device time,
iterations and per-pass times.  The workloads are those of bench.py, plus
"zprobe": a 64x64x256 brick (2 RHS; 512-point z lines like the 256^3 sphere's,
a few hundred MB per spectral array) and "box" (a brick of any size, --box)
for captures that must stay small.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="sphere256",
                    choices=["sphere16", "sphere64", "ellipsoid", "sphere256", "zprobe", "box"])
    ap.add_argument("--box", default="256,96,96",
                    help="nx,ny,nz of the brick the 'box' workload solves (2 RHS, LDR)")
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--precision", default="fp32_refined")
    ap.add_argument("--solver", default="bicgstab")
    ap.add_argument("--z-schedule", default="",
                    help="tile,kind,threads: override the tuned FP32 z pass (kind 0/1/2/3/6/7)")
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import torch

    from dda_inputs import targets as tg
    from dda_inputs import workloads as W
    from paper_1305_6497_gb300 import binding as B

    if args.workload in ("zprobe", "box"):
        dims = (64, 64, 256) if args.workload == "zprobe" else \
            tuple(int(v) for v in args.box.split(","))
        occ, comp = tg.rect_prism(*dims)
        w = W.Workload("brick%dx%dx%d" % dims, occ, comp, [1.33 + 0.01j], 0.19,
                       *W._lab_incidence([(0.0, 0.0, 0.0)]), 2, "LDR", 1e-8, 0.0)
    else:
        fn = {"sphere16": "c1_sphere16", "sphere64": "c2_sphere64",
              "ellipsoid": "c3_ellipsoid", "sphere256": "c5_sphere256"}[args.workload]
        w = getattr(W, fn)()
    t = B.Target(w.occ, w.comp, w.m, method=w.method)
    t.autotune(w.kd, w.n_rhs)
    if args.z_schedule:
        tile, stage, threads = (int(v) for v in args.z_schedule.split(","))
        sch = t.schedule("fp32")
        sch.update(z_tile=tile, z_pitch=3 * tile, z_stage_ghat=stage, z_threads=threads)
        t.set_schedule(sch, "fp32")
    kw = dict(yhat=w.yhat, npol=2, tol=w.tol, max_iter=5000, precision=args.precision,
              want_P=False, solver=args.solver)
    for _ in range(args.warmup):
        t.solve(w.kd, w.khat, w.e01, **kw)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    outs = [t.solve(w.kd, w.khat, w.e01, profile=True, **kw) for _ in range(args.solves)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    sched = t.schedule("fp32")
    t.close()
    print(json.dumps({
        "workload": w.name, "N": w.n_dipoles, "rhs": w.n_rhs, "precision": args.precision,
        "solve_ms": [o["t_solve_ms"] for o in outs],
        "iters": [int(np.sum(o["iters"])) for o in outs],
        "rhs_matvecs": [int(o["matvecs"]) for o in outs],
        "pass_ms": {f"{p}:{k}": v for (p, k), v in outs[-1]["kernel_ms"].items()},
        "pass_calls": {f"{p}:{k}": v for (p, k), v in outs[-1]["kernel_calls"].items()},
        "schedule_fp32": sched,
    }))


if __name__ == "__main__":
    main()
