#!/usr/bin/env python
"""Benchmark of the DDA solve (default: the sphere-256^3 workload).

Default workload: sphere on a 256^3 lattice (N = 8,783,848 dipoles, FFT grid
512^3), m = 1.33 + 0.01i, x = 2 pi a_eff / lambda = 25, LATTDR polarizability,
incidence along x with both polarizations (2 right-hand sides), tolerance 1e-8
on the FP64 relative residual -- the largest single-GPU configuration of the
refined-FP32-versus-FP64 comparison.  A step is one complete solve of both
polarizations (every BiCGSTAB iteration, the FP64 refinement residuals, the
final FP64 true residual and the cross sections and forward amplitudes),
FFT-convolution matvec in complex FP32 inside FP64 iterative refinement.  The
plain FP64 solve is timed beside it on the same GPU and both are checked for
equal Q_ext (relative difference <= 1e-6).  --workload picks another
configuration (sphere16, sphere64, ellipsoid).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on
bounded samples of the same workload on the host cores (FFT-convolution
BiCGSTAB in FP64 up to 2 M dipoles, the direct sum on sampled rows,
extrapolated, above).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "dipole*iters/s"
UNIT = "dipole*iterations/s"
# --workload choices (the default is the largest single-GPU configuration)
WORKLOADS = {
    "sphere64": ("c2_sphere64", "sphere64^3 N=137376, m=1.5+0.02i, x=5, LDR, 2 pol, tol 1e-8"),
    "sphere16": ("c1_sphere16", "sphere16^3 N=2176, m=1.33+0.01i, x=1, LDR, 2 pol, tol 1e-8"),
    "ellipsoid": ("c3_ellipsoid", "ellipsoid 48x96x144 N=347432, m=1.7+0.1i, x=8, FCD, "
                                  "32 orientations x 2 pol = 64 RHS, tol 1e-8"),
    "sphere256": ("c5_sphere256", "sphere256^3 N=8783848, m=1.33+0.01i, x=25, LDR, 2 pol, "
                                  "grid 512^3, tol 1e-8"),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(pw), "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic bytes of the five matvec passes (per right-hand side)
# ---------------------------------------------------------------------------
def pass_bytes(box, grid, s):
    nx, ny, nz = box
    Lx, Ly, Lz = grid
    nbox = nx * ny * nz
    rows_x = 3 * nz * ny * Lx          # spectral rows after the x pass
    full_yz = 3 * nz * Ly * Lx         # after the y pass
    per_rhs = {
        "x_fwd": s * (3 * nbox + rows_x),
        "y_fwd": s * (rows_x + full_yz),
        "z_mul": s * (2 * full_yz),
        "y_inv": s * (full_yz + rows_x),
        "x_inv": s * (rows_x + 3 * nbox + 3 * nbox) + nbox,   # + composition bytes
    }
    H = (Lx // 2 + 1) * (Ly // 2 + 1) * (Lz // 2 + 1)
    per_launch = {"z_mul": 6 * H * s}    # the Green transform octant, read once
    return per_rhs, per_launch


def _source_hash():
    h = hashlib.sha256()
    for f in ("matvec_impl.cuh", "fft_core.cuh", "fft_plan.cuh", "matvec_fixed.cu",
              "zpass_pair.cuh", "dda_common.cuh"):
        with open(os.path.join(ROOT, "paper_1305_6497_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` (all right-hand sides active) from the
    committed ncu summary, or None if it was taken on a different version of
    the kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = _source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#"):
            k, w, sha, per_launch = parts[:4]
            if k == kernel and w == workload and sha == src:
                return float(per_launch)
    return None


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(w, iters=3):
    """Time the oracle on a bounded sample of the workload.

    Up to 2 M dipoles: the oracle's FFT-convolution BiCGSTAB (FP64), stopped
    after `iters` iterations of one polarization.  Larger: the oracle's direct
    O(N^2) sum on a block of rows, extrapolated to the 2 matvecs of one
    iteration (labelled extrapolated).  Returns (dipole*iters/s, seconds timed,
    setup seconds, iterations, cores, description)."""
    import numpy as np
    from oracle import dda as O
    flat, pos = O.site_positions(w.occ)
    N = len(flat)
    e1, _ = O.polarization_pair(w.khat[0], w.e01[0])
    ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, w.method, w.kd, w.khat[0], e1)
    if N > 2_000_000:
        rows = np.arange(0, N, N // 4)[:4]
        x = np.ones((N, 3), np.complex128)
        t1 = time.perf_counter()
        c1 = time.process_time()
        O.matvec_direct(x, pos, ainv, w.kd, w.method, rows=rows, block=4, col_block=1 << 19)
        dt = time.perf_counter() - t1
        cores = (time.process_time() - c1) / dt
        t_iter = 2.0 * N / len(rows) * dt        # two full matvecs
        return (N / t_iter, dt, 0.0, 1, cores,
                f"extrapolated: direct-sum rows {len(rows)} of {N} in {dt:.1f} s, "
                f"scaled to the 2 matvecs of one BiCGSTAB iteration")
    E = O.incident_field(pos, w.kd, w.khat[0], e1)
    t0 = time.perf_counter()
    ainv_box = np.zeros(w.occ.size, np.complex128)
    ainv_box[flat] = ainv
    op = O.FFTOperator(w.occ, ainv_box.reshape(w.occ.shape), w.kd, w.method)

    def mv(x):
        return O.box_to_sites(op(O.sites_to_box(x.reshape(-1, 3), flat, w.occ.shape)),
                              flat).reshape(-1)
    t1 = time.perf_counter()
    c1 = time.process_time()
    _, it, _ = O.bicgstab(mv, E.reshape(-1), 1e-30, iters)
    t2 = time.perf_counter()
    cores = (time.process_time() - c1) / (t2 - t1)
    return (N * it / (t2 - t1), (t2 - t1), (t1 - t0), it, cores,
            f"{it} BiCGSTAB iterations (+1 residual matvec) of one polarization of this "
            f"workload (numpy FFT convolution, FP64; {t2 - t1:.1f} s, setup "
            f"{t1 - t0:.1f} s excluded)")


def _workload(name):
    from dda_inputs import workloads as W
    fn, desc = WORKLOADS[name]
    return getattr(W, fn)(), desc


def _smooth_at_least(m):
    """Smallest 2^a 3^b 5^c >= m (the FFT grid rule of the library)."""
    n = max(1, m)
    while True:
        k = n
        for f in (2, 3, 5):
            while k % f == 0:
                k //= f
        if k == 1:
            return n
        n += 1


def _config(w, desc, world):
    """The `config` object of both arms' JSON lines (identical for a workload)."""
    return {"workload": desc, "N": w.n_dipoles, "box": list(w.shape),
            "grid": [_smooth_at_least(2 * n - 1) for n in w.shape], "rhs": w.n_rhs,
            "precision": "fp32_refined", "tol": w.tol,
            "l2": "flushed between steps (256 MB write)",
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def _host_cpu():
    """(logical cores, CPU model) of the host running the oracle."""
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return os.cpu_count(), model or platform.machine()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w, desc = _workload(args.workload)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(w, 1)
    vals, times, cores = [], [], []
    for _ in range(args.steps):
        v, dt, _, it, c, sample = oracle_sample(w, 2)
        vals.append(v)
        times.append(dt)
        cores.append(c)
    value = statistics.mean(vals)
    ncpu, model = _host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": _config(w, desc, world),
        "cpu_baseline": {"value": value, "unit": UNIT,
                         "cores": round(statistics.mean(cores), 2), "kind": "oracle",
                         "host_cores": ncpu, "cpu_model": model,
                         "sample": sample + " per step; cores = process CPU time / wall time"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def aggregate_over_ranks(iters, dev_s, wall_s, world):
    """Whole-job totals of N independent replicas: iterations summed over the
    ranks, device and wall time the maximum over the ranks (every rank has
    passed the same barriers around its timed steps)."""
    tot = {"iters": float(iters), "dev_s": float(dev_s), "wall_s": float(wall_s)}
    if world > 1:
        import torch
        import torch.distributed as dist
        v = torch.tensor([tot["iters"], tot["dev_s"], tot["wall_s"]], dtype=torch.float64)
        s_it = v.clone()
        dist.all_reduce(s_it, op=dist.ReduceOp.SUM)
        m_t = v.clone()
        dist.all_reduce(m_t, op=dist.ReduceOp.MAX)
        tot = {"iters": s_it[0].item(), "dev_s": m_t[1].item(), "wall_s": m_t[2].item()}
    return tot


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from dda_inputs import workloads as W
    from paper_1305_6497_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w, desc = _workload(args.workload)
    N = w.n_dipoles
    R = w.n_rhs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    kw = dict(yhat=w.yhat, npol=2, tol=w.tol, max_iter=5000, dirs=None, want_famp=True,
              solver=args.solver)
    t = B.Target(w.occ, w.comp, w.m, method=w.method)
    grid = t.grid
    # schedule autotuning for this target and batch (setup, not timed)
    schedule = t.autotune(w.kd, R)
    # warm-up (includes the one-time Green-tensor transform build)
    setup = t.solve(w.kd, w.khat, w.e01, precision="fp32_refined", want_P=False, **kw)
    for _ in range(max(0, args.warmup - 1)):
        t.solve(w.kd, w.khat, w.e01, precision="fp32_refined", want_P=False, **kw)

    # ---- timed region: refined FP32 ----
    clocks = ClockSampler(local_rank)
    step_ms, iters, launches = [], [], 0
    kern_ms, kern_calls = {}, {}
    fp32_rhs_mv = fp64_rhs_mv = 0
    qext = None
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    l0 = B.dda_launch_count()
    # NVTX range: lets a profiler restrict its launch list to the timed steps
    torch.cuda.nvtx.range_push("timed")
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)                       # evict L2 between steps
        torch.cuda.synchronize()
        out = t.solve(w.kd, w.khat, w.e01, precision="fp32_refined", want_P=False,
                      profile=True, **kw)
        step_ms.append(out["t_solve_ms"])
        iters.append(int(np.sum(out["iters"])))
        fp32_rhs_mv += out["matvecs"] - out["matvecs_fp64"]
        fp64_rhs_mv += out["matvecs_fp64"]
        sweeps = out["sweeps"]
        for k, v in out["kernel_ms"].items():
            kern_ms[k] = kern_ms.get(k, 0.0) + v
            kern_calls[k] = kern_calls.get(k, 0) + out["kernel_calls"][k]
        qext = out["Qext"]
        resid = out["resid"]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    torch.cuda.nvtx.range_pop()
    launches = B.dda_launch_count() - l0
    clk = clocks.stop()
    barrier()

    dev_s = sum(step_ms) / 1e3
    value_local = N * sum(iters) / dev_s
    solves_local = R * args.steps / dev_s

    # ---- plain FP64 on the same GPU (fewer steps: it is ~10x slower) ----
    k64 = 1 if N > 1_000_000 else max(1, min(args.steps, 3))
    ms64, it64 = [], []
    for _ in range(k64):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        o64 = t.solve(w.kd, w.khat, w.e01, precision="fp64", want_P=False, **kw)
        ms64.append(o64["t_solve_ms"])
        it64.append(int(np.sum(o64["iters"])))
    q64 = o64["Qext"]
    qerr = float(np.max(np.abs(qext / q64 - 1)))

    # ---- the other Krylov methods on the same refined FP32 solve (on request) ----
    solver_cmp = {}
    # normal-equation CG needs many more iterations; it is timed on the smaller
    # workloads only
    others = ["bicgstab", "qmr", "bicgstab2", "gpbicg"] + (["petrkp"] if N <= 1_000_000 else [])
    if not args.compare_solvers:
        others = []
    for other in [s for s in others if s != args.solver]:
        kwo = dict(kw, solver=other)
        t.solve(w.kd, w.khat, w.e01, precision="fp32_refined", want_P=False, **kwo)
        ms_o, it_o, mv_o = [], [], []
        for _ in range(k64):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            oo = t.solve(w.kd, w.khat, w.e01, precision="fp32_refined", want_P=False, **kwo)
            ms_o.append(oo["t_solve_ms"])
            it_o.append(int(np.sum(oo["iters"])))
            mv_o.append(oo["matvecs"])
        solver_cmp[other] = {
            "ms_per_solve_batch": statistics.mean(ms_o),
            "iters_per_rhs": sum(it_o) / (R * k64),
            "rhs_matvecs_per_solve_batch": sum(mv_o) / k64,
            "speedup_vs_headline": statistics.mean(step_ms) / statistics.mean(ms_o),
            "qext_rel_diff_vs_fp64": float(np.max(np.abs(oo["Qext"] / q64 - 1))),
            "resid": [float(r) for r in oo["resid"]]}
    solver_cmp["headline_rhs_matvecs_per_solve_batch"] = (fp32_rhs_mv + fp64_rhs_mv) / args.steps

    # ---- end to end through the C ABI with host buffers ----
    e2e_ms = []
    h2d = int(w.occ.nbytes + w.comp.nbytes)
    d2h = R * N * 3 * 16
    for _ in range(1 if N > 1_000_000 else max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        te = B.Target(w.occ, w.comp, w.m, method=w.method)
        oe = te.solve(w.kd, w.khat, w.e01, precision="fp32_refined", want_P=True, **kw)
        te.close()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_iters = int(np.sum(oe["iters"]))
    t.close()

    # ---- roofline of the dominant pass ----
    per_rhs, per_launch = pass_bytes(w.shape, grid, 8)
    wl = args.workload
    dom = max(((kern_ms[("fp32", p)], p) for p in B.PASSES))[1]
    tms = kern_ms[("fp32", dom)]
    ncall = kern_calls[("fp32", dom)]
    alg = per_rhs[dom] * fp32_rhs_mv + per_launch.get(dom, 0) * ncall
    achieved = alg / (tms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic_launch = _ncu_traffic(dom, wl)
    # the z pass runs the column-pair kernel for z kinds 2..7, else the
    # one-column-tile kernels
    zk = schedule["fp32"]["z_stage_ghat"]
    kname = {"z_mul": "k_fft_z_pairs" if zk >= 2 else "k_fft_z_mul"}.get(dom, f"k_fft_{dom}")
    share = {f"{p}": round(kern_ms[("fp32", p)] / sum(step_ms), 4) for p in B.PASSES}
    share.update({f"{p}_fp64": round(kern_ms[("fp64", p)] / sum(step_ms), 4)
                  for p in B.PASSES})

    # ---- aggregate over ranks (replicas) ----
    tot = aggregate_over_ranks(float(sum(iters)), dev_s, t_wall, world)
    if rank != 0:
        return 0
    value = N * tot["iters"] / tot["dev_s"]
    cpu = None
    if world == 1:  # the host-core oracle baseline is taken at one GPU only
        v_cpu, dt_cpu, setup_cpu, it_cpu, c_cpu, sample = oracle_sample(w, 3)
        ncpu, model = _host_cpu()
        cpu = {"value": v_cpu, "unit": UNIT, "cores": round(c_cpu, 2), "kind": "oracle",
               "host_cores": ncpu, "cpu_model": model,
               "sample": sample + "; cores = process CPU time / wall time"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot["dev_s"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 inner / c128 refinement", "data": "synthetic",
        "config": _config(w, desc, world),
        "schedule": schedule,
        "solves_per_s": R * args.steps * world / tot["dev_s"],
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1,
                                                   int(math.ceil(0.99 * len(step_ms))) - 1)]},
        "iters_per_rhs": sum(iters) / (R * args.steps),
        "refinement": {"sweeps_per_rhs": [int(x) for x in sweeps],
                       "fp64_rhs_matvecs_per_step": fp64_rhs_mv / args.steps,
                       "fp32_rhs_matvecs_per_step": fp32_rhs_mv / args.steps},
        "fp64_vs_refined": {
            "fp64_ms_per_solve_batch": statistics.mean(ms64),
            "fp64_dipole_iters_per_s": N * sum(it64) / (sum(ms64) / 1e3),
            "fp64_iters_per_rhs": sum(it64) / (R * k64),
            "refined_speedup": statistics.mean(ms64) / statistics.mean(step_ms),
            "qext_rel_diff": qerr, "qext": [float(q) for q in qext],
            "resid_refined": [float(r) for r in resid]},
        "solver": args.solver,
        "other_solvers": solver_cmp or None,
        "setup_ms": setup["t_setup_ms"],
        "roofline": {"bound": "hbm", "kernel": f"{kname} (fp32)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_rhs": per_rhs[dom],
                     "algorithmic_bytes_per_launch": alg / ncall,
                     "launches": ncall,
                     "traffic": traffic_launch,
                     "share_of_step": share},
        "cpu_baseline": cpu,
        "e2e": {"value": N * e2e_iters / (statistics.mean(e2e_ms) / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms),
                "includes": "target create (occupancy upload, Green-tensor transform), "
                            "solve, P download, destroy"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=7,
                    help="timed steps (7 refined solves of the 256^3 sphere: about a minute)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sphere256", choices=sorted(WORKLOADS))
    ap.add_argument("--compare-solvers", action="store_true",
                    help="also time QMR, BiCGstab(2), GPBi-CG (and PETRKP up to 1 M dipoles)")
    ap.add_argument("--solver", default="bicgstab", choices=["bicgstab", "qmr", "bicgstab2", "gpbicg", "petrkp"],
                    help="Krylov method of the timed solves (the others are timed beside)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
