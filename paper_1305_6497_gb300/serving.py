"""Continuous-batching serving loop for DDA solves (host-side scheduler).

Each request is a target (occupancy, composition, refractive indices) with its
incident waves.  The server keeps up to ``max_slots`` solves in flight on the
GPU at once, each on its own ``dda_target`` and therefore its own CUDA stream,
so their kernels overlap on the device.  A request is admitted as soon as a
slot is free AND the device bytes it needs fit in the HBM budget.  Its bytes
are the library's host-only estimate for a new target of its shape
(``dda_estimate_solve_bytes``: creation arrays, Green-tensor transform with its
transient build grids, solve workspace); nothing is allocated before
admission.  Finished solves return their reservation at once, so requests that
arrive while others run start as room appears -- not a queue drained one at a
time.

Targets are cached by geometry and optical constants (LRU), so a repeated
target reuses its resident Green-tensor transform.  An idle cached target keeps
its device memory (``dda_target_device_bytes``), and that memory counts against
the same budget: reservations of running solves plus the bytes of idle cached
targets never exceed it.  When a request does not fit, idle cached targets are
evicted, least recently used first, before the request waits.

The GPU work is in libdda.so; the binding's ctypes calls release the GIL, so
worker threads run their solves concurrently.  ``solver`` can be replaced (the
CPU tests inject a fake) to exercise admission and accounting without a GPU.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import hashlib
import json
import math
import queue
import statistics
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    id: int
    occ: np.ndarray
    comp: np.ndarray
    m: list
    kd: float
    khat: np.ndarray
    yhat: np.ndarray
    e01: np.ndarray
    method: str = "LDR"
    npol: int = 2
    t_arrival: float = 0.0      # seconds after the stream starts

    def key(self) -> str:
        h = hashlib.sha1()
        h.update(np.ascontiguousarray(self.occ).tobytes())
        h.update(np.ascontiguousarray(self.comp).tobytes())
        h.update(np.asarray(self.m, np.complex128).tobytes())
        h.update(self.method.encode())
        return h.hexdigest()


@dataclasses.dataclass
class Result:
    id: int
    Qext: np.ndarray
    Qabs: np.ndarray
    Qsca: np.ndarray
    iters: np.ndarray
    resid: np.ndarray
    status: int
    n_dipoles: int
    t_arrival: float
    t_admit: float
    t_start: float
    t_finish: float
    bytes_reserved: int

    @property
    def latency(self):
        return self.t_finish - self.t_arrival


class GpuSolver:
    """Runs requests through libdda.so with an LRU cache of idle targets.

    Interface used by Server: estimate_bytes(req) (host-only), acquire(req) ->
    handle, solve_on(handle, req), release(handle) (the target becomes an idle
    cache entry), cached_bytes() and evict(nbytes).  solve(req) runs all three
    steps for callers without a Server."""

    def __init__(self, precision="fp32_refined", tol=1e-8, max_iter=5000, cache_targets=8):
        from . import binding as B
        self.B = B
        self.precision = precision
        self.tol = tol
        self.max_iter = max_iter
        self.cache = collections.OrderedDict()   # key -> (Target, device bytes), idle only
        self.cache_targets = cache_targets
        self.lock = threading.Lock()

    def estimate_bytes(self, req: Request) -> int:
        return self.B.dda_estimate_solve_bytes(
            req.occ, len(req.m), req.method, req.kd, req.khat, req.e01, npol=req.npol,
            precision=self.precision)

    def acquire(self, req: Request):
        k = req.key()
        with self.lock:
            hit = self.cache.pop(k, None)
        t = hit[0] if hit is not None else self.B.Target(req.occ, req.comp, req.m,
                                                          method=req.method)
        return (t, k)

    def solve_on(self, handle, req: Request) -> dict:
        t, _ = handle
        return t.solve(req.kd, req.khat, req.e01, yhat=req.yhat, npol=req.npol, tol=self.tol,
                       max_iter=self.max_iter, precision=self.precision, want_P=False,
                       want_famp=False)

    def release(self, handle) -> None:
        t, k = handle
        nbytes = t.device_bytes
        drop = []
        with self.lock:
            if k in self.cache:
                drop.append(t)           # another copy is already cached
            else:
                self.cache[k] = (t, nbytes)
                while len(self.cache) > self.cache_targets:
                    drop.append(self.cache.popitem(last=False)[1][0])
        for old in drop:
            old.close()

    def cached_bytes(self) -> int:
        with self.lock:
            return sum(b for _, b in self.cache.values())

    def evict(self, nbytes: int) -> int:
        """Free idle cached targets, oldest first, until nbytes are freed or the
        cache is empty.  Returns the bytes freed."""
        freed, drop = 0, []
        with self.lock:
            while self.cache and freed < nbytes:
                _, (t, b) = self.cache.popitem(last=False)
                drop.append(t)
                freed += b
        for t in drop:
            t.close()
        return freed

    def solve(self, req: Request) -> dict:
        h = self.acquire(req)
        try:
            return self.solve_on(h, req)
        finally:
            self.release(h)

    def close(self):
        with self.lock:
            for t, _ in self.cache.values():
                t.close()
            self.cache.clear()


class Server:
    """Admission by slots and HBM bytes; worker threads run admitted solves.

    Invariant (checked at every admission and release): the reservations of
    admitted solves plus the solver's idle cached bytes stay within budget."""

    def __init__(self, solver, hbm_budget_bytes: int, max_slots: int = 8):
        self.solver = solver
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.cv = threading.Condition()
        self.in_use = 0
        self.slots = 0
        self.peak_in_use = 0
        self.peak_total = 0
        self.peak_slots = 0
        self.evicted_bytes = 0
        self.queue_depth_max = 0
        self.work = queue.Queue()
        self.results = []
        self.errors = []
        self.workers = [threading.Thread(target=self._worker, daemon=True)
                        for _ in range(self.max_slots)]
        for th in self.workers:
            th.start()

    def _note_total_locked(self):
        total = self.in_use + self.solver.cached_bytes()
        self.peak_total = max(self.peak_total, total)
        return total

    def _admit(self, nbytes):
        """Block until a slot and `nbytes` of budget are free (evicting idle
        cached targets first); False if the request can never fit (it is
        rejected, not queued forever)."""
        if nbytes > self.budget:
            return False
        with self.cv:
            while True:
                if self.slots < self.max_slots:
                    over = self.in_use + self.solver.cached_bytes() + nbytes - self.budget
                    if over > 0:
                        self.evicted_bytes += self.solver.evict(over)
                        over = self.in_use + self.solver.cached_bytes() + nbytes - self.budget
                    if over <= 0:
                        break
                self.cv.wait()
            self.slots += 1
            self.in_use += nbytes
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.peak_slots = max(self.peak_slots, self.slots)
            self._note_total_locked()
        return True

    def _worker(self):
        while True:
            item = self.work.get()
            if item is None:
                return
            req, t0, nbytes, t_admit = item
            t_start = time.perf_counter() - t0
            handle = None
            try:
                handle = self.solver.acquire(req)
                out = self.solver.solve_on(handle, req)
                t_fin = time.perf_counter() - t0
                self.results.append(Result(
                    req.id, np.asarray(out["Qext"]), np.asarray(out["Qabs"]),
                    np.asarray(out["Qsca"]), np.asarray(out["iters"]),
                    np.asarray(out["resid"]), int(out["status"]),
                    int(np.count_nonzero(req.occ)), req.t_arrival, t_admit, t_start, t_fin,
                    nbytes))
            except Exception as e:  # noqa: BLE001 -- reported, never hides a result
                self.errors.append((req.id, repr(e)))
            finally:
                # the target turns into an idle cache entry and the reservation
                # ends in one step, so the two are never counted apart
                with self.cv:
                    if handle is not None:
                        self.solver.release(handle)
                    self.slots -= 1
                    self.in_use -= nbytes
                    self._note_total_locked()
                    self.cv.notify_all()

    def run(self, requests, realtime=True):
        """Replay `requests` (sorted by t_arrival); returns the results."""
        t0 = time.perf_counter()
        admitter = threading.Thread(target=self._admit_loop, args=(requests, t0, realtime))
        admitter.start()
        admitter.join()
        for _ in self.workers:
            self.work.put(None)
        for th in self.workers:
            th.join()
        self.wall = time.perf_counter() - t0
        return sorted(self.results, key=lambda r: r.id)

    def _admit_loop(self, requests, t0, realtime):
        # admission runs in arrival order; a request that does not fit waits
        # while later ones wait behind it (no reordering, no starvation)
        import bisect
        arrivals = [r.t_arrival for r in requests]
        for i, req in enumerate(requests):
            if realtime:
                dt = req.t_arrival - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            try:
                nbytes = self.solver.estimate_bytes(req)
            except Exception as e:  # noqa: BLE001 -- reported per request
                self.errors.append((req.id, repr(e)))
                continue
            if not self._admit(nbytes):
                self.errors.append((req.id, f"rejected: needs {nbytes} B of a "
                                            f"{self.budget} B budget"))
                continue
            now = time.perf_counter() - t0
            self.work.put((req, t0, nbytes, now))
            # requests that have arrived and still wait for admission
            waiting = bisect.bisect_right(arrivals, now) - (i + 1) if realtime else 0
            self.queue_depth_max = max(self.queue_depth_max, waiting)

    def stats(self):
        lat = sorted(r.latency for r in self.results)
        n = len(lat)

        def pct(q):
            return lat[min(n - 1, max(0, int(math.ceil(q * n)) - 1))] if n else float("nan")
        svc = [r.t_finish - r.t_start for r in self.results]
        dip_it = sum(r.n_dipoles * int(np.sum(r.iters)) for r in self.results)
        return {
            "requests": n, "errors": len(self.errors), "wall_s": self.wall,
            "solves_per_s": sum(len(r.Qext) for r in self.results) / self.wall,
            "dipole_iters_per_s": dip_it / self.wall,
            "latency_s": {"p50": pct(0.5), "p99": pct(0.99), "max": lat[-1] if n else None},
            "service_s_mean": statistics.mean(svc) if svc else None,
            "queue_depth_max": self.queue_depth_max,
            "peak_concurrent_solves": self.peak_slots,
            "peak_hbm_reserved_bytes": self.peak_in_use,
            "peak_hbm_reserved_plus_cached_bytes": self.peak_total,
            "evicted_bytes": self.evicted_bytes,
            "hbm_budget_bytes": self.budget,
        }


def requests_from_stream(stream):
    return [Request(id=s["id"], occ=s["occ"], comp=s["comp"], m=s["m"], kd=s["kd"],
                    khat=s["khat"], yhat=s["yhat"], e01=s["e01"], method=s["method"],
                    npol=s["npol"], t_arrival=s["t_arrival"]) for s in stream]


def main():
    ap = argparse.ArgumentParser(description="Replay the seeded serving stream on the GPU.")
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--budget-frac", type=float, default=0.8)
    ap.add_argument("--rate", type=float, default=0.0,
                    help="arrivals/s; 0 = 0.8 x the measured single-stream capacity")
    ap.add_argument("--n-max", type=float, default=1e6)
    args = ap.parse_args()
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    from dda_inputs import workloads as W
    free, _ = torch.cuda.mem_get_info()
    solver = GpuSolver()
    rate = args.rate
    if rate <= 0:
        # single-stream capacity on a small calibration sample of the stream
        cal = requests_from_stream(W.serving_stream(n_requests=24, seed=7, n_max=args.n_max))
        t0 = time.perf_counter()
        for r in cal:
            solver.solve(r)
        rate = 0.8 * len(cal) / (time.perf_counter() - t0)
    reqs = requests_from_stream(W.serving_stream(n_requests=args.requests, rate_hz=rate,
                                                 n_max=args.n_max))
    srv = Server(solver, int(args.budget_frac * free), args.slots)
    srv.run(reqs)
    st = srv.stats()
    st["arrival_rate_hz"] = rate
    st["config"] = {"requests": args.requests, "slots": args.slots, "N": "1e3-1e6 log-uniform",
                    "burst": "4x rate over 10% of the stream", "precision": solver.precision,
                    "tol": solver.tol}
    solver.close()
    print(json.dumps(st))


if __name__ == "__main__":
    main()
