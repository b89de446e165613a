"""Serving loop: admission by slots and HBM bytes (CPU, with a fake solver that
sleeps), and on the GPU, each request's result alone equals its result in the
concurrent mix."""
import collections
import threading
import time

import numpy as np
import pytest

from dda_inputs import workloads as W
from paper_1305_6497_gb300 import serving as S


class FakeSolver:
    """Stands in for the GPU: sleeps in proportion to N, records concurrency,
    and keeps an LRU cache of idle 'targets' that hold half of a request's
    bytes after its solve (like a real target's transform and workspace)."""

    def __init__(self, cache_targets=8, server=None):
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.bytes_active = 0
        self.max_bytes = 0
        self.cache = collections.OrderedDict()
        self.cache_targets = cache_targets
        self.server = server
        self.max_total = 0

    def estimate_bytes(self, req):
        return int(np.count_nonzero(req.occ)) * 1000

    def acquire(self, req):
        with self.lock:
            self.cache.pop(req.key(), None)
        return req

    def solve_on(self, req, _req):
        nb = self.estimate_bytes(req)
        self._check()
        with self.lock:
            self.active += 1
            self.bytes_active += nb
            self.max_active = max(self.max_active, self.active)
            self.max_bytes = max(self.max_bytes, self.bytes_active)
        time.sleep(1e-6 * np.count_nonzero(req.occ) + 0.002)
        with self.lock:
            self.active -= 1
            self.bytes_active -= nb
        self._check()
        q = np.array([float(req.id), 0.0])
        return dict(Qext=q, Qabs=q * 0, Qsca=q, iters=np.array([3, 3]),
                    resid=np.array([1e-9, 1e-9]), status=0)

    def release(self, req):
        with self.lock:
            self.cache[req.key()] = self.estimate_bytes(req) // 2
            while len(self.cache) > self.cache_targets:
                self.cache.popitem(last=False)

    def cached_bytes(self):
        with self.lock:
            return sum(self.cache.values())

    def evict(self, nbytes):
        freed = 0
        with self.lock:
            while self.cache and freed < nbytes:
                freed += self.cache.popitem(last=False)[1]
        return freed

    def _check(self):
        # what any other thread can see: reservations + idle cache, read under
        # the server's lock
        if self.server is not None:
            with self.server.cv:
                self.max_total = max(self.max_total, self.server.in_use + self.cached_bytes())

    def solve(self, req):
        self.acquire(req)
        out = self.solve_on(req, req)
        self.release(req)
        return out


def _stream(n, n_max=3e4):
    return S.requests_from_stream(W.serving_stream(n_requests=n, rate_hz=400.0, n_max=n_max))


def test_admission_respects_slots_and_budget():
    reqs = _stream(24)
    fake = FakeSolver()
    budget = 3 * max(fake.estimate_bytes(r) for r in reqs)
    srv = S.Server(fake, budget, max_slots=4)
    res = srv.run(reqs, realtime=True)
    assert [r.id for r in res] == [r.id for r in reqs]
    assert fake.max_active <= 4
    assert srv.peak_slots <= 4
    assert srv.peak_in_use <= budget
    assert fake.max_bytes <= budget
    assert srv.peak_slots >= 2                # work overlapped
    st = srv.stats()
    assert st["requests"] == 24 and st["errors"] == 0
    assert st["latency_s"]["p50"] <= st["latency_s"]["p99"]


def test_request_larger_than_budget_is_rejected_not_queued_forever():
    reqs = _stream(4)
    fake = FakeSolver()
    small = min(fake.estimate_bytes(r) for r in reqs)
    srv = S.Server(fake, small, max_slots=2)
    res = srv.run(reqs, realtime=False)
    assert len(res) + len(srv.errors) == 4
    assert all("rejected" in e for _, e in srv.errors)
    assert len(res) >= 1


def test_budget_covers_reservations_and_idle_cached_targets():
    """Running solves' reservations plus the bytes idle cached targets hold stay
    within the budget: idle targets are evicted (oldest first) to admit work."""
    reqs = _stream(32)
    fake = FakeSolver(cache_targets=16)
    budget = 3 * max(fake.estimate_bytes(r) for r in reqs)
    srv = S.Server(fake, budget, max_slots=4)
    fake.server = srv
    res = srv.run(reqs, realtime=False)
    assert len(res) == 32 and not srv.errors
    assert srv.peak_total <= budget
    assert fake.max_total <= budget
    assert srv.evicted_bytes > 0              # the cache had to give way
    assert srv.in_use == 0 and srv.slots == 0
    assert srv.stats()["peak_hbm_reserved_plus_cached_bytes"] <= budget


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    """Each request solved alone must give the same Q's as in the concurrent
    stream (same kernels, no cross-request interaction)."""
    reqs = _stream(10, n_max=2e4)
    alone = S.GpuSolver(tol=1e-8)
    ref = {r.id: alone.solve(r) for r in reqs}
    alone.close()
    mixed = S.GpuSolver(tol=1e-8)
    srv = S.Server(mixed, 8 << 30, max_slots=6)
    res = srv.run(reqs, realtime=False)
    mixed.close()
    assert not srv.errors
    assert srv.peak_slots >= 2
    for r in res:
        q = ref[r.id]
        assert np.allclose(r.Qext, q["Qext"], rtol=1e-9, atol=0)
        assert np.allclose(r.Qabs, q["Qabs"], rtol=1e-9, atol=1e-14)
        assert np.all(r.resid <= 1e-8 * 1.01)


@pytest.mark.gpu
def test_served_requests_match_the_oracle():
    """A seeded subset of the serving stream (N <= 2e4, two of every shape:
    sphere, CYLINDER1, HEX_PRISM, RCTGLPRSM, random orientations, LDR) served
    concurrently; each request's Q_ext and Q_abs equal the FP64 oracle's
    (FFT-convolution BiCGSTAB to 1e-11) to 1e-6."""
    from oracle import dda as O
    stream = W.serving_stream(n_requests=40, rate_hz=400.0, n_max=2e4)
    picked, seen = [], collections.Counter()
    for s in stream:
        if seen[s["shape"]] < 2:
            picked.append(s)
            seen[s["shape"]] += 1
    assert set(seen) == {"sphere", "cylinder", "hex_prism", "rect"}
    reqs = S.requests_from_stream(picked)
    solver = S.GpuSolver(tol=1e-8)
    srv = S.Server(solver, 8 << 30, max_slots=4)
    res = {r.id: r for r in srv.run(reqs, realtime=False)}
    solver.close()
    assert not srv.errors
    for q in reqs:
        ref = O.solve_target(q.occ, q.comp, q.m, q.kd, q.khat[0], q.yhat[0], q.e01[0],
                             q.method, npol=q.npol, tol=1e-11)
        r = res[q.id]
        for l in range(q.npol):
            assert abs(r.Qext[l] / ref["Qext"][l] - 1) < 1e-6, (q.id, l)
            assert abs(r.Qabs[l] - ref["Qabs"][l]) < 1e-6 * abs(ref["Qext"][l]), (q.id, l)


@pytest.mark.gpu
def test_admission_estimate_bounds_what_a_target_holds():
    """dda_estimate_solve_bytes (host-only, before the target exists) is an upper
    bound on what the target holds after its first solve."""
    from paper_1305_6497_gb300 import binding as B
    for s in W.serving_stream(n_requests=6, rate_hz=400.0, n_max=3e4, seed=5):
        for prec in ("fp32_refined", "fp64"):
            est = B.dda_estimate_solve_bytes(s["occ"], len(s["m"]), "LDR", s["kd"],
                                             s["khat"], s["e01"], precision=prec)
            t = B.Target(s["occ"], s["comp"], s["m"], method="LDR")
            t.solve(s["kd"], s["khat"], s["e01"], yhat=s["yhat"], tol=1e-6, precision=prec,
                    want_P=False)
            held = t.device_bytes
            t.close()
            assert 0 < held <= est, (prec, held, est)
