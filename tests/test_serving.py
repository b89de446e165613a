"""Serving loop: admission by slots and HBM bytes (CPU, with a fake solver that
sleeps), and on the GPU, each request's result alone equals its result in the
concurrent mix."""
import threading
import time

import numpy as np
import pytest

from dda_inputs import workloads as W
from paper_1305_6497_gb300 import serving as S


class FakeSolver:
    """Stands in for the GPU: sleeps in proportion to N, records concurrency."""

    def __init__(self):
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.bytes_active = 0
        self.max_bytes = 0

    def estimate_bytes(self, req):
        return int(np.count_nonzero(req.occ)) * 1000

    def solve(self, req):
        nb = self.estimate_bytes(req)
        with self.lock:
            self.active += 1
            self.bytes_active += nb
            self.max_active = max(self.max_active, self.active)
            self.max_bytes = max(self.max_bytes, self.bytes_active)
        time.sleep(1e-6 * np.count_nonzero(req.occ) + 0.002)
        with self.lock:
            self.active -= 1
            self.bytes_active -= nb
        q = np.array([float(req.id), 0.0])
        return dict(Qext=q, Qabs=q * 0, Qsca=q, iters=np.array([3, 3]),
                    resid=np.array([1e-9, 1e-9]), status=0)


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
