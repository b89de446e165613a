"""The N>1 path of bench.py on CPU: two gloo ranks (replicas only, no
data-path collective).  The whole-job totals sum the ranks' iterations and take
the slowest rank's time; under torchrun the reference arm prints one line from
rank 0 and every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r ran 100 (r + 1) iterations in 2 + r s of device time, 3 + r s wall
    tot = bench.aggregate_over_ranks(100.0 * (rank + 1), 2.0 + rank, 3.0 + rank, world)
    queue.put((rank, tot))
    dist.destroy_process_group()


def test_replica_totals_sum_work_and_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == {"iters": 300.0, "dev_s": 3.0, "wall_s": 4.0}


def test_single_rank_totals_are_the_rank_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(7, 1.5, 2.5, 1) == {"iters": 7.0, "dev_s": 1.5,
                                                          "wall_s": 2.5}


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1",
           "--workload", "sphere16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


@pytest.mark.timeout(300)
def test_reference_arm_single_rank_line():
    """One process: the reference arm's JSON line carries the contract's keys."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
           "--workload", "sphere16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["host_cores"] >= 1 and d["cpu_baseline"]["cpu_model"]
    # the same config object the GPU arm prints for this workload
    sys.path.insert(0, ROOT)
    import bench
    from dda_inputs import workloads as W
    assert d["config"] == bench._config(W.c1_sphere16(), bench.WORKLOADS["sphere16"][1], 1)
    assert d["config"]["grid"] == [32, 32, 32]
