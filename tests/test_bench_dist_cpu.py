"""The benchmark's multi-process logic on CPU (gloo, two ranks): the timed
region's whole-job rate takes the slowest rank's time and every rank's
bytes, and under a two-rank launch the reference arm prints one line from
rank 0 while rank 1 exits 0 without work.  (The fragmentation itself has
no exchange step: N GPUs run N independent replicas.)"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        # rank r took (r + 1) x 100 ms for 10 steps of 1 GB each
        ms, gbps = bench.job_rate(dist, 100.0 * (rank + 1), 1e9, 10, world, "cpu")
        out[rank] = (ms, gbps)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_bytes():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    # the slowest rank: 200 ms for 10 steps; 2 ranks x 10 GB in 0.2 s
    for r in range(world):
        ms, gbps = out[r]
        assert ms == pytest.approx(20.0)
        assert gbps == pytest.approx(100.0)


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms, gbps = bench.job_rate(None, 50.0, 2e9, 5, 1, "cpu")
    assert ms == pytest.approx(10.0) and gbps == pytest.approx(200.0)


def test_reference_arm_under_two_ranks():
    """torchrun with two ranks: one JSON line (rank 0), both ranks exit 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "aesfull", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
