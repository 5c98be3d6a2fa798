"""Multi-GPU runs of the solver are independent replicas (the batched and
serving workloads shard by instance; nothing is exchanged on the data path).
The host logic of a replicated bench run -- the slowest rank's time taken by
an all-reduce (max), the whole-job value over all ranks, and the reference arm
running on rank 0 alone -- is checked here with world_size-2 gloo process
groups on the CPU."""
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


def _worker(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank_ms(dist, times[rank], torch.device("cpu"))
        out[rank] = (ms, bench.whole_job_value(1000.0, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_value_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    times = [12.5, 40.0]
    mp.start_processes(_worker, args=(2, _free_port(), times, out), nprocs=2, join=True,
                       start_method="spawn")
    assert out[0][0] == out[1][0] == 40.0
    assert out[0][1] == out[1][1] == pytest.approx(2 * 1000.0 / 0.040)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(None, 7.0, "cpu") == 7.0
    assert bench.whole_job_value(10.0, 1, 1000.0) == 10.0


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun the reference arm prints one line from rank 0; the
    other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "er2000", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
