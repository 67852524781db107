"""The N > 1 path of the benchmark on the CPU: one process per rank over gloo.  The
single-instance path does not shard, so N ranks run independent replicas; the job's
time is the maximum over ranks and its throughput the sum of the replicas' work over
that time.  The reference arm under torchrun runs on rank 0 alone."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms, value = bench.aggregate_replicas(1.0 + rank, 1000, 10, world, dist, device="cpu")
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_replicas_take_the_max_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the work of both replicas counts
    assert [g[1] for g in got] == [2.0, 2.0]
    assert all(abs(g[2] - 1000 * 10 * 2 / 2e-3) < 1e-6 for g in got)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--steps", "1", "--warmup", "3", "--ppc", "4",
           "--ref-sample", "2048"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference"
    assert lines[0]["value"] > 0 and lines[0]["cpu_baseline"]["kind"] == "oracle"
