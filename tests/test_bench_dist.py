"""Host logic of bench.py's multi-rank path, on CPU with gloo (world size 2).

Replicas only: each rank times its own walk; the job's time is the slowest
rank's (all-reduce MAX) and the value counts every rank's site-steps.  The
reference arm runs on rank 0 alone; the other ranks exit without work.
"""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 40.0][rank]
    worst = bench.max_over_ranks(ms, world, "cpu")
    value = bench.job_value(1000, 10, 4, world, worst)
    # rank != 0 in the reference arm returns at once and prints nothing
    out = io.StringIO()
    if rank != 0:
        args = bench.argparse.Namespace(warmup=1, steps=1, gpus=world)
        with redirect_stdout(out):
            bench.run_reference(args, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, worst, value, out.getvalue()))


def test_max_over_ranks_and_job_value_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, value, printed in res:
        assert worst == 40.0
        assert value == pytest.approx(1000 * 10 * 4 * 2 / 0.040)
        if rank != 0:
            assert printed == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.job_value(10, 2, 3, 1, 1000.0) == 60.0


def test_all_core_oracle_baseline_runs():
    """The all-core leg spawns one process per core, each running the single-core sample."""
    import bench
    r = bench.oracle_cpu_baseline_all_cores(seconds=0.3)
    assert r["cores"] >= 1 and r["value"] > 0
