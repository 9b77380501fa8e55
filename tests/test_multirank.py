"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun launches them.

Each rank evaluates its own copy of the workload (replicas: no collective on the data
path); the job's time is the slowest rank's, and the whole-job rate counts every rank's
units.  The reduction runs through torch.distributed exactly as under NCCL.
"""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, units, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        import bench
        rate, slowest = bench.whole_job_rate(units, seconds[rank], world, torch.device("cpu"))
        largest = bench.max_over_ranks(float(rank), world, torch.device("cpu"))
        out.put((rank, rate, slowest, largest))
    finally:
        dist.destroy_process_group()


def run_ranks(world, seconds, units):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, seconds, units, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_ranks_take_the_slowest_time():
    res = run_ranks(2, seconds=[1.5, 2.0], units=1000.0)
    for rank, rate, slowest, largest in res:
        assert slowest == 2.0              # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 2.0)   # both ranks' units over that time
        assert largest == 1.0


def test_single_rank_needs_no_process_group():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    rate, slowest = bench.whole_job_rate(500.0, 0.25, 1, torch.device("cpu"))
    assert (rate, slowest) == (2000.0, 0.25)


def test_reference_arm_runs_on_rank_zero_only():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(free_port()))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
