"""The N > 1 path of bench.py (replicas only: every rank extracts independently; the job's time is
the slowest rank's and its cells the sum over ranks), run as two gloo ranks on the CPU, and the
reference arm's rank rule (rank 0 alone runs it)."""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, cells = bench.job_totals(100.0 + 50.0 * rank, 1000 * (rank + 1), world, "cpu")
    q.put((rank, ms, cells))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_summed_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, cells in out:
        assert ms == 150.0 and cells == 3000.0          # max of 100 / 150 ms, sum of 1000 + 2000 cells


def test_single_rank_totals_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(12.5, 7, 1, "cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
