"""The multi-rank plumbing of bench.py on CPU (gloo, two ranks): the barrier, the
maximum over ranks that the timed region reports, and the whole-job rate (units
of every rank over the slowest rank's time).  The solver itself runs one
independent replica per GPU; no data-path collective exists to test."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ranks = bench.Ranks(world, torch.device("cpu"))
        ranks.barrier()
        ms = 10.0 + 5.0 * rank                  # rank 1 is the slow one
        slowest = ranks.max(ms)
        units = 1000.0 * (rank + 1)             # 1000 + 2000 units
        rate = bench.job_rate(ranks, units, slowest)
        ranks.barrier()
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 15.0
        assert rate == pytest.approx(3000.0 / 0.015 / 1e6)


def test_single_rank_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    ranks = bench.Ranks(1, None)
    ranks.barrier()
    assert ranks.max(3.5) == 3.5 and ranks.sum(2.0) == 2.0
    assert bench.job_rate(ranks, 2e6, 1000.0) == pytest.approx(2.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=120, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
