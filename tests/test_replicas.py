"""Multi-GPU is replicas only (independent solves, no data-path collective):
the benchmark's whole-job figures over ranks -- the slowest rank's time and
the sum of the ranks' iterations -- checked with two gloo ranks on the CPU,
and the reference arm's rank rule (only rank 0 works and prints)."""
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed 100 + 25 r ms and ran 40 + r iterations
    t, u = bench.aggregate_over_ranks(100.0 + 25.0 * rank, 40 + rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, u))


def test_whole_job_figures_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in got:
        assert t == 125.0 and u == 81.0  # max over ranks, sum over ranks, on every rank


def test_single_rank_returns_its_own_figures():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_over_ranks(12.5, 7, "cpu") == (12.5, 7.0)


@pytest.mark.parametrize("rank", ["1", "3"])
def test_reference_arm_other_ranks_exit_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="4", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "4"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
