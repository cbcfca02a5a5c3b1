"""bench.py's multi-rank logic on the CPU: two gloo ranks (world_size 2, 127.0.0.1).

Each rank runs its own streams (replicas; no data-path collective). The only cross-rank steps are
the reductions of the timing: the whole-job value is every rank's samples over the slowest rank's
time, and the serving line sums per-rank throughputs. The reference arm prints from rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [2.0, 3.0][rank]                      # rank 1 is the slowest
        value = bench.job_gsamples(10**9, 4, seconds, "cpu")
        slowest = bench.rank_reduce(seconds, "max", "cpu")
        total = bench.rank_reduce([1.5, 2.5][rank], "sum", "cpu")
        q.put((rank, value, slowest, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, slowest, total in got:
        assert slowest == 3.0
        assert value == pytest.approx(2 * 4 * 1.0 / 3.0)   # 2 ranks x 4 steps x 1e9 / 3 s, in G
        assert total == 4.0
    del torch


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_reduce(1.25, "max", "cpu") == 1.25
    assert bench.job_gsamples(2 * 10**9, 3, 2.0, "cpu") == pytest.approx(3.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
