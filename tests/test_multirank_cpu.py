"""The benchmark's multi-GPU path is replicas only: every rank solves its own copy of the workload,
the job's time is the slowest rank's, and the job's rate counts every rank's solves. These CPU
tests run that host-side logic on two gloo ranks (no GPU): rank and world parsing, the
max-over-ranks reduction, the whole-job rate, and the reference arm's rank-0-only rule."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.env_rank()
        ms = 100.0 + 25.0 * rank  # rank 1 is the slower replica
        mx = bench.max_over_ranks(ms, w, "cpu")
        dist.barrier()
        q.put((r, w, lr, mx, bench.job_rate(w, 4, mx)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 125.0 for o in out)  # both ranks see the slowest rank's time
    assert all(abs(o[4] - 2 * 4 / 0.125) < 1e-9 for o in out)  # 8 solves in 125 ms


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1, 5, 500.0) == 10.0


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun the reference arm's rank 1 exits 0 at once, printing nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
