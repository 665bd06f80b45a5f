"""The multi-GPU form of the bench (independent replicas, one per rank) on
CPU: two gloo ranks check the max-over-ranks timing, the job throughput,
that ranks get different frames, and that only rank 0 runs the reference
arm.  No GPU; no data-path collective exists to test."""
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) ms for step A and (10 - r) ms for step B
        got = bench.max_over_ranks([rank + 1.0, 10.0 - rank], world)
        frames = bench.make_frames(rank, 2)
        sums = [None] * world
        dist.all_gather_object(sums, int(frames.astype("int64").sum()))
        q.put((rank, got, sums))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_frames():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, sums in out:
        assert got == [2.0, 10.0]  # the slowest rank of each step
        assert sums[0] != sums[1]  # each replica has its own frames


def test_job_throughput_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 64 frames x 10 steps in 1.0 s (the slowest rank) = 1280 frames/s
    assert bench.job_throughput(64, 10, 2, 1000.0) == pytest.approx(1280.0)
    assert bench.job_throughput(64, 10, 1, 500.0) == pytest.approx(1280.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
