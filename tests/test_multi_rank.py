"""The benchmark's multi-rank host logic on CPU with the gloo backend
(world size 2): independent replicas, one chain per rank; the job's time is the
slowest rank's and its value all ranks' sweeps over that time.  The reference
arm does its work on rank 0 only."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, seconds = bench.job_rate(1000, 1.0 + 0.5 * rank, world, "cpu")
        q.put((rank, value, seconds))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, seconds in out:
        assert seconds == pytest.approx(1.5)
        assert value == pytest.approx(2 * 1000 / 1.5)


def test_single_rank_rate_needs_no_process_group():
    import bench
    assert bench.job_rate(500, 2.0, 1, "cpu") == (250.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only():
    import bench
    assert bench.run_reference(None, 1) is None
