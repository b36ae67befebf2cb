"""The bench's multi-rank path, on CPU. The lattice-sum step does not shard: with N GPUs each
rank runs its own replica of the workload, the job's step time is the slowest rank's, and the
whole-job rate counts every rank's units. Two gloo ranks (spawned processes, 127.0.0.1) check
that every rank gets the slowest rank's time and the same rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank_ms, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(per_rank_ms[rank], dist, "cpu")
        rate = bench.whole_job_rate(world, 1000, ms / 1e3)
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_ranks_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    per_rank_ms = [12.5, 17.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, per_rank_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert [g[0] for g in got] == [0, 1]
    assert [g[1] for g in got] == [17.25, 17.25]
    for g in got:
        assert g[2] == pytest.approx(2 * 1000 / 0.01725, rel=1e-12)
    assert all(p.exitcode == 0 for p in procs)


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 67046, 0.0241) == 67046 / 0.0241
