"""The multi-rank path of bench.py on CPU: two gloo ranks, disjoint event shards, max-over-ranks
timing and the whole-job rate (the GPU path runs the same functions over NCCL)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.5 + rank            # rank 1 is the slow one
    t_max = bench.max_over_ranks(t_local, world, "cpu")
    seeds = [bench.rank_seed0(rank) + e for e in range(64)]
    q.put((rank, t_max, seeds, bench.whole_job_rate(64, 10, world, t_max)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, v0), (r1, t1, s1, v1) = res
    assert t0 == t1 == 2.5                       # both ranks see the slowest rank's time
    assert not set(s0) & set(s1)                 # disjoint event shards
    assert v0 == v1 == pytest.approx(64 * 10 * 2 / 2.5)


def test_single_rank_no_collective():
    import bench
    assert bench.max_over_ranks(0.75, 1, "cpu") == 0.75
    assert bench.whole_job_rate(64, 10, 1, 0.5) == 1280.0
