"""Multi-process path of bench.py on CPU ranks (gloo, world size 2).

The method shards only as independent replicas (one field per GPU, no data
exchange), so the N > 1 path is: each rank runs its own seeded trajectory,
the timed region is bracketed by barriers, and rank 0 reports the whole-job
throughput over the slowest rank. This checks that logic with the gloo
backend on two host processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2507_21748_gb300 import inputs
    t = 1.0 + rank  # rank 1 is the slower one
    dist.barrier()
    t_max = bench.max_over_ranks(t)
    value = bench.job_throughput(world, 10, 1000.0, t_max)
    seed = bench.replica_seed(rank)
    field = inputs.uniform_field((4, 4, 4), seed=seed)
    q.put((rank, t_max, value, seed, float(field.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, v0, s0, f0), (_, t1, v1, s1, f1) = out
    assert t0 == t1 == 2.0                      # max over ranks
    assert v0 == v1 == 2 * 10 * 1000.0 / 2.0    # all ranks' voxel-steps / slowest time
    assert s0 != s1 and f0 != f1                # independent replicas


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 200, 8.0, 2.0) == 800.0
