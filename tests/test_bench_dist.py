"""The replicas path of bench.py on CPU: two gloo ranks (no GPU), each
reporting its own time and voxel-evaluations; the whole-job figures are
the slowest rank's time and the sum of the work."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, vox = bench.aggregate(10.0 + 5.0 * rank, 1e6 * (rank + 1))
    out.put((rank, ms, vox))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, vox in res:
        assert ms == 15.0            # the slowest rank
        assert vox == 3e6            # all ranks' work


def test_aggregate_without_a_process_group_is_local():
    import bench
    assert bench.aggregate(7.5, 2e6) == (7.5, 2e6)
