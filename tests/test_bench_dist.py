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


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints
    one JSON line with the reference arm's keys; no GPU is involved."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], cwd=root,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == d["unit"] == "Gvoxel-iters/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] >= 3
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
