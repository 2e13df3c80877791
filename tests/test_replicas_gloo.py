"""The N > 1 host logic of bench.py (replicas, weak scaling) on two CPU
ranks over gloo: the slowest rank sets the time, every rank runs its own
seeded replica, the job value counts all ranks' images, and the reference
arm runs on rank 0 only."""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = {}
    out["max"] = bench.max_over_ranks([10.0 + rank, 5.0 - rank], world, device="cpu")
    out["seed"] = bench.replica_seed(dict(bench.CONFIGS["m32"]), rank)
    args = types.SimpleNamespace(cpu_sample=1, warmup=0, steps=1, config="m32", gpus=world,
                                 algo="auto", images=0)
    buf = io.StringIO()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(args, dict(bench.CONFIGS["m32"]), rank, world)
    out["ref_out"] = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0]["max"] == res[1]["max"] == [11.0, 5.0]
    assert res[0]["seed"] != res[1]["seed"]
    assert res[1]["ref_out"] == ""              # rank 1 of the reference arm does no work


def test_job_value_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(4, 1024, 10, 1000.0) == 4 * 1024 * 10
    assert bench.max_over_ranks([3.0, 1.0], 1) == [3.0, 1.0]
