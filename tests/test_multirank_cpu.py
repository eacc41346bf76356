"""Multi-rank host logic on CPU (gloo, world size 2).

The transform has no exchange step, so N GPUs run N independent replicas;
bench.py reports the whole-job throughput from the slowest rank's time.
This checks that aggregation with two gloo ranks on 127.0.0.1.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 2.0 if rank == 0 else 3.0
    ms, value = bench.replica_throughput(ms_local, 1_000_000)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 3.0                     # slowest rank
        assert abs(value - 2 * 1_000_000 / 3.0e-3) < 1e-6 * value
