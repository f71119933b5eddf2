"""The replica (N > 1) timing path of bench.py on CPU with gloo, world size 2:
max over ranks of the timed region and the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # the slower rank decides
    ms = bench.reduce_max(local_ms, world, "cpu")
    rate = bench.aggregate_rate(1000, 10, world, ms)
    dist.barrier()
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_replicas_reduce_max_and_aggregate_with_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 150.0
        assert rate == pytest.approx(1000 * 10 * 2 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(12.5, 1, "cpu") == 12.5
