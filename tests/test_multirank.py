"""The replicas-only multi-GPU path of the benchmark, on CPU: two gloo ranks
each report their own elapsed time; the whole-job value uses the slowest
rank's time and all ranks' work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    max_ms, value = bench.aggregate_over_ranks(local_ms, units_per_rank=1e9, world=world,
                                               device="cpu")
    q.put((rank, max_ms, value))
    dist.destroy_process_group()


def test_two_rank_replicas_use_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, value in out:
        assert max_ms == 150.0
        assert abs(value - 2 * 1e9 / 0.150 / 1e9) < 1e-9
