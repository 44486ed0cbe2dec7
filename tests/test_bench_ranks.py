"""The multi-rank path of bench.py on CPU: two gloo ranks with different local
times report the slowest rank's time and the whole-job throughput."""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1000.0 * (rank + 1)  # rank 1 is the slow one (2 s)
    v = bench.job_throughput(cells_per_rank=100, steps=4, world=world, local_ms=local_ms)
    m = bench.max_over_ranks(local_ms)
    q.put((rank, v, m))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, v, m in out:
        assert m == pytest.approx(2000.0)
        assert v == pytest.approx(2 * 100 * 4 / 2.0)
