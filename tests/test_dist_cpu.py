"""The multi-rank path of bench.py on CPU: two gloo ranks, whole-job
throughput = all ranks' samples over the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [400.0, 500.0][rank]  # rank 1 is the slow one
    value, tmax = bench.aggregate(local_ms, samples_per_rank=1_000_000, steps=10, dist=dist, device="cpu")
    q.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, tmax in res:
        assert tmax == 500.0
        assert abs(value - 2 * 1_000_000 * 10 / 0.5 / 1e6) < 1e-9  # 40 Msamples/s
