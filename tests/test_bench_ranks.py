"""The replicas path of bench.py with two gloo ranks on the CPU: the job time
is the slowest rank's and the value counts every rank's node updates."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 1000.0 * (rank + 1)            # rank 1 is the slow one
        ms, value = bench.aggregate_ranks(ms_local, 4.0e9, 2, world, device="cpu")
        dist.barrier()
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
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
    for rank, ms, value in out:
        assert ms == 2000.0
        # 2 ranks x 4e9 updates x 2 steps in 2 s
        assert value == pytest.approx(2 * 4.0e9 * 2 / 2.0 / 1e6)
