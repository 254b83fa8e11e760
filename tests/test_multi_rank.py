"""Host logic of the multi-GPU bench run on CPU: two gloo ranks agree on the slowest
rank's time, and the whole-job rate counts every rank's replica."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + 5.0 * rank)
    rate = bench.whole_job_rate(world, 1e9, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 15.0
        assert abs(rate - 2 * 1e9 / 15e-3) < 1e-3 * rate


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.25) == 3.25
    assert bench.whole_job_rate(1, 2e9, 500.0) == 4e9
