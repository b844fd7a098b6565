"""The replica path of bench.py with two gloo ranks on CPU: the job time is
the slowest rank's, the work the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, w = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1))
    out[rank] = (t, w)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    assert out[0] == out[1] == (150.0, 3000.0)


def test_single_process_is_unchanged():
    import bench
    assert bench.reduce_over_ranks(12.5, 77) == (12.5, 77.0)
