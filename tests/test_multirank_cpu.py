"""The replica path of bench.py on two CPU ranks (gloo): each rank runs its own
registration; the whole-job time is the slowest rank's and the work is the sum
over ranks, with no collective on the data path."""
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


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, pts = bench.aggregate_ranks(1.0 + rank, 10.0 * (rank + 1), dist, "cpu")
    dist.barrier()
    out[rank] = (secs, pts)
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == (2.0, 30.0)


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate_ranks(1.5, 7.0) == (1.5, 7.0)
