"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
replica of the work, combine to the slowest rank's time and the sum of the
units (weak scaling, no collective in the data path)."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    t, u = bench.combine_ranks(dist, "cpu", 1.5 + rank, 1000 * (rank + 1))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_time_and_units():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        t, u = out[rank]
        assert t == pytest.approx(2.5)  # slowest rank
        assert u == 3000                # all ranks' units


def test_single_process_is_unchanged():
    import bench
    assert bench.combine_ranks(None, "cpu", 1.25, 77) == (1.25, 77)
