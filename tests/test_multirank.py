"""The multi-rank path of bench.py (one independent replica per rank, barrier, max-over-ranks time,
whole-job throughput) on two CPU ranks with the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slowest
    mlups, ms_max = bench.whole_job_mlups(world, 1000, 10, ms_local, device="cpu")
    out[rank] = (mlups, ms_max)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        mlups, ms_max = out[rank]
        assert ms_max == 150.0
        assert abs(mlups - 2 * 1000 * 10 / 0.150 / 1e6) < 1e-12
