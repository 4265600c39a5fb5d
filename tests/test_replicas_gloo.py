"""The replicas path of bench.py (one process per GPU, no data-path
collective): the timing aggregation over ranks, run as world-size-2 gloo
process groups on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        total_ms, mpix = bench.whole_job(10.0 * (rank + 1), 1_000_000, 5, world, dist)
        out[rank] = (total_ms, mpix)
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_and_sums_the_pixels():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    # every rank sees the slowest rank's 20 ms and the pixels of both ranks
    for r in range(world):
        total_ms, mpix = res[r]
        assert total_ms == pytest.approx(20.0)
        assert mpix == pytest.approx(1_000_000 * world * 5 / 0.020 / 1e6)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    total_ms, mpix = bench.whole_job(8.0, 3_732_928, 100, 1, None)
    assert total_ms == 8.0 and mpix == pytest.approx(3_732_928 * 100 / 0.008 / 1e6)
