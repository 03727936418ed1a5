"""Host-side logic of bench.py on CPU: the cross-rank aggregation of the
timings (2 gloo ranks) and the whole-job MLUPS formula."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
        out[rank] = bench.max_over_ranks(local_ms, world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_process_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_whole_job_mlups():
    # 8.4 M cells, 1000 steps, 4 replicas, slowest rank 400 ms
    assert bench.whole_job_mlups(2048 * 4096, 1000, 4, 400.0) == pytest.approx(
        2048 * 4096 * 1000 * 4 / 0.4 / 1e6)
