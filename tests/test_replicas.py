"""The multi-rank path of bench.py: independent replicas, a barrier and a max-reduction of
times, exercised with two gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_19855_gb300.replicas import aggregate_rate, barrier, frame_indices, max_over_ranks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = frame_indices(rank, 4, 64)
        barrier(world)
        # each rank "measures" its own times; the slowest rank decides
        mine = [1.0 + rank, 10.0 - rank, 3.0]
        worst = max_over_ranks(mine, world)
        out[rank] = (frames, worst)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_frames_and_take_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    f0, w0 = out[0]
    f1, w1 = out[1]
    assert f0 == [0, 1, 2, 3] and f1 == [4, 5, 6, 7]
    assert not set(f0) & set(f1)
    assert w0 == w1 == [2.0, 10.0, 3.0]


def test_frame_indices_wrap_around_the_path():
    assert frame_indices(3, 24, 64) == [(72 + k) % 64 for k in range(24)]


def test_aggregate_rate_counts_every_rank():
    assert aggregate_rate(1000, 4, 10, 2.0) == pytest.approx(4 * 1000 * 10 / 2.0)
    assert max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
