"""The multi-GPU path of bench.py is "replicas only": every rank searches its
own roots on its own GPU and the ranks only meet to combine their numbers.
That combination is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hm = [80.0, 70.0][rank]          # GTEPS of each replica
    t = [0.50, 0.75][rank]           # its timed device seconds
    value, step_ms = bench.combine_replicas(dist, world, hm, t, steps=5)
    out[rank] = (value, step_ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine_on_gloo():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in (0, 1):
        value, step_ms = out[r]
        assert value == pytest.approx(150.0)        # sum over replicas
        assert step_ms == pytest.approx(150.0)      # slowest rank: 0.75 s / 5 steps


def test_single_rank_is_unchanged():
    assert bench.combine_replicas(None, 1, 81.0, 0.4, 4) == (81.0, 100.0)
