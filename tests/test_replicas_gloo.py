"""The multi-GPU path on the CPU: two gloo ranks, independent replicas, whole-job aggregation."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_13512_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r completes 3 + r units in 1.5 + r seconds
        rate, units, t = replicas.aggregate(1.5 + rank, 3 + rank)
        out[rank] = (rate, units, t)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_is_total_units_over_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        rate, units, t = res[r]
        assert units == 7.0 and t == 2.5
        assert abs(rate - 7.0 / 2.5) < 1e-12


def test_single_process_without_process_group():
    assert replicas.aggregate(2.0, 4) == (2.0, 4.0, 2.0)
