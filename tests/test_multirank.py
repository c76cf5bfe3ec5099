"""Host logic of the multi-GPU form (independent replicas, weak scaling) on
CPU ranks with the gloo backend: each rank gets its own seed, the timing is
the maximum over ranks, and the throughput counts every rank's steps."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2505_20418_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.replica_workload("nacl64", rank)
        pos, _, _ = synth.make_state(w)
        local_seconds = 1.0 + 0.5 * rank          # rank 1 is the slow one
        total = bench.max_over_ranks(local_seconds, dist)
        value = bench.weak_scaling_value(world, 10, total)
        first = torch.tensor(pos[0], dtype=torch.float64)
        gathered = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, first)
        out[rank] = (total, value, [g.tolist() for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_weak_scaling():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        total, value, firsts = out[r]
        assert total == 1.5                          # the slowest rank's time
        assert value == pytest.approx(2 * 10 / 1.5)  # all ranks' steps / max time
        assert not np.allclose(firsts[0], firsts[1])  # independent replicas


def test_single_rank_is_identity():
    assert bench.max_over_ranks(2.5, None) == 2.5
    assert bench.weak_scaling_value(1, 100, 2.0) == 50.0
