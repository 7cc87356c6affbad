"""Division of independent grids over ranks (one process per GPU), and the
host-side reductions of a multi-process run, on CPU with the gloo backend."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2302_13903_gb300 import inputs
from paper_2302_13903_gb300.sharding import (gather_statuses, max_over_ranks, partition_lpt,
                                             sum_over_ranks)


def batch_cells():
    return [s["n"] ** 3 for s in inputs.batch_specs(512)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_lpt_shares_cover_once_and_balance(world):
    cells = batch_cells()
    shares = partition_lpt(cells, world)
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(len(cells)))
    loads = [sum(cells[i] for i in s) for s in shares]
    lower = max(max(cells), sum(cells) / world)  # no division beats this
    assert max(loads) <= 4.0 / 3.0 * lower + 1e-9
    assert partition_lpt(cells, world) == shares  # deterministic


def test_lpt_small_cases():
    assert partition_lpt([], 2) == [[], []]
    assert partition_lpt([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    with pytest.raises(ValueError):
        partition_lpt([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        cells = batch_cells()
        share = partition_lpt(cells, world)[rank]
        parts = [None] * world
        dist.all_gather_object(parts, share)
        union = sorted(i for p in parts for i in p)
        ok_cover = union == list(range(len(cells)))
        slow = max_over_ranks(10.0 + rank)
        total = sum_over_ranks(sum(cells[i] for i in share))
        statuses = gather_statuses(share, [i % 3 for i in share], world)
        out[rank] = (ok_cover, slow, total, statuses)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    cells = batch_cells()
    for r in range(world):
        ok_cover, slow, total, statuses = out[r]
        assert ok_cover
        assert slow == 11.0
        assert total == sum(cells)
        assert statuses == [i % 3 for i in range(len(cells))]
