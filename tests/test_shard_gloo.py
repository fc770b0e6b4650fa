"""Sharding of the batched form across ranks, on the CPU with the gloo
backend (world size 2): the box split, the slowest-rank timing and the
per-box result gather.  No GPU is involved: the data path has no collective,
so what is tested here is all the multi-process logic there is."""
import os
import socket

import numpy as np
import pytest

from paper_2504_15508_gb300.shard import box_costs, gather_by_box, partition, slowest
from workloads.water import batched_boxes


def _costs(nbox=96):
    specs = batched_boxes(nbox=nbox, seed=5)
    return box_costs([4 * s["n_mol"] for s in specs], [s["mesh"] for s in specs])


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_box_once_and_balances(world):
    c = _costs()
    parts = partition(c, world)
    flat = sorted(b for p in parts for b in p)
    assert flat == list(range(len(c)))
    loads = [c[p].sum() for p in parts]
    # longest-processing-time-first: within 4/3 of the ideal split, and never
    # more than one box above the mean
    assert max(loads) <= max(c.sum() / world + c.max(), 0)
    assert max(loads) <= 4.0 / 3.0 * max(c.sum() / world, c.max()) + 1e-9
    assert partition(c, world) == parts  # the same split on every rank


def test_partition_rejects_empty_world():
    with pytest.raises(ValueError):
        partition([1.0, 2.0], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = _costs()
        mine = partition(c, world)[rank]
        # stand-in per-box results: what a rank would read back from its BatchPlan
        energies = np.array([1000.0 + b for b in mine])
        virials = np.array([[b + 0.5 * k for k in range(6)] for b in mine]).reshape(len(mine), 6)
        e_all = gather_by_box(len(c), mine, energies)
        v_all = gather_by_box(len(c), mine, virials)
        t = slowest(1.0 + rank)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([e_all, v_all.ravel(), [t]]))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_gather_and_slowest(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    c = _costs()
    expect_e = 1000.0 + np.arange(len(c))
    expect_v = np.array([[b + 0.5 * k for k in range(6)] for b in range(len(c))]).ravel()
    for r in range(world):
        got = np.load(os.path.join(tmp_path, f"r{r}.npy"))
        assert np.array_equal(got[:len(c)], expect_e)
        assert np.array_equal(got[len(c):len(c) + 6 * len(c)], expect_v)
        assert got[-1] == 2.0  # the slowest rank's time, on every rank


def test_single_process_fallbacks():
    assert slowest(3.5) == 3.5
    v = gather_by_box(4, [2, 0], np.array([7.0, 9.0]))
    assert np.array_equal(v, [9.0, 0.0, 7.0, 0.0])
