"""Sharding the batched form across GPUs: one process per GPU, each holding a
share of the independent boxes.

Boxes never exchange data, so the data path has no collective: every rank
builds a ``BatchPlan`` for its own boxes and computes them.  Collectives are
used only outside the data path, to time a step (the slowest rank's time) and
to gather per-box results (energies, virials) on request.

The split balances the cost of a box, taken as its site count plus its mesh
point count (the spread/gather and the FFT work), by longest-processing-time
first: boxes in decreasing cost, each to the currently lightest rank.  The
assignment depends only on the costs and the rank count, so every rank
computes the same split without communicating.
"""
from __future__ import annotations

import numpy as np


def box_costs(n_sites, meshes) -> np.ndarray:
    """Cost of each box: its sites plus its mesh points."""
    n_sites = np.asarray(n_sites, dtype=np.float64)
    meshes = np.asarray(meshes, dtype=np.float64).reshape(len(n_sites), 3)
    return n_sites + np.prod(meshes, axis=1)


def partition(costs, world: int) -> list[list[int]]:
    """Box indices of each rank (each list in increasing box order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(b)
        load[r] += float(costs[b])
    return [sorted(p) for p in parts]


def slowest(ms: float, group=None) -> float:
    """The largest value of ms over the ranks (the step time of a sharded run)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(ms)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_by_box(nbox: int, boxes: list[int], values, group=None) -> np.ndarray:
    """Per-box rows (values[i] belongs to box boxes[i]) from every rank,
    assembled in box order on every rank."""
    import torch.distributed as dist
    values = np.asarray(values)
    if not (dist.is_available() and dist.is_initialized()):
        out = np.zeros((nbox,) + values.shape[1:], dtype=values.dtype)
        out[list(boxes)] = values
        return out
    pieces = [None] * dist.get_world_size(group)
    dist.all_gather_object(pieces, (list(boxes), values), group=group)
    out = np.zeros((nbox,) + values.shape[1:], dtype=values.dtype)
    for bx, vals in pieces:
        if len(bx):
            out[bx] = vals
    return out
