"""Data parallelism over images: one process per GPU, each solving its own
share of the samples; the only exchange is the gather of the 6x6 results.

The images of a batch are independent problems, so nothing crosses GPUs
while they are solved.  `assign` splits a list of images over the ranks by
voxel count (largest first, each to the least-loaded rank; ties to the
lower rank), which is deterministic, so every rank computes the same split
without communicating.  `solve_distributed` runs the local share through one
batched CUDA-graph solve (BatchContext) and gathers every rank's C with
torch.distributed (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def assign(sizes, world: int):
    """Owner rank of each item: greedy longest-processing-time split of the
    items' sizes (voxel counts) over `world` ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda q: (-int(sizes[q]), q)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(sizes[i])
    return owner


def local_items(sizes, rank: int, world: int):
    return [i for i, r in enumerate(assign(sizes, world)) if r == rank]


def gather(local: dict, group=None):
    """All ranks' {item index: value} merged into one dict on every rank."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return dict(local)
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    out = {}
    for p in parts:
        out.update(p)
    return out


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest of every rank's value (e.g. a timed region)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def solve_distributed(images, solve_local, rank: int, world: int, group=None):
    """C of every image, each solved on its owner rank by
    `solve_local(list of (K, G)) -> array (n, 6, 6)`, gathered on all ranks."""
    sizes = [np.asarray(K).size for K, _ in images]
    mine = local_items(sizes, rank, world)
    Cs = solve_local([images[i] for i in mine]) if mine else np.zeros((0, 6, 6))
    got = gather({i: np.asarray(C, dtype=np.float64).tolist() for i, C in zip(mine, Cs)}, group)
    return np.array([got[i] for i in range(len(images))])


def batch_solver(St=None, n_check=32, tol=1e-5, max_iter=100_000, tile=(0, 0, 0)):
    """solve_local for GPUs: one BatchContext over the local share."""
    def run(local):
        from . import ce
        with ce.BatchContext(local, St=St, n_check=n_check, tile=tile) as b:
            b.solve(tol=tol, max_iter=max_iter)
            return b.ceff()
    return run
