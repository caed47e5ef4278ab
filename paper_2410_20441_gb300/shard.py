"""Data parallelism: one process per GPU, each solving its own share of
independent problems; the only exchange is a gather of small results.

Two independent axes are sharded:
* the images of a batch (each rank solves whole images; the 6x6 C's are
  gathered), and
* the six load cases of one image (every rank holds the moduli, solves its
  cases, and the volume averages <sigma>, <eps> of every case are gathered,
  after which every rank forms C = S E^-1 itself).

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


def case_owner(m: int, world: int) -> int:
    """Load case m (0..5) belongs to rank m mod world."""
    return m % world


def solve_cases_distributed(solve_cases, rank: int, world: int, group=None):
    """C of one image whose six unit load cases are split over the ranks.
    `solve_cases(list of case indices) -> (sig, eps)`, each (len, 6) with the
    volume averages of those cases (Voigt, engineering shear).  Returns C and
    the gathered (S, E) with the averages of case m in column m."""
    mine = [m for m in range(6) if case_owner(m, world) == rank]
    if mine:
        sig, eps = solve_cases(mine)
        local = {m: (np.asarray(sig[q], dtype=np.float64).tolist(), np.asarray(eps[q], dtype=np.float64).tolist())
                 for q, m in enumerate(mine)}
    else:
        local = {}
    got = gather(local, group)
    S = np.array([got[m][0] for m in range(6)]).T
    E = np.array([got[m][1] for m in range(6)]).T
    # C = S E^-1 by the library (averages passed as sums over a unit volume)
    from . import ce
    sums = np.concatenate([S.T, E.T], axis=1)
    return ce.ceff_from_sums(sums, (1, 1, 1)), S, E


def case_solver(K, G, tol=1e-5, max_iter=100_000, **ctx_kw):
    """solve_cases for GPUs: one FP32 context per call on this rank's GPU."""
    def run(cases):
        from . import ce
        with ce.Context(K, G, **ctx_kw) as c:
            c.solve(np.eye(6)[cases], tol=tol, max_iter=max_iter)
            return c.averages()
    return run


def batch_solver(St=None, n_check=32, tol=1e-5, max_iter=100_000, tile=(0, 0, 0)):
    """solve_local for GPUs: one BatchContext over the local share."""
    def run(local):
        from . import ce
        with ce.BatchContext(local, St=St, n_check=n_check, tile=tile) as b:
            b.solve(tol=tol, max_iter=max_iter)
            return b.ceff()
    return run
