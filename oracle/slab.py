"""ORACLE -- test infrastructure only.  A z-slab domain decomposition of the
oracle's pseudo-time sweeps, run as one process per rank (torch.distributed,
gloo on CPU), for checking the decomposition itself: with the same per-point
code, a split run must give bitwise the fields of the unsplit oracle.

Rank r owns the index planes k0 <= k < k1 of a partition of 0..nz (every
field lives on the (nx+1)(ny+1)(nz+1) index grid).  Each rank holds the
whole state and the whole moduli, updates only its own planes, and before
each half of a sweep receives the planes next to its range that the half
reads (Sec. 3.2 updates the stresses from the velocities, then the
velocities from the stresses):
  * the stress update of plane k reads w of planes k-1, k, k+1 (the cell's
    e_zz needs w_z of plane k+1; the xz and yz edges need w of plane k-1);
  * the velocity update of plane k reads stresses of planes k-1, k, k+1 (the
    z face needs the cells of plane k-1; the x and y faces the xz and yz
    edges of plane k+1).
So one exchange of a single plane with each neighbour precedes each half;
gather() assembles the owned planes on every rank at the end.
"""
from __future__ import annotations

import numpy as np

from . import apt

W_FIELDS = (6, 7, 8)           # w_x, w_y, w_z
S_FIELDS = (0, 1, 2, 3, 4, 5)  # p, tau_xx, tau_yy, tau_xy, tau_xz, tau_yz


def plane_ranges(nz: int, world: int):
    """Contiguous, balanced split of the index planes 0..nz over the ranks."""
    n = nz + 1
    if not 1 <= world <= n:
        raise ValueError("need 1 <= world <= nz + 1")
    cuts = [r * n // world for r in range(world + 1)]
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def _exchange(state, fields, k0, k1, nz, rank, world, group=None):
    """Send plane k0 down and plane k1-1 up; receive plane k0-1 from below and
    plane k1 from above (the fields given)."""
    import torch
    import torch.distributed as dist
    reqs, bufs = [], []
    fl = list(fields)
    if rank > 0:
        out = torch.from_numpy(np.ascontiguousarray(state[fl, k0]))
        reqs.append(dist.isend(out, rank - 1, group=group))
        inn = torch.empty(out.shape, dtype=out.dtype)
        reqs.append(dist.irecv(inn, rank - 1, group=group))
        bufs.append((k0 - 1, inn))
    if rank < world - 1:
        out = torch.from_numpy(np.ascontiguousarray(state[fl, k1 - 1]))
        reqs.append(dist.isend(out, rank + 1, group=group))
        inn = torch.empty(out.shape, dtype=out.dtype)
        reqs.append(dist.irecv(inn, rank + 1, group=group))
        bufs.append((k1, inn))
    for r in reqs:
        r.wait()
    for k, t in bufs:
        state[fl, k] = t.numpy()


def sweeps(K, G, e6, state, n, par, rank, world, bc=0, group=None):
    """n sweeps of the rank's planes of `state` (a full-size oracle state)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nz, ny, nx = K.shape
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    assert state.flags.c_contiguous and state.shape == apt.state_shape(nx, ny, nz)
    k0, k1 = plane_ranges(nz, world)[rank]
    Hn = apt.node_moduli(K, G)
    L = apt.lib()
    for _ in range(n):
        _exchange(state, W_FIELDS, k0, k1, nz, rank, world, group)
        L.oracle_stress_planes(nx, ny, nz, bc, par.dtt, par.dt, apt._p(K), apt._p(G), apt._p(e6),
                               apt._p(state), k0, k1)
        _exchange(state, S_FIELDS, k0, k1, nz, rank, world, group)
        L.oracle_velocity_planes(nx, ny, nz, par.cdr, apt._p(Hn), apt._p(state), k0, k1)
    return state


def gather(state, rank, world, group=None):
    """The whole state with every rank's own planes, on every rank."""
    import torch
    import torch.distributed as dist
    nz = state.shape[1] - 1
    k0, k1 = plane_ranges(nz, world)[rank]
    parts = [None] * world
    dist.all_gather_object(parts, (k0, k1, state[:, k0:k1].copy()), group=group)
    out = state.copy()
    for a, b, blk in parts:
        out[:, a:b] = blk
    return out
