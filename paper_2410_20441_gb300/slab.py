"""z-slab domain decomposition of one image: the multi-GPU extension the
paper plans (Sec. 5.3, item 1), built on the library's slab contexts
(ce_create_slab and the ce_slab_* calls of ce.h).

The index planes 0..nz are split into contiguous slabs; slab r updates its
own planes and, after every sweep, swaps one plane of w with each neighbour
(the only data a sweep reads across a slab boundary).  Every N sweeps the
slabs' squared residuals are summed; at the end their stress and strain sums
are.  Each point is computed by the whole-grid arithmetic, so the fields
equal the whole-grid solve's after as many sweeps.

Two drivers share one loop (`drive`):
* `SlabGroup`: all slabs in this process on one GPU, each on its own CUDA
  stream, the messages moved by device copies ordered with events;
* `DistSlab`: one slab per torch.distributed rank, the messages moved with
  point-to-point send/receive and the sums with all_reduce.
"""
from __future__ import annotations

import numpy as np

from . import ce


def plane_ranges(nz: int, parts: int):
    """Contiguous split of the index planes 0..nz into `parts` slabs of
    near-equal size, as [(z0, z1), ...]; every slab gets at least two planes
    (so that the top slab's window, which ends at the grid's top face, still
    holds two cell layers)."""
    n = nz + 1
    if parts < 1 or 2 * parts > n:
        raise ValueError("need 1 <= parts <= (nz + 1) / 2")
    edges = [n * r // parts for r in range(parts + 1)]
    return [(edges[r], edges[r + 1]) for r in range(parts)]


def drive(slabs, exchange, allsum, loads=None, tol=1e-5, max_iter=100_000, n_check=None, overlap=None):
    """The pseudo-time loop over this process's slabs.
    exchange(): refresh every local slab's ghost planes after a sweep.
    allsum(x): the sum of x (numpy) over all processes.
    overlap: None, or (begin, end) for an exchange that overlaps the sweep:
    every sweep that does not measure the residual runs as part 1 (the
    boundary planes), begin() (pack and start the transfers), part 2 (the
    interior), end() (finish the transfers and unpack).
    Returns (iterations per case, relative residual per case, status per case)
    with the meaning of ce_solve's: a case stops at
    ||div sigma(w)|| <= tol ||div sigma(0)||, checked every n_check sweeps on
    the state before the interval's last sweep."""
    b2 = allsum(np.sum([s.start(loads) for s in slabs], axis=0))
    n = b2.shape[0]
    r0 = np.sqrt(b2)
    rel = np.where(r0 > 0, 1.0, 0.0)
    iters = np.zeros(n, dtype=int)
    status = np.where(rel <= tol, ce.CE_OK, ce.CE_ENOTCONV)
    active = [m for m in range(n) if status[m] == ce.CE_ENOTCONV]
    nx = slabs[0].shape[0]
    n_check = n_check or max(16, nx // 4)
    it = 0
    while active and it < max_iter:
        ns = min(n_check, max_iter - it)
        for q in range(ns):
            last = q == ns - 1
            if overlap is not None and not last:
                begin, end = overlap
                for s in slabs:
                    s.sweep_part(active, 1)
                h = begin()
                for s in slabs:
                    s.sweep_part(active, 2)
                end(h)
                continue
            for s in slabs:
                s.sweep(active, 1, check=last)
            exchange()
        r2 = allsum(np.sum([s.residual(len(active)) for s in slabs], axis=0))
        it += ns
        keep = []
        for q, m in enumerate(active):
            rel[m] = np.sqrt(r2[q]) / r0[m] if r0[m] > 0 else 0.0
            iters[m] = it
            if not np.isfinite(rel[m]) or rel[m] > 1e10:
                status[m] = ce.CE_EDIVERGED
            elif rel[m] <= tol:
                status[m] = ce.CE_OK
            else:
                keep.append(m)
        active = keep
    return iters, rel, status


def ceff_from_sums(sums, shape):
    """C = S E^-1 (Eq. eq:4) from the summed 12 values per case (six cases),
    by the library (ce_ceff_from_sums)."""
    return ce.ceff_from_sums(sums, shape)


class SlabGroup:
    """One image split into `parts` z-slabs on one GPU, each slab a context on
    its own CUDA stream.  The exchange after a sweep: every slab packs its two
    boundary planes; each slab's stream waits for its neighbours' packs, copies
    their messages into its own receive buffers and unpacks them; the next
    sweep of a slab waits until its neighbours have copied its messages."""

    def __init__(self, K, G, parts=2, bc="kubc", St=None, Ct=None, n_check=0, tile=(0, 0, 0, 0)):
        import torch
        self.torch = torch
        nz, ny, nx = K.shape
        self.shape = (nx, ny, nz)
        self.ranges = plane_ranges(nz, parts)
        self.streams = [torch.cuda.Stream() for _ in self.ranges]
        self.n_check = n_check
        self.slabs = []
        for (z0, z1), st in zip(self.ranges, self.streams):
            with torch.cuda.stream(st):
                self.slabs.append(ce.Slab(K, G, z0, z1, bc=bc, St=St, Ct=Ct, n_check=n_check, tile=tile,
                                          stream=st.cuda_stream))
        self.msg = None
        self.stats = None

    def _buffers(self):
        torch = self.torch
        nb = self.slabs[0].halo_bytes()
        self.msg = []
        for s, st in zip(self.slabs, self.streams):
            with torch.cuda.stream(st):
                # [side][0 = outgoing, 1 = incoming]
                self.msg.append([[torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)]
                                 for _ in range(2)])
        self.packed = [torch.cuda.Event() for _ in self.slabs]
        self.copied = [torch.cuda.Event() for _ in self.slabs]

    def _exchange(self):
        torch = self.torch
        S = len(self.slabs)
        for r, (s, st) in enumerate(zip(self.slabs, self.streams)):
            with torch.cuda.stream(st):
                if s.lower:
                    s.pack(0, self.msg[r][0][0])
                if s.upper:
                    s.pack(1, self.msg[r][1][0])
                self.packed[r].record(st)
        for r, (s, st) in enumerate(zip(self.slabs, self.streams)):
            with torch.cuda.stream(st):
                if s.lower:
                    st.wait_event(self.packed[r - 1])
                    self.msg[r][0][1].copy_(self.msg[r - 1][1][0])
                    s.unpack(0, self.msg[r][0][1])
                if s.upper and r + 1 < S:
                    st.wait_event(self.packed[r + 1])
                    self.msg[r][1][1].copy_(self.msg[r + 1][0][0])
                    s.unpack(1, self.msg[r][1][1])
                self.copied[r].record(st)
        # a slab packs into its outgoing buffers again only after its
        # neighbours have copied them
        for r, st in enumerate(self.streams):
            if r > 0:
                st.wait_event(self.copied[r - 1])
            if r + 1 < S:
                st.wait_event(self.copied[r + 1])

    def solve(self, loads=None, tol=1e-5, max_iter=100_000):
        self.msg = None

        def exchange():
            if self.msg is None:
                self._buffers()
            self._exchange()

        iters, rel, status = drive(self.slabs, exchange, lambda x: x, loads, tol, max_iter, self.n_check)
        self.stats = {"iters": iters.tolist(), "rel_res": rel.tolist(), "status": status.tolist()}
        return self.stats

    def sweeps(self, n, loads=None):
        """Start and run n sweeps with no convergence test (for comparisons)."""
        for s in self.slabs:
            s.start(loads)
        self._buffers()
        for _ in range(n):
            for s in self.slabs:
                s.sweep(None, 1, False)
            self._exchange()
        self.torch.cuda.synchronize()

    def sums(self):
        return np.sum([s.sums() for s in self.slabs], axis=0)

    def ceff(self):
        return ceff_from_sums(self.sums(), self.shape)

    def field(self, case, name):
        """A field on the whole index grid, each plane from its owner."""
        nx, ny, nz = self.shape
        out = np.zeros((nz + 1, ny + 1, nx + 1))
        for s in self.slabs:
            loc = s.field(case, name)
            out[s.z0:s.z1] = loc[s.z0 - s.c0:s.z1 - s.c0]
        return out

    def close(self):
        for s in self.slabs:
            s.close()
        self.slabs = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class DistSlab:
    """One slab per torch.distributed rank (NCCL on GPUs).  After every sweep
    rank r sends its plane z0 to rank r - 1 and its plane z1 - 1 to rank r + 1
    and receives their boundary planes into its ghost planes; residual and
    average sums are all_reduced.  `slab` is any object with the Slab
    interface (start, sweep, residual, halo_bytes, pack, unpack, sums,
    lower, upper, shape; pack and unpack take a message tensor); messages
    and sums live on `device` (a CUDA device under NCCL, "cpu" under gloo).
    The send/receive calls are ordered on torch's current stream, so a
    library slab must run on that stream (ce.Slab's default).  A library
    slab with device="cpu" (gloo) stages every message through a device
    buffer: pack on the GPU, copy to host, send; receive, copy to the GPU,
    unpack."""

    def __init__(self, slab, device="cuda", group=None):
        import torch
        import torch.distributed as dist
        self.torch = torch
        self.dist = dist
        self.slab = slab
        self.group = group
        self.device = torch.device(device)
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.msg = None
        self.stage = isinstance(slab, ce.Slab) and self.device.type == "cpu"
        self.dev = None

    def buffer(self, nbytes):
        return self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)

    def _pack(self, side):
        s = self.slab
        if self.stage:
            s.pack(side, self.dev[side])
            self.msg[side][0].copy_(self.dev[side])       # synchronous device-to-host copy
        else:
            s.pack(side, self.msg[side][0])

    def _unpack(self, side):
        s = self.slab
        if self.stage:
            self.dev[side].copy_(self.msg[side][1])
            s.unpack(side, self.dev[side])
        else:
            s.unpack(side, self.msg[side][1])

    def _begin(self):
        """Pack the boundary planes and start the sends and receives."""
        dist, s = self.dist, self.slab
        if self.msg is None:
            nb = s.halo_bytes()
            self.msg = [[self.buffer(nb) for _ in range(2)] for _ in range(2)]
            if self.stage:
                self.dev = [self.torch.empty(nb, dtype=self.torch.uint8, device="cuda") for _ in range(2)]
        ops = []
        if s.lower:
            self._pack(0)
            ops += [dist.P2POp(dist.isend, self.msg[0][0], self.rank - 1, self.group),
                    dist.P2POp(dist.irecv, self.msg[0][1], self.rank - 1, self.group)]
        if s.upper:
            self._pack(1)
            ops += [dist.P2POp(dist.isend, self.msg[1][0], self.rank + 1, self.group),
                    dist.P2POp(dist.irecv, self.msg[1][1], self.rank + 1, self.group)]
        return dist.batch_isend_irecv(ops) if ops else []

    def _end(self, reqs):
        """Wait for the transfers and unpack into the ghost planes."""
        s = self.slab
        for w in reqs:
            w.wait()
        if s.lower:
            self._unpack(0)
        if s.upper:
            self._unpack(1)

    def _exchange(self):
        self._end(self._begin())

    def _allsum(self, x):
        t = self.torch.as_tensor(np.asarray(x, dtype=np.float64)).to(self.device)
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def solve(self, loads=None, tol=1e-5, max_iter=100_000, n_check=None, overlap=True):
        """The distributed pseudo-time loop; with overlap (library slabs) the
        halo transfers of a sweep run while its interior planes are swept."""
        self.msg = None
        ov = (self._begin, self._end) if overlap and hasattr(self.slab, "sweep_part") else None
        return drive([self.slab], self._exchange, self._allsum, loads, tol, max_iter, n_check, overlap=ov)

    def sweeps(self, n, loads=None, overlap=True):
        """Start and run n sweeps with no convergence test (for comparisons)."""
        self.msg = None
        self.slab.start(loads)
        split = overlap and hasattr(self.slab, "sweep_part")
        for _ in range(n):
            if split:
                self.slab.sweep_part(None, 1)
                h = self._begin()
                self.slab.sweep_part(None, 2)
                self._end(h)
            else:
                self.slab.sweep(None, 1, False)
                self._exchange()

    def ceff(self):
        return ceff_from_sums(self._allsum(self.slab.sums()), self.slab.shape)
