"""Host logic of the z-slab decomposition, on CPU: the slab window the
library computes (ce_slab_cells), the plane split, C from summed averages,
and the distributed driver (DistSlab over gloo ranks) around a numpy slab
that has the library slab's interface and a stencil with the same reach
(plane k reads planes k - 1 and k + 1).  Planes a slab neither owns nor
holds as ghosts are NaN, so a missing or misplaced exchange shows."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2410_20441_gb300 import ce, slab

NZ, P = 17, 5
NCHECK = 4


class NumpySlab:
    """Jacobi sweeps x_k <- x_k / 2 + (x_{k-1} + x_{k+1}) / 4 + f_k on the
    interior planes 0 < k < nz of the own range, x = 0 on planes 0 and nz."""

    def __init__(self, z0, z1, nz=NZ):
        self.shape = (P, 1, nz)
        self.nz = nz
        self.z0, self.z1 = z0, z1
        self.lower, self.upper = z0 > 0, z1 < nz + 1
        self.f = np.random.default_rng(3).normal(size=(nz + 1, P))

    def _own(self):
        return [k for k in range(self.z0, self.z1) if 0 < k < self.nz]

    def start(self, loads=None):
        n = 6 if loads is None else len(loads)
        self.x = np.full((n, self.nz + 1, P), np.nan)
        self.x[:, max(self.z0 - 1, 0):min(self.z1 + 1, self.nz + 1)] = 0.0
        self.fc = np.stack([(m + 1) * self.f for m in range(n)])
        own = self._own()
        return np.array([np.sum(self.fc[m, own] ** 2) for m in range(n)])

    def sweep(self, cases=None, n_sweeps=1, check=False):
        cases = list(range(len(self.x))) if cases is None else list(cases)
        r2 = []
        for m in cases:
            x = self.x[m]
            new = x.copy()
            acc = 0.0
            for k in self._own():
                d = 0.25 * (x[k - 1] + x[k + 1]) - 0.5 * x[k] + self.fc[m, k]
                acc += float(np.sum(d * d))
                new[k] = 0.5 * x[k] + 0.25 * (x[k - 1] + x[k + 1]) + self.fc[m, k]
            self.x[m] = new
            r2.append(acc)
        if check:
            self.r2 = np.array(r2)

    def residual(self, n):
        return self.r2[:n]

    def halo_bytes(self):
        return self.x.shape[0] * P * 8

    def pack(self, side, msg):
        k = self.z0 if side == 0 else self.z1 - 1
        msg.view(torch.float64).copy_(torch.from_numpy(np.ascontiguousarray(self.x[:, k]).reshape(-1)))

    def unpack(self, side, msg):
        k = self.z0 - 1 if side == 0 else self.z1
        self.x[:, k] = msg.view(torch.float64).numpy().reshape(self.x.shape[0], P)

    def sums(self):
        own = list(range(self.z0, self.z1))
        s = np.nansum(self.x[:, own], axis=(1, 2))
        return np.stack([s * (t + 1) for t in range(12)], axis=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z0, z1 = slab.plane_ranges(NZ, world)[rank]
        s = NumpySlab(z0, z1)
        d = slab.DistSlab(s, device="cpu")
        iters, rel, status = d.solve(np.eye(6)[:3], tol=1e-4, max_iter=3000, n_check=NCHECK)
        sums = d._allsum(s.sums())
        np.savez(os.path.join(out, f"r{rank}.npz"), x=s.x[:, z0:z1], iters=iters, rel=rel, status=status, sums=sums)
    finally:
        dist.destroy_process_group()


def test_plane_ranges_split_the_planes_into_slabs_of_two_or_more():
    for nz in (3, 8, 17, 191):
        for parts in range(1, (nz + 1) // 2 + 1):
            r = slab.plane_ranges(nz, parts)
            assert r[0][0] == 0 and r[-1][1] == nz + 1
            assert all(b - a >= 2 for a, b in r) and all(r[q][1] == r[q + 1][0] for q in range(parts - 1))
    for bad in (0, 10):
        with pytest.raises(ValueError):
            slab.plane_ranges(17, bad)


def test_slab_window_of_the_library():
    """Own planes [z0, z1) read the cells of planes z0 - 1 .. z1 (clipped to the
    grid's cells 0 .. nz - 1): one ghost layer on each side with a neighbour."""
    shape = (9, 7, 20)
    assert ce.slab_cells(shape, 0, 21) == (0, 20)          # the whole grid
    assert ce.slab_cells(shape, 0, 7) == (0, 8)            # bottom slab: ghost cell layer 7
    assert ce.slab_cells(shape, 7, 14) == (6, 15)          # middle slab
    assert ce.slab_cells(shape, 14, 21) == (13, 20)        # top slab ends at the top face
    assert ce.slab_cells(shape, 19, 20) == (18, 20)
    for z0, z1 in ((20, 21), (-1, 5), (5, 5), (5, 22), (7, 3)):
        with pytest.raises(ce.CeError):
            ce.slab_cells(shape, z0, z1)


def test_ceff_from_summed_averages():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(6, 6))
    C = A @ A.T + 6 * np.eye(6)
    E = np.eye(6) + 0.1 * rng.normal(size=(6, 6))
    shape = (4, 5, 6)
    V = 4 * 5 * 6
    sums = np.concatenate([(C @ E).T, E.T], axis=1) * V      # row m: case m's sigma sums, then eps sums
    assert np.allclose(slab.ceff_from_sums(sums, shape), C, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_slabs_match_one_slab(tmp_path, world):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    one = NumpySlab(0, NZ + 1)
    iters, rel, status = slab.drive([one], lambda: None, lambda x: x, np.eye(6)[:3], tol=1e-4, max_iter=3000,
                                    n_check=NCHECK)
    assert list(status) == [ce.CE_OK] * 3 and iters.max() < 3000 and iters.min() > NCHECK
    sums = one.sums()
    got = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    x = np.concatenate([g["x"] for g in got], axis=1)
    assert np.array_equal(x, one.x)
    for g in got:
        assert np.array_equal(g["iters"], iters) and np.array_equal(g["status"], status)
        assert np.allclose(g["rel"], rel, rtol=1e-12, atol=0)
        assert np.allclose(g["sums"], sums, rtol=1e-12, atol=1e-12)


def test_every_split_of_plane_ranges_has_a_library_window():
    """Every slab plane_ranges makes is one the library accepts, and the
    windows cover the cells each slab reads: its own planes' cells plus one
    layer on each side with a neighbour."""
    for nz in (3, 4, 9, 20, 47):
        for parts in range(1, (nz + 1) // 2 + 1):
            for z0, z1 in slab.plane_ranges(nz, parts):
                c0, c1 = ce.slab_cells((5, 4, nz), z0, z1)
                assert c0 == max(z0 - 1, 0) and c1 == min(z1 + 1, nz)
                assert c1 - c0 >= 2
