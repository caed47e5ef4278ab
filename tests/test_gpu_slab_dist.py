"""The distributed slab driver (slab.DistSlab) around real library slabs
(ce.Slab), one per process: two gloo processes share the one GPU of the
call, and every halo message is staged through host memory (pack on the
GPU, copy to host, send over gloo, copy back, unpack).  No kernel of one
process waits on the other's.  After a fixed number of sweeps the two
slabs' own planes are, bit for bit, the whole-grid context's fields, both
with the plain exchange after each sweep and with the exchange overlapped
with the interior (ce_slab_sweep_part: boundary planes, pack and send,
interior, receive and unpack); a converged distributed solve (overlapped)
gives the whole grid's iteration counts and C.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (29, 18, 23)
LOADS = np.array([[1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 0, 1], [0.3, -0.2, 0.5, 0.1, -0.4, 0.2]], dtype=np.float64)
NSWEEPS = 19
FIELDS = ("w_x", "w_y", "w_z", "u_x", "u_y", "u_z")


def _image():
    from paper_2410_20441_gb300 import images
    return images.random_spheres(SHAPE, 0.15, seed=17)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import apt
        from paper_2410_20441_gb300 import ce, slab
        K, G = _image()
        nz = K.shape[0]
        z0, z1 = slab.plane_ranges(nz, world)[rank]
        s = ce.Slab(K, G, z0, z1, St=apt.ST_POROUS)
        d = slab.DistSlab(s, device="cpu")
        f = {}
        for ov in (False, True):
            d.sweeps(NSWEEPS, LOADS, overlap=ov)
            torch.cuda.synchronize()
            f.update({f"{int(ov)}_{m}_{n}": s.field(m, n)[z0 - s.c0:z1 - s.c0] for m in range(3) for n in FIELDS})
        iters, rel, status = d.solve(None, tol=1e-5, max_iter=100000)
        C = d.ceff()
        s.close()
        np.savez(os.path.join(out, f"r{rank}.npz"), z0=z0, z1=z1, iters=iters, rel=rel, status=status, C=C, **f)
    finally:
        dist.destroy_process_group()


def test_two_processes_share_one_gpu_and_match_the_whole_grid(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from oracle import apt
    from paper_2410_20441_gb300 import ce
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    K, G = _image()
    got = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    with ce.Context(K, G, prec="fp32", kernel="fused", St=apt.ST_POROUS) as c:
        # the double-word state of unrefined solves, which slabs keep
        c.solve(LOADS, tol=0.0, max_iter=NSWEEPS, check=False, refine="off")
        for m in range(3):
            for n in FIELDS:
                ref = c.field(m, n)
                for g in got:
                    part = ref[int(g["z0"]):int(g["z1"])]
                    for ov in (0, 1):
                        assert np.array_equal(g[f"{ov}_{m}_{n}"], part), (ov, m, n, int(g["z0"]))
        c.solve(None, tol=1e-5, max_iter=100000, refine="off")
        C = c.ceff()
        iters = c.info["iters"]
    for g in got:
        assert list(g["status"]) == [ce.CE_OK] * 6
        assert list(g["iters"]) == iters
        assert np.abs(g["C"] - C).max() <= 1e-9 * np.abs(C).max()
