"""The z-slab decomposition on the GPU (ce_create_slab and the ce_slab_*
calls), all slabs on one device, each on its own CUDA stream.

* After a fixed number of sweeps every field of every own plane equals,
  bit for bit, the whole-grid context's (the per-point arithmetic is the
  same; only the slab boundaries differ), for two and three slabs, ragged
  grids, z-chunks inside each slab and both boundary modes.
* A converged slab solve gives the whole grid's iteration counts and C up to
  the order of the sums, and C within 1e-4 of the FP64 oracle's.
Slabs keep the double-word state of unrefined solves, so the whole-grid
reference solves run with refine="off".
"""
import json
import os

import numpy as np
import pytest

from oracle import apt
from paper_2410_20441_gb300 import images

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LOADS = np.array([[1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0], [0.3, -0.2, 0.5, 0.1, -0.4, 0.2]], dtype=np.float64)


@pytest.fixture(scope="module")
def ce():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_20441_gb300 import ce as cemod
    cemod.load()
    return cemod


@pytest.mark.parametrize("parts,shape,tile,bc", [
    (2, (37, 21, 41), (3, 16, 16, 1), "kubc"),
    (3, (29, 18, 47), (2, 8, 8, 1), "kubc"),
    (4, (24, 20, 33), (0, 0, 0, 0), "kubc"),
    (2, (33, 16, 30), (3, 16, 5, 1), "roller"),
])
def test_slab_fields_equal_the_whole_grid_bitwise(ce, parts, shape, tile, bc):
    from paper_2410_20441_gb300 import slab
    K, G = images.random_spheres(shape, 0.15, seed=11)
    n = 23
    with ce.Context(K, G, prec="fp32", kernel="fused", bc=bc, tile=tile) as c:
        c.solve(LOADS, tol=0.0, max_iter=n, check=False, refine="off")
        assert c.info["iters"] == [n] * 3
        ref = {(m, f): c.field(m, f) for m in range(3) for f in range(12)}
    with slab.SlabGroup(K, G, parts=parts, bc=bc, tile=tile) as g:
        assert len(g.slabs) == parts
        g.sweeps(n, LOADS)
        for (m, f), r in ref.items():
            got = g.field(m, f)
            assert np.any(r) or f in (3, 4, 5), (m, f)
            assert np.array_equal(got, r), (m, f, np.abs(got - r).max())


def test_slab_solve_matches_the_whole_grid_and_the_oracle(ce):
    from paper_2410_20441_gb300 import slab
    gold = json.load(open(os.path.join(GOLDEN, "porous48.json")))
    K, G = images.random_spheres(48, 0.10, seed=2)
    Cg = np.array(gold["C"])
    with ce.Context(K, G, prec="fp32", kernel="fused", St=apt.ST_POROUS) as c:
        c.solve(None, tol=1e-5, max_iter=200000, refine="off")
        C = c.ceff()
        iters = c.info["iters"]
    with slab.SlabGroup(K, G, parts=3, St=apt.ST_POROUS) as g:
        st = g.solve(None, tol=1e-5, max_iter=200000)
        Cs = g.ceff()
    assert st["status"] == [ce.CE_OK] * 6
    assert st["iters"] == iters
    assert np.abs(Cs - C).max() <= 1e-9 * np.abs(C).max()
    assert np.abs(Cs - Cg).max() <= 1e-4 * np.abs(Cg).max()


def test_slab_calls_refuse_what_they_do_not_do(ce):
    from paper_2410_20441_gb300 import slab
    K, G = images.random_moduli((12, 10, 14), seed=4)
    s = ce.Slab(K, G, 5, 10)
    try:
        assert (s.c0, s.c1) == (4, 11) and s.lower and s.upper
        with pytest.raises(ce.CeError) as ei:
            s.sweep()                                     # before start
        assert ei.value.status == ce.CE_ESTATE
        s.start(np.eye(6)[:2])
        assert s.halo_bytes() == 2 * 18 * 11 * 32         # n_cases * 18 * (ny + 1) * pitch
        with pytest.raises(ce.CeError) as ei:
            s.residual(2)                                 # no checked sweep yet
        assert ei.value.status == ce.CE_ESTATE
        assert s._L.ce_solve(s._h, None, 6, 1e-5, 10, 0, None) == ce.CE_ENOTIMPL
        assert s._L.ce_autotune(s._h, 1, None, None) == ce.CE_ENOTIMPL
        C = np.zeros(36)
        assert s._L.ce_ceff(s._h, ce._dp(C)) == ce.CE_ESTATE
    finally:
        s.close()
    top = ce.Slab(K, G, 10, 15)
    try:
        assert top.lower and not top.upper
        top.start(np.eye(6)[:1])
        import torch
        buf = torch.empty(top.halo_bytes(), dtype=torch.uint8, device="cuda")
        with pytest.raises(ce.CeError) as ei:
            top.unpack(1, buf)                            # no neighbour above
        assert ei.value.status == ce.CE_EINVAL
        with pytest.raises(ce.CeError) as ei:
            top.pack(0, buf.data_ptr() + 8)               # misaligned message
        assert ei.value.status == ce.CE_EINVAL
    finally:
        top.close()
    with pytest.raises(ValueError):
        slab.plane_ranges(14, 8)


def test_two_plane_slabs_and_device_moduli(ce):
    """The finest split (every slab owns two index planes), moduli given as
    CUDA tensors, a subset of load cases: still the whole grid's bits."""
    import torch
    from paper_2410_20441_gb300 import slab
    K, G = images.random_moduli((19, 14, 11), seed=31)
    loads = np.eye(6)[[1, 3]]
    n = 17
    with ce.Context(K, G, prec="fp32", kernel="fused") as c:
        c.solve(loads, tol=0.0, max_iter=n, check=False, refine="off")
        ref = {(m, f): c.field(m, f) for m in range(2) for f in range(12)}
    Kd, Gd = torch.tensor(K, device="cuda"), torch.tensor(G, device="cuda")
    with slab.SlabGroup(Kd, Gd, parts=6) as g:
        assert [b - a for a, b in g.ranges] == [2] * 6
        g.sweeps(n, loads)
        for (m, f), r in ref.items():
            assert np.array_equal(g.field(m, f), r), (m, f)


def test_distributed_driver_on_one_rank(ce, tmp_path):
    """DistSlab on a one-rank NCCL group (no neighbours, so no exchange; the
    sums go through all_reduce on the device): the whole grid's C."""
    import torch
    import torch.distributed as dist
    from paper_2410_20441_gb300 import slab
    K, G = images.random_spheres(32, 0.1, seed=5)
    with ce.Context(K, G, prec="fp32", kernel="fused", St=apt.ST_POROUS) as c:
        c.solve(None, tol=1e-5, max_iter=100000, refine="off")
        C = c.ceff()
        iters = c.info["iters"]
    dist.init_process_group("nccl", init_method=f"file://{tmp_path}/pg", rank=0, world_size=1)
    try:
        s = ce.Slab(K, G, 0, 33, St=apt.ST_POROUS)
        d = slab.DistSlab(s, device="cuda")
        it, rel, status = d.solve(None, tol=1e-5, max_iter=100000)
        Cd = d.ceff()
        s.close()
    finally:
        dist.destroy_process_group()
    assert list(status) == [ce.CE_OK] * 6 and list(it) == iters
    assert np.abs(Cd - C).max() <= 1e-9 * np.abs(C).max()
