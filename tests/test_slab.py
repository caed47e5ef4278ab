"""z-slab domain decomposition of the oracle's sweeps (the halo-exchange
step a multi-GPU split of one image needs), run as 2 and 3 gloo ranks on
CPU: the split run gives bitwise the fields, and hence the averages and C,
of the unsplit oracle."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import apt, slab
from paper_2410_20441_gb300 import images

SHAPE = (7, 6, 9)      # nx, ny, nz: 10 index planes over the ranks
NSWEEP = 14


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out, bc):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        K, G = images.random_moduli(SHAPE, seed=21)
        par = apt.numerical_parameters(SHAPE)
        states = []
        for m in range(6):
            e6 = np.eye(6)[m]
            st = apt.init_state(K, G, e6, bc=bc)
            slab.sweeps(K, G, e6, st, NSWEEP, par, rank, world, bc=bc)
            states.append(slab.gather(st, rank, world))
        np.save(os.path.join(out, f"s{rank}.npy"), np.stack(states))
    finally:
        dist.destroy_process_group()


def test_plane_ranges_partition_the_index_planes():
    for nz in (1, 4, 9, 31):
        for world in range(1, nz + 2):
            r = slab.plane_ranges(nz, world)
            assert r[0][0] == 0 and r[-1][1] == nz + 1
            assert all(a < b for a, b in r) and all(r[q][1] == r[q + 1][0] for q in range(world - 1))
    with pytest.raises(ValueError):
        slab.plane_ranges(3, 5)


@pytest.mark.parametrize("world,bc", [(2, 0), (3, 1)])
def test_slab_split_is_bitwise_the_unsplit_oracle(tmp_path, world, bc):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path), bc), nprocs=world, join=True,
                       start_method="spawn")
    K, G = images.random_moduli(SHAPE, seed=21)
    par = apt.numerical_parameters(SHAPE)
    ref = []
    for m in range(6):
        st = apt.init_state(K, G, np.eye(6)[m], bc=bc)
        apt.sweeps(K, G, np.eye(6)[m], st, NSWEEP, par, bc=bc)
        ref.append(st)
    ref = np.stack(ref)
    assert np.any(ref[:, 6:9])
    S = np.stack([apt.average(np.eye(6)[m], ref[m])[0] for m in range(6)], axis=1)
    for r in range(world):
        got = np.load(tmp_path / f"s{r}.npy")
        assert np.array_equal(got, ref)
        Sg = np.stack([apt.average(np.eye(6)[m], got[m])[0] for m in range(6)], axis=1)
        assert np.array_equal(Sg, S)
