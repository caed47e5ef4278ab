"""Data-parallel split of a batch over ranks and the gather of results,
run as two gloo processes on CPU (the CPU oracle stands in for the GPU
solver, so the multi-rank logic is checked without a GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2410_20441_gb300 import images, shard


def test_assign_balances_voxels_and_is_deterministic():
    sizes = [n ** 3 for n in (138, 94, 106, 117, 132, 91, 117, 74, 64, 117, 122, 110, 82, 91, 79, 124)]
    for world in (1, 2, 3, 4, 8):
        own = shard.assign(sizes, world)
        assert own == shard.assign(sizes, world)
        load = np.bincount(own, weights=sizes, minlength=world)
        assert sorted(set(own)) == list(range(min(world, len(sizes))))
        # greedy LPT: no rank exceeds the mean by more than the largest item
        assert load.max() - load.mean() <= max(sizes)
        mine = [shard.local_items(sizes, r, world) for r in range(world)]
        assert sorted(sum(mine, [])) == list(range(len(sizes)))
    assert shard.assign([5, 5, 5, 5], 2) == [0, 1, 0, 1]
    with pytest.raises(ValueError):
        shard.assign([1], 0)


def _oracle_solver(local):
    from oracle import apt
    return np.array([apt.solve(K, G, tol=1e-9).C for K, G in local])


def _oracle_cases(K, G):
    from oracle import apt

    def run(cases):
        r = apt.solve(K, G, loads=np.eye(6)[cases], tol=1e-9)
        return r.S.T, r.E.T
    return run


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        imgs = [images.random_moduli((3 + i % 2, 4, 3), seed=40 + i) for i in range(5)]
        C = shard.solve_distributed(imgs, _oracle_solver, rank, world)
        t = shard.max_over_ranks(float(rank + 1))
        np.save(os.path.join(out, f"C{rank}.npy"), C)
        np.save(os.path.join(out, f"t{rank}.npy"), np.array([t]))
        K, G = images.random_moduli((4, 3, 5), seed=77)
        Cc, S, E = shard.solve_cases_distributed(_oracle_cases(K, G), rank, world)
        np.save(os.path.join(out, f"Cc{rank}.npy"), Cc)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_the_serial_result(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    imgs = [images.random_moduli((3 + i % 2, 4, 3), seed=40 + i) for i in range(5)]
    serial = _oracle_solver(imgs)
    for r in range(world):
        C = np.load(tmp_path / f"C{r}.npy")
        assert C.shape == (5, 6, 6)
        assert np.array_equal(C, serial)
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == 2.0
    # load cases split over the ranks: the same C as all six on one rank
    from oracle import apt
    K, G = images.random_moduli((4, 3, 5), seed=77)
    Cs = apt.solve(K, G, tol=1e-9).C
    for r in range(world):
        assert np.allclose(np.load(tmp_path / f"Cc{r}.npy"), Cs, rtol=0, atol=1e-12 * np.abs(Cs).max())


def test_case_owner_covers_six_cases_once():
    for world in (1, 2, 3, 4, 6, 8):
        owners = [shard.case_owner(m, world) for m in range(6)]
        assert all(0 <= o < world for o in owners)
        assert sorted(sum(([m for m in range(6) if shard.case_owner(m, world) == r] for r in range(world)), [])) \
            == list(range(6))


def test_single_process_falls_back_to_local_values():
    imgs = [images.random_moduli((3, 3, 3), seed=1), images.random_moduli((3, 4, 3), seed=2)]
    C = shard.solve_distributed(imgs, _oracle_solver, 0, 1)
    assert np.array_equal(C, _oracle_solver(imgs))
    assert shard.max_over_ranks(3.5) == 3.5
