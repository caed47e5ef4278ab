"""Write the stored expected values of the GPU parity tests.

Calls only the CPU oracle (oracle/) on seeded synthetic images from
paper_2410_20441_gb300.images; never the CUDA library.  Run from the repo
root:  python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import apt  # noqa: E402
from paper_2410_20441_gb300 import images  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # 31^3, centred sphere r = 0.25 L (K = 2.25, G = 1e-3) in 70/30 GPa, FP64, tol 1e-8
    "sphere31": dict(make=lambda: images.single_sphere(31), tol=1e-8, St=apt.ST_3D, n_check=16,
                     recipe="images.single_sphere(31)"),
    # 48^3 random overlapping spheres (r 3-10) to 10 % porosity, pores 1e-4 GPa, seed 2
    "porous48": dict(make=lambda: images.random_spheres(48, 0.10, seed=2), tol=1e-8, St=apt.ST_POROUS,
                     n_check=16, recipe="images.random_spheres(48, 0.10, seed=2)"),
    # 63^3 random overlapping spheres (r 3-10) to 10 % porosity, pores 1e-4 GPa, seed 3: the C
    # error versus tolerance curve, FP64 to tol 1e-9
    "porous63": dict(make=lambda: images.random_spheres(63, 0.10, seed=3), tol=1e-9, St=apt.ST_POROUS,
                     n_check=16, recipe="images.random_spheres(63, 0.10, seed=3)"),
    # 191^3 random overlapping spheres (r 3-10) to 10 % porosity, pores 1e-4 GPa, seed 1: the
    # benchmark image, FP64 to tol 1e-7 (about 33,000 case-sweeps, two to three hours on 8 x86
    # cores).  The Strouhal number changes the path, not the converged C; half the paper's
    # value needs the fewest sweeps at this tolerance on this image
    "porous191": dict(make=lambda: images.porous_191(), tol=1e-7, St=0.5 * apt.ST_3D, n_check=64,
                      recipe="images.porous_191()"),
}


def make(name):
    spec = CASES[name]
    K, G = spec["make"]()
    t = time.time()
    r = apt.solve(K, G, tol=spec["tol"], St=spec["St"], n_check=spec["n_check"], max_iter=400000)
    out = {
        "name": name,
        "written_by": "tests/golden/make_golden.py (CPU oracle, FP64)",
        "recipe": spec["recipe"],
        "tol": spec["tol"], "St": spec["St"], "Ct": apt.CFL_3D, "n_check": spec["n_check"],
        "iters": [c.iters for c in r.cases],
        "status": [c.status for c in r.cases],
        "rel_res": [c.rel for c in r.cases],
        "C": r.C.tolist(),
        "oracle_threads": apt.num_threads(),
        "oracle_seconds": time.time() - t,
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["iters"], out["status"], f"{out['oracle_seconds']:.1f}s")


if __name__ == "__main__":
    for n in sys.argv[1:] or list(CASES):
        make(n)
