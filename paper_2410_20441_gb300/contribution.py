"""Compliance contribution tensor H of one spheroidal inclusion from GPU
solves (Sec. 4.2 and App. B: S* = S1 + phi H, Eq. eqN2), over aspect
ratios and contrasts (the study of H versus alpha, Sec. 4.2).

Two set-ups:
* full: the spheroid (semi-axes a, a, alpha a; the larger of a and alpha a
  is `size` times the box edge L) centred in an L^3 box, kinematic boundary
  (KUBC), all six load cases: every component of H;
* octant: the corner octant of that box, (L/2)^3 voxels with the spheroid's
  centre on the corner, roller boundary (CE_BC_ROLLER).  The three symmetry
  planes of the spheroid carry no shear traction and no normal motion
  relative to the affine field, which is what the rollers impose, so under
  the three normal loads the octant reproduces the full box with rollers at
  an eighth of the voxels -- the quarter-domain device of Sec. 4.2.  Only
  the normal block (H11, H22, H33, H12, H13, H23 in Voigt compliance) is
  defined there.

H is returned in Voigt compliance form (engineering shear strains): for the
compliance S = C^-1 of the Voigt stiffness, H = (S* - S1) / phi with phi the
voxel volume fraction.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ce, images

MATRIX = (36.0, 44.0)                        # Sec. 4.2 background (K, G), GPa
CONTRASTS = {
    "void": (1e-3, 2e-3),                    # Sec. 4.2's near-void inclusion
    "soft": (36.0 / 5, 44.0 / 5),            # soft inhomogeneity: K1/K2 = G1/G2 = 5
    "stiff": (36.0 * 5, 44.0 * 5),           # stiff inhomogeneity: K2/K1 = G2/G1 = 5
}


def c_iso(K, G):
    lam = K - 2.0 * G / 3.0
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2.0 * G
    C[np.arange(3, 6), np.arange(3, 6)] = G
    return C


def semi_axes(L, alpha, size):
    """(a, c = alpha a) with max(a, c) = size * L."""
    a = size * L / max(1.0, alpha)
    return a, alpha * a


def image(L, alpha, size=0.2, inclusion=CONTRASTS["void"], matrix=MATRIX, octant=False):
    a, _ = semi_axes(L, alpha, size)
    if octant:
        h = L // 2
        return images.spheroid((h, h, h), (0.0, 0.0, 0.0), a, alpha, matrix, inclusion)
    return images.spheroid((L, L, L), (L / 2, L / 2, L / 2), a, alpha, matrix, inclusion)


def contribution(L, alpha, size=0.2, inclusion=CONTRASTS["void"], matrix=MATRIX, octant=False, tol=1e-5,
                 St=None, max_iter=400_000):
    """One GPU solve: dict with phi, C (6x6), H (6x6 Voigt compliance, or its
    normal 3x3 block for the octant), iterations and seconds."""
    K, G, phi = image(L, alpha, size, inclusion, matrix, octant)
    t0 = time.perf_counter()
    loads = np.eye(6)[:3] if octant else None
    with ce.Context(K, G, prec="fp32", bc="roller" if octant else "kubc", St=St) as c:
        c.solve(loads, tol=tol, max_iter=max_iter)
        if octant:
            sig, eps = c.averages()
            C = np.zeros((6, 6))
            C[:3, :3] = (np.asarray(sig)[:, :3].T) @ np.linalg.inv(np.asarray(eps)[:, :3].T)
        else:
            C = c.ceff()
        iters = c.info["iters"]
    S1 = np.linalg.inv(c_iso(*matrix))
    if octant:
        H = (np.linalg.inv(C[:3, :3]) - S1[:3, :3]) / phi
    else:
        H = (np.linalg.inv(C) - S1) / phi
    return {"L": int(L), "alpha": float(alpha), "octant": bool(octant), "phi": phi, "C": C.tolist(),
            "H": H.tolist(), "iters": iters, "seconds": time.perf_counter() - t0}


def main(argv=None):
    ap = argparse.ArgumentParser(description="H of a spheroid versus aspect ratio (GPU)")
    ap.add_argument("--L", type=int, default=192, help="edge of the full box in voxels")
    ap.add_argument("--alphas", default="0.1,0.2,0.5,1,2,5,10")
    ap.add_argument("--contrasts", default="void,soft,stiff")
    ap.add_argument("--size", type=float, default=0.2)
    ap.add_argument("--octant", action="store_true", help="corner octant with rollers (normal block only)")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--st", type=float, default=None)
    a = ap.parse_args(argv)
    out = []
    for name in a.contrasts.split(","):
        for al in (float(v) for v in a.alphas.split(",")):
            r = contribution(a.L, al, a.size, CONTRASTS[name], MATRIX, a.octant, a.tol, a.st)
            r["contrast"] = name
            out.append(r)
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
