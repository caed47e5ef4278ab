"""Resolution study: C_eff of one geometry rasterised at several grid sizes,
and the observed order of convergence (the paper's convergence-rate study
of the single-inclusion model, Sec. 4.2, and its several resolutions of the
cracked-marble image, Sec. 4.3).

Two geometries.  `--model cracked`: one set of randomly oriented cracks
defined in the unit box (images.cracked_scaled) rasterised at n = 191 ..
479, with the time to C at each n (Sec. 4.3 runs 191^3 to 703^3).
`--model sphere` (default): a spheroid with semi-axes (a, a, alpha a), a = a_frac * n,
centred in an n^3 box with the moduli of Sec. 4.2 (matrix K = 36, G = 44 GPa;
a near-void inclusion).  The voxel volume fraction phi(n) of a rasterised
spheroid jumps with n, so the quantity followed is the change of C per unit
volume fraction, D(n) = (C(n) - C1) / phi(n), the discrete counterpart of the
compliance-contribution picture of Eq. eqN2.  Its limit and the order p come
from a least-squares fit of D(n) = D_inf + b n^-p.

    python -m paper_2410_20441_gb300.resolution --sizes 32,48,64,96,128
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ce, images

MATRIX = (36.0, 44.0)
INCLUSION = (1e-3, 2e-3)
# Voigt entries followed: C11, C33, C44 (yz), C66 (xy), C12, C13
ENTRIES = ((0, 0), (2, 2), (3, 3), (5, 5), (0, 1), (0, 2))


def c_iso(K, G):
    """6x6 Voigt stiffness of an isotropic phase."""
    lam = K - 2.0 * G / 3.0
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2.0 * G
    C[np.arange(3, 6), np.arange(3, 6)] = G
    return C


def fit_rate(ns, values, pmin=0.05, pmax=4.0, step=0.005):
    """Least-squares fit of v(n) = v_inf + b n^-p over a grid of p; returns
    (p, v_inf, b, rms residual).  Needs three or more sizes."""
    ns = np.asarray(ns, dtype=np.float64)
    v = np.asarray(values, dtype=np.float64)
    if ns.size < 3 or ns.size != v.size:
        raise ValueError("need three or more (n, value) pairs")
    best = None
    for p in np.arange(pmin, pmax + step / 2, step):
        A = np.stack([np.ones_like(ns), ns ** -p], axis=1)
        coef, *_ = np.linalg.lstsq(A, v, rcond=None)
        r = float(np.sqrt(np.mean((A @ coef - v) ** 2)))
        if best is None or r < best[3]:
            best = (float(p), float(coef[0]), float(coef[1]), r)
    return best


def error_rate(ns, values, ref):
    """Observed order against a reference value: the least-squares slope of
    log|v(n) - ref| / |ref| over log n, negated (the paper's convergence rate
    against the analytical solution, Sec. 4.2); returns (rate, relative
    errors)."""
    ns = np.asarray(ns, dtype=np.float64)
    e = np.abs(np.asarray(values, dtype=np.float64) - ref) / abs(ref)
    A = np.stack([np.ones_like(ns), np.log(ns)], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.log(e), rcond=None)
    return float(-coef[1]), e


def spheroid_series(ns, a_frac=0.2, alpha=1.0, tol=1e-5, max_iter=200_000, St=None, tile=(0, 0, 0, 0)):
    """C(n) for each n of `ns` (GPU, FP32 fields): list of dicts with n, phi,
    C, D = (C - C1) / phi, iterations and seconds."""
    C1 = c_iso(*MATRIX)
    out = []
    for n in ns:
        K, G, phi = images.single_spheroid(int(n), a_frac * int(n), alpha, matrix=MATRIX, inclusion=INCLUSION)
        t0 = time.perf_counter()
        with ce.Context(K, G, prec="fp32", St=St, tile=tile) as c:
            c.solve(None, tol=tol, max_iter=max_iter)
            C = c.ceff()
            iters = c.info["iters"]
        out.append({"n": int(n), "phi": phi, "C": C.tolist(), "D": ((C - C1) / phi).tolist(), "iters": iters,
                    "seconds": time.perf_counter() - t0})
    return out


def cracked_series(ns, seed=7, tol=1e-5, max_iter=200_000, St=None, tile="auto"):
    """C(n) of one crack set (images.cracked_scaled) at each n of `ns`: list of
    dicts with n, crack volume fraction, C, iterations and seconds (create,
    solve and C, the paper's time-to-C per resolution)."""
    out = []
    for n in ns:
        K, G = images.cracked_scaled(int(n), seed)
        frac = float((K < 1.0).mean())
        t0 = time.perf_counter()
        with ce.Context(K, G, prec="fp32", St=St, tile=tile) as c:
            t1 = time.perf_counter()
            c.solve(None, tol=tol, max_iter=max_iter)
            C = c.ceff()
            iters = c.info["iters"]
        t2 = time.perf_counter()
        out.append({"n": int(n), "crack_fraction": frac, "C": C.tolist(), "iters": iters,
                    "seconds": t2 - t0, "solve_seconds": t2 - t1})
    return out


def study(series, key="D"):
    """Per followed entry: the values of `key` ("D" for the spheroid, "C" for
    the cracked image) over n, the fitted order, limit and rms residual."""
    ns = [s["n"] for s in series]
    res = {}
    for (p, q) in ENTRIES:
        d = [s[key][p][q] for s in series]
        rate, dinf, b, rms = fit_rate(ns, d)
        res[f"C{p + 1}{q + 1}"] = {key: d, "order": rate, key + "_inf": dinf, "b": b, "rms": rms}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--model", choices=("sphere", "cracked"), default="sphere")
    ap.add_argument("--sizes", default=None, help="default 32,48,64,96,128 (sphere), 191,255,319,383,479 (cracked)")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--a-frac", type=float, default=0.2)
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--st", type=float, default=None, help="Strouhal number (default 2 pi sqrt 3)")
    a = ap.parse_args(argv)
    sizes = a.sizes or ("32,48,64,96,128" if a.model == "sphere" else "191,255,319,383,479")
    ns = [int(v) for v in sizes.split(",")]
    if a.model == "sphere":
        series = spheroid_series(ns, a.a_frac, a.alpha, a.tol, St=a.st)
        print(json.dumps({"model": "sphere", "sizes": ns, "a_frac": a.a_frac, "alpha": a.alpha, "tol": a.tol,
                          "series": series, "fit": study(series)}))
    else:
        series = cracked_series(ns, a.seed, a.tol, St=a.st)
        print(json.dumps({"model": "cracked", "sizes": ns, "seed": a.seed, "tol": a.tol, "series": series,
                          "fit": study(series, "C")}))


if __name__ == "__main__":
    main()
