"""Adjoint gradient dJ/dK, dJ/dG of J = sum_mn w_mn C_mn on porous images
(the FP32 forward + adjoint, i.e. the autograd path; w seeded, N(0, 1)).

* 24^3, 15 % porosity: against the FP64 CPU oracle's closed-form gradient
  from a sparse direct solve, voxel by voxel.
* 127^3 (the adjoint workload), 15 % porosity: against central finite
  differences of J, one voxel at a time, on 16 seeded voxels: 6 matrix
  voxels next to a pore, 4 pore voxels next to the matrix and 6 matrix
  voxels at least 3 voxels from any pore; dJ/dK and dJ/dG each.  Every J
  comes from a refined FP32 solve (the FP64 residual decides convergence,
  the averages are FP64) converged to tol 1e-13, warm-started from the base
  fields (ce_set_moduli).
* 48^3: the same on 4 voxels (2 next to a pore, 1 pore, 1 far from any
  pore) with every J from the FP64 path (prec="fp64"), the plain
  one-case-at-a-time FP64 solve.

Accuracy of the FP32 gradient.  The residual weighs each equation by the
local modulus, so the strains inside near-void pores (1e-4 GPa, six orders
below the matrix) converge last; the gradient's error in pores follows the
tolerance (measured at 24^3 against the oracle: 2.7e-2, 1.1e-3 and 2.1e-5 of
the pores' largest entry at tol 1e-6, 1e-8, 1e-10; matrix voxels 1.2e-6,
2.8e-8, 1.9e-8).  The tests solve to tol 1e-10 and allow 2e-4 in pores, 1e-6
in the matrix.

Finite differences.  Central, with h = 5 % of the modulus in the matrix
and 10 % in pores (a pore voxel's neighbours are pores of the same modulus,
so its response is smooth only on the scale of its own modulus: a secant
over [0.1, 10] x the modulus was off by a factor 2).  Measured at 127^3, the
central difference of a pore voxel changes by less than 1e-3 between
h = 5, 10 and 20 %.  Each derivative is held to 1e-2 of its value plus
0.05 tol sum |w_mn C_mn| over the step (the part of J the tolerance leaves
unresolved).
"""
import numpy as np
import pytest

from oracle import apt, operator
from paper_2410_20441_gb300 import images

pytestmark = pytest.mark.gpu

FD_TOL = 1e-13


@pytest.fixture(scope="module")
def ce():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_20441_gb300 import ce as cemod
    cemod.load()
    return cemod


def _autograd(K, G, W, tol, St):
    import torch
    from paper_2410_20441_gb300 import autograd
    Kt = torch.tensor(K, device="cuda", requires_grad=True)
    Gt = torch.tensor(G, device="cuda", requires_grad=True)
    C = autograd.ceff(Kt, Gt, tol=tol, St=St)
    (C * torch.tensor(W, device="cuda")).sum().backward()
    return C.detach().cpu().numpy(), Kt.grad.cpu().numpy(), Gt.grad.cpu().numpy()


def _phase_err(g, ref, mask):
    return np.abs(g - ref)[mask].max() / np.abs(ref[mask]).max()


def test_adjoint_24_fp32_matches_fp64_cpu_oracle(ce):
    K, G = images.random_spheres(24, 0.15, seed=24)
    W = images.adjoint_weights(7)
    d = operator.solve_all(K, G)
    dK, dG = d["op"].grad_C(d["strains"], W)
    C, gK, gG = _autograd(K, G, W, 1e-10, apt.ST_POROUS)
    pore = K < 1.0
    assert np.abs(C - d["C"]).max() <= 1e-9 * np.abs(d["C"]).max()
    for g, ref in ((gK, dK), (gG, dG)):
        assert _phase_err(g, ref, ~pore) <= 1e-6
        assert _phase_err(g, ref, pore) <= 2e-4


def fd_voxels(K, seed, small=False):
    """6 matrix voxels next to a pore, 4 pore voxels next to the matrix, 6
    matrix voxels at least 3 voxels from any pore (flat indices)."""
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    pore = K < 1.0
    st = ndimage.generate_binary_structure(3, 1)
    near_pore = ndimage.binary_dilation(pore, st)
    near_solid = ndimage.binary_dilation(~pore, st)
    far = ~pore & ~ndimage.binary_dilation(pore, st, iterations=3)
    sets = ((~pore & near_pore, 6, "interface"), (pore & near_solid, 4, "pore"), (far, 6, "far"))
    if small:
        sets = ((~pore & near_pore, 2, "interface"), (pore & near_solid, 1, "pore"), (far, 1, "far"))
    out = []
    for mask, n, kind in sets:
        idx = np.flatnonzero(mask.ravel())
        out += [(int(v), kind) for v in rng.choice(idx, n, replace=False)]
    return out


def per_voxel_fd(ce, K, G, W, prec, St, vox):
    """dJ/dK and dJ/dG at each voxel by finite differences of warm-started
    solves converged to FD_TOL; returns {(voxel, 'K'|'G'): (fd, budget)}."""
    out = {}
    Kf, Gf = K.ravel(), G.ravel()
    with ce.Context(K, G, prec=prec, St=St) as c:
        c.solve(None, tol=FD_TOL, max_iter=400000)
        C0 = c.ceff()
        scale = float(np.abs(W * C0).sum())
        for v, kind in vox:
            for which, base in (("K", Kf), ("G", Gf)):
                m0 = float(base[v])
                h = 0.1 if kind == "pore" else 0.05
                lo, hi = (1.0 - h) * m0, (1.0 + h) * m0
                J = []
                for val in (hi, lo):
                    Kp, Gp = Kf.copy(), Gf.copy()
                    (Kp if which == "K" else Gp)[v] = val
                    c.set_moduli(Kp.reshape(K.shape), Gp.reshape(G.shape))
                    c.solve(None, tol=FD_TOL, max_iter=400000, warm=True)
                    J.append(float((c.ceff() * W).sum()))
                # the moduli are FP32: difference of the values actually applied
                step = float(np.float32(hi)) - float(np.float32(lo))
                out[(v, which)] = ((J[0] - J[1]) / step, 0.05 * FD_TOL * scale / step)
        c.set_moduli(K, G)
    return out


def _check_fd(fd, gK, gG, vox):
    worst = 0.0
    for v, kind in vox:
        for which, g in (("K", gK.ravel()[v]), ("G", gG.ravel()[v])):
            val, budget = fd[(v, which)]
            err = abs(val - g)
            assert err <= 1e-2 * abs(g) + budget, (kind, which, v, val, g, budget)
            worst = max(worst, err / max(abs(g), 1e-30))
    return worst


def test_adjoint_48_fp64_central_differences_per_voxel(ce):
    K, G = images.random_spheres(48, 0.15, seed=48)
    W = images.adjoint_weights(7)
    _, gK, gG = _autograd(K, G, W, 1e-10, apt.ST_POROUS)
    vox = fd_voxels(K, seed=16, small=True)
    fd = per_voxel_fd(ce, K, G, W, "fp64", apt.ST_POROUS, vox)
    worst = _check_fd(fd, gK, gG, vox)
    print(f"\n48^3 FP64 finite differences: worst relative difference {worst:.2e} over {2 * len(vox)} derivatives")


def test_adjoint_127_central_differences_per_voxel(ce):
    K, G = images.random_spheres(127, 0.15, seed=127)
    W = images.adjoint_weights(7)
    _, gK, gG = _autograd(K, G, W, 1e-10, apt.ST_POROUS)
    vox = fd_voxels(K, seed=16)
    fd = per_voxel_fd(ce, K, G, W, "fp32", apt.ST_POROUS, vox)
    worst = _check_fd(fd, gK, gG, vox)
    print(f"\n127^3 refined-FP32 finite differences: worst relative difference {worst:.2e} over "
          f"{2 * len(vox)} derivatives")
