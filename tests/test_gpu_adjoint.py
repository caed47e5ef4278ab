"""Adjoint gradient dJ/dK, dJ/dG of J = sum_mn w_mn C_mn on porous images.

* 24^3 (15 % porosity): the FP32 forward + adjoint (the autograd path)
  against the FP64 CPU oracle's closed-form gradient from a sparse direct
  solve;
* 127^3 (15 % porosity, the adjoint workload): the FP32 gradient against the
  FP64 GPU gradient, and both against a central finite difference of J in
  the direction of a perturbation of K and G on 16 voxels (8 in the matrix,
  8 in pores), solved in FP64 with warm starts from the base fields.

Gradient tolerances are relative to the largest |entry|: the FP32 fields at
tol 1e-6 carry ~1e-6 relative error and the gradient is a product of two
strains, so 1e-3 leaves room; the pore voxels converge last and dominate.
"""
import numpy as np
import pytest

from oracle import apt, operator
from paper_2410_20441_gb300 import images

pytestmark = pytest.mark.gpu


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


def test_adjoint_24_fp32_matches_fp64_cpu_oracle(ce):
    K, G = images.random_spheres(24, 0.15, seed=24)
    W = images.adjoint_weights(7)
    d = operator.solve_all(K, G)
    dK, dG = d["op"].grad_C(d["strains"], W)
    C, gK, gG = _autograd(K, G, W, 1e-6, apt.ST_POROUS)
    assert np.abs(C - d["C"]).max() <= 1e-4 * np.abs(d["C"]).max()
    assert np.abs(gK - dK).max() <= 1e-3 * np.abs(dK).max()
    assert np.abs(gG - dG).max() <= 1e-3 * np.abs(dG).max()


@pytest.mark.slow
def test_adjoint_127_fp32_and_fp64_against_finite_differences(ce):
    K, G = images.random_spheres(127, 0.15, seed=127)
    W = images.adjoint_weights(7)
    C32, gK32, gG32 = _autograd(K, G, W, 1e-6, apt.ST_POROUS)
    with ce.Context(K, G, prec="fp64", St=apt.ST_POROUS) as c:
        c.solve(None, tol=1e-12, max_iter=400000)
        C64 = c.ceff()
        gK64, gG64 = c.grad(W)
        assert np.abs(C32 - C64).max() <= 1e-4 * np.abs(C64).max()
        assert np.abs(gK32 - gK64).max() <= 1e-3 * np.abs(gK64).max()
        assert np.abs(gG32 - gG64).max() <= 1e-3 * np.abs(gG64).max()

        rng = np.random.default_rng(16)
        pore = np.flatnonzero(K.ravel() < 1.0)
        solid = np.flatnonzero(K.ravel() >= 1.0)
        vox = np.concatenate([rng.choice(solid, 8, replace=False), rng.choice(pore, 8, replace=False)])
        dKp = np.zeros(K.size)
        dGp = np.zeros(K.size)
        h = 1e-3
        dKp[vox] = h * K.ravel()[vox] * rng.choice([-1.0, 1.0], 16)
        dGp[vox] = h * G.ravel()[vox] * rng.choice([-1.0, 1.0], 16)
        dKp = dKp.reshape(K.shape).astype(np.float32)
        dGp = dGp.reshape(K.shape).astype(np.float32)
        J = []
        for sgn in (1.0, -1.0):
            Kp, Gp = (K + sgn * dKp).astype(np.float32), (G + sgn * dGp).astype(np.float32)
            c.set_moduli(Kp, Gp)
            c.solve(None, tol=1e-12, max_iter=400000, warm=True)
            J.append(float((c.ceff() * W).sum()))
        # the perturbation actually applied (float32 moduli)
        aK = ((K + dKp).astype(np.float32).astype(np.float64) - (K - dKp).astype(np.float32)) / 2
        aG = ((G + dGp).astype(np.float32).astype(np.float64) - (G - dGp).astype(np.float32)) / 2
        fd = (J[0] - J[1]) / 2
        for gK, gG, bound in ((gK64, gG64, 1e-4), (gK32, gG32, 2e-3)):
            pred = float((gK.astype(np.float64) * aK).sum() + (gG.astype(np.float64) * aG).sum())
            assert abs(fd - pred) <= bound * abs(pred), (fd, pred)
