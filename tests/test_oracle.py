"""Pins of the CPU oracle against facts fixed from outside it: closed forms,
values the paper prints, mathematical invariants and an independent route
(direct solve of the assembled operator).  No GPU is needed."""
import json
import os

import numpy as np
import pytest

from oracle import analytic, apt, operator
from paper_2410_20441_gb300 import images

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


# ------------------------------------------------------------ closed forms
def test_backus_reproduces_table2():
    """Backus averaging of the Table 1 layers at the stiff fraction 90/191
    gives the analytical column of Table 2 to its printed digits."""
    g = json.load(open(os.path.join(GOLDEN, "table2_backus.json")))
    f = g["layers"]["stiff_fraction_voxels"]
    C = analytic.backus(g["layers"]["K"], g["layers"]["G"], [f[0], f[1] - f[0]])
    tab = {"C11": C[0, 0], "C22": C[1, 1], "C33": C[2, 2], "C44": C[3, 3], "C55": C[4, 4],
           "C66": C[5, 5], "C12": C[0, 1], "C13": C[0, 2], "C23": C[1, 2]}
    for k, v in tab.items():
        assert round(v, 3) == pytest.approx(g[k], abs=1e-9), (k, v, g[k])


def test_h_tensor_appendix_b_matches_textbook_sphere():
    """Appendix B's H (Eq. eqN21 with Q of Eq. eqN22) satisfies the exact
    identity C1 H C1 = (C1 - C2) A, where A is the textbook strain
    concentration of a sphere; the Gamma form (Eq. eqN24) agrees."""
    for K1, G1, K2, G2 in [(70.0, 30.0, 2.25, 1e-3), (36.0, 44.0, 1e-3, 2e-3), (10.0, 5.0, 80.0, 60.0)]:
        C1, C2 = analytic.c_iso(K1, G1), analytic.c_iso(K2, G2)
        s = analytic.eshelby_sphere_mandel(analytic.poisson(K1, G1))
        H = analytic.h_tensor(C1, C2, s)
        Hg = analytic.h_tensor_gamma(C1, C2, s)
        assert np.allclose(H, Hg, rtol=1e-10, atol=1e-14)
        AK, AG = analytic.sphere_strain_concentration(K1, G1, K2, G2)
        Pv, Pd = analytic._vol_dev_mandel()
        A = AK * Pv + AG * Pd
        M1 = analytic.voigt_to_mandel_stiffness(C1)
        M2 = analytic.voigt_to_mandel_stiffness(C2)
        assert np.allclose(M1 @ H @ M1, (M1 - M2) @ A, rtol=1e-9, atol=1e-9 * np.abs(M1).max())


def test_hashin_shtrikman_contains_voigt_reuss_order():
    Kl, Ku, Gl, Gu = analytic.hashin_shtrikman(70.0, 30.0, 2.25, 1e-3, 0.2)
    assert Kl <= Ku and Gl <= Gu
    CV = analytic.voigt_bound([70.0] * 4 + [2.25], [30.0] * 4 + [1e-3])
    assert Ku <= (CV[0, 0] + 2 * CV[0, 1]) / 3 + 1e-9


# ------------------------------------------------------- homogeneous body
@pytest.mark.parametrize("shape", [(5, 6, 7), (9, 4, 3)])
def test_homogeneous_cube_is_exact(shape):
    K, G = images.homogeneous(shape, 70.0, 30.0)
    r = apt.solve(K, G, tol=1e-12)
    assert all(c.iters == 0 and c.status == 0 for c in r.cases)
    assert rel(r.C, analytic.c_iso(70.0, 30.0)) < 1e-14
    d = operator.solve_all(K, G)
    assert rel(d["C"], analytic.c_iso(70.0, 30.0)) < 1e-13


# ------------------------------------------------- R1 (APT) == R2 (direct)
@pytest.mark.parametrize("maker", [lambda: images.random_moduli(8, seed=3),
                                   lambda: images.two_phase_random((5, 6, 7), seed=4, frac=0.3,
                                                                   inclusion=(5.0, 2.0))])
def test_apt_fixed_point_equals_direct_solve(maker):
    K, G = maker()
    r = apt.solve(K, G, tol=1e-13, n_check=8, keep_state=True)
    assert all(c.status == 0 for c in r.cases)
    d = operator.solve_all(K, G)
    assert rel(r.C, d["C"]) < 1e-10
    op = d["op"]
    nz, ny, nx = K.shape
    for m in range(6):
        st = r.cases[m].state
        w = np.concatenate([st[6][:nz, :ny, :].ravel(), st[7][:nz, :, :nx].ravel(),
                            st[8][:, :ny, :nx].ravel()])
        assert np.abs(w - d["w"][m]).max() < 1e-9 * max(1.0, np.abs(d["w"][m]).max())


def test_c_residual_is_gradient_of_energy():
    """The C oracle's elastic-operator residual equals ||B^T D s(w)|| of the
    independently assembled energy, for an arbitrary state."""
    K, G = images.random_moduli((5, 4, 6), seed=11)
    op = operator.Operator(K, G)
    rng = np.random.default_rng(0)
    e6 = rng.normal(size=6)
    wf = rng.normal(size=op.A.shape[0])
    wfull = op.full_w(wf)
    nz, ny, nx = K.shape
    st = np.zeros(apt.state_shape(nx, ny, nz))
    st[6][:nz, :ny, :] = wfull[:op.off_wy].reshape(op.shp_wx)
    st[7][:nz, :, :nx] = wfull[op.off_wy:op.off_wz].reshape(op.shp_wy)
    st[8][:, :ny, :nx] = wfull[op.off_wz:].reshape(op.shp_wz)
    r_c = apt.residual_norm(K, G, e6, st)
    r_np = np.linalg.norm(op.residual(wfull, e6))
    assert abs(r_c - r_np) <= 1e-12 * r_np


def test_operator_is_symmetric_positive_definite():
    K, G = images.random_moduli((4, 5, 3), seed=2)
    A = operator.Operator(K, G).A.toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    np.linalg.cholesky(A)


# ---------------------------------------------------------- invariants
def test_average_form_equals_energy_form_and_major_symmetry():
    K, G = images.two_phase_random((6, 5, 7), seed=8, frac=0.35, inclusion=(2.25, 1e-3))
    d = operator.solve_all(K, G)
    assert rel(d["C"], d["C_energy"]) < 1e-10
    assert rel(d["C"], d["C"].T) < 1e-10
    assert np.abs(d["E"] - np.eye(6)).max() < 1e-13


def test_mean_strain_is_the_macroscopic_strain():
    K, G = images.random_moduli((6, 7, 5), seed=5)
    r = apt.solve(K, G, tol=1e-6)
    assert np.abs(r.E - np.eye(6)).max() < 1e-13


def test_voigt_and_reuss_bounds():
    K, G = images.random_moduli(7, seed=21)
    C = operator.solve_all(K, G)["C"]
    Cs = 0.5 * (C + C.T)
    assert np.linalg.eigvalsh(analytic.voigt_bound(K, G) - Cs).min() > -1e-9
    assert np.linalg.eigvalsh(Cs - analytic.reuss_bound(K, G)).min() > -1e-9


def test_axis_permutation_permutes_c():
    K, G = images.random_moduli((5, 6, 7), seed=9)
    C = operator.solve_all(K, G)["C"]
    # swap x and z: array axes (z,y,x) -> (x,y,z); Voigt xx<->zz, yz<->xy
    Ct = operator.solve_all(np.ascontiguousarray(K.transpose(2, 1, 0)),
                            np.ascontiguousarray(G.transpose(2, 1, 0)))["C"]
    perm = [2, 1, 0, 5, 4, 3]
    assert rel(Ct, C[np.ix_(perm, perm)]) < 1e-10


def test_mirror_flips_odd_couplings():
    K, G = images.random_moduli((5, 4, 6), seed=13)
    C = operator.solve_all(K, G)["C"]
    Cm = operator.solve_all(np.ascontiguousarray(K[:, :, ::-1]), np.ascontiguousarray(G[:, :, ::-1]))["C"]
    sgn = np.array([1, 1, 1, 1, -1, -1])   # xz and xy change sign under x -> -x
    assert rel(Cm, C * np.outer(sgn, sgn)) < 1e-10


def test_scaling_moduli_scales_c():
    K, G = images.random_moduli(5, seed=17)
    K, G = K.astype(np.float64), G.astype(np.float64)
    C = apt.solve(K, G, tol=1e-12).C
    C2 = apt.solve(2.0 * K, 2.0 * G, tol=1e-12).C     # exact scaling in binary
    assert rel(C2, 2.0 * C) < 1e-13


# ------------------------------------------------------------ laminates
def test_roller_laminate_normal_block_is_backus():
    """Model 1 (Sec. 4.1): with rollers (Appendix A.1: normal velocity
    prescribed, tangential motion free) the 1-D layer solution is exact on the
    grid, so the normal block equals Backus at any lateral size."""
    K, G = images.laminate((3, 3, 191))
    r = apt.solve(K, G, loads=np.eye(6)[:3], tol=1e-12, bc=1, max_iter=400000)
    assert all(c.status == 0 for c in r.cases)
    Cn = r.S[:3, :3] @ np.linalg.inv(r.E[:3, :3])
    B = analytic.backus([7.2, 36.0], [8.8, 44.0], [101, 90])
    assert rel(Cn, B[:3, :3]) < 1e-7


def test_kubc_laminate_in_plane_shear_is_mean_g():
    """Layers normal to z under uniform kinematic conditions: the affine
    in-plane shear field is already in equilibrium, so C66 = <G> exactly."""
    K, G = images.laminate((6, 5, 30), layer=4)
    r = apt.solve(K, G, loads=np.eye(6)[5:6], tol=1e-12)
    assert r.cases[0].iters == 0
    assert abs(r.S[5, 0] - float(np.mean(G.astype(np.float64)))) < 1e-12


# ----------------------------------------------------------- inclusions
def test_centred_sphere_has_cubic_symmetry():
    K, G = images.single_sphere(11, radius_frac=0.3)
    C = operator.solve_all(K, G)["C"]
    s = np.abs(C).max()
    assert abs(C[0, 0] - C[1, 1]) < 1e-10 * s and abs(C[0, 0] - C[2, 2]) < 1e-10 * s
    assert abs(C[3, 3] - C[4, 4]) < 1e-10 * s and abs(C[3, 3] - C[5, 5]) < 1e-10 * s
    assert abs(C[0, 1] - C[0, 2]) < 1e-10 * s and abs(C[0, 1] - C[1, 2]) < 1e-10 * s
    assert np.abs(C[:3, 3:]).max() < 1e-10 * s and np.abs(C[3:, 3:] - np.diag(np.diag(C[3:, 3:]))).max() < 1e-10 * s


@pytest.mark.slow
@pytest.mark.parametrize("nu", [0.0658, 0.25, 0.3])
def test_spheroid_eshelby_limits(nu):
    """The spheroid's Eshelby tensor reduces to the sphere's at alpha = 1, to
    the penny-shaped crack's (s3333 = 1, s3311 = nu/(1-nu), s1313 = 1/2,
    others 0) as alpha -> 0 and to the circular cylinder's
    (s1111 = (5-4nu)/(8(1-nu)), s1122 = (4nu-1)/(8(1-nu)),
    s1133 = nu/(2(1-nu)), s1212 = (3-4nu)/(8(1-nu)), s1313 = 1/4, s33kl = 0)
    as alpha -> infinity; its normal block keeps s1111 = s2222, s1133 = s2233."""
    sph = analytic.eshelby_sphere_mandel(nu)
    # the closed forms cancel near alpha = 1: compare the symmetric mean of
    # alpha = 1 -+ h (first-order terms cancel, the rest is O(h^2))
    h = 1e-3
    mid = 0.5 * (analytic.eshelby_spheroid_mandel(nu, 1.0 - h) + analytic.eshelby_spheroid_mandel(nu, 1.0 + h))
    assert np.abs(mid - sph).max() < 1e-5
    P = analytic.eshelby_spheroid_mandel(nu, 1e-7)
    pen = np.zeros((6, 6))
    pen[2, 2] = 1.0
    pen[2, 0] = pen[2, 1] = nu / (1.0 - nu)
    pen[3, 3] = pen[4, 4] = 1.0                      # Mandel: 2 * s1313
    assert np.abs(P - pen).max() < 1e-5
    Cy = analytic.eshelby_spheroid_mandel(nu, 1e8)
    cyl = np.zeros((6, 6))
    cyl[0, 0] = cyl[1, 1] = (5 - 4 * nu) / (8 * (1 - nu))
    cyl[0, 1] = cyl[1, 0] = (4 * nu - 1) / (8 * (1 - nu))
    cyl[0, 2] = cyl[1, 2] = nu / (2 * (1 - nu))
    cyl[5, 5] = 2 * (3 - 4 * nu) / (8 * (1 - nu))
    cyl[3, 3] = cyl[4, 4] = 0.5
    assert np.abs(Cy - cyl).max() < 1e-6
    for a in (0.1, 0.5, 3.0):
        S = analytic.eshelby_spheroid_mandel(nu, a)
        assert S[0, 0] == S[1, 1] and S[0, 2] == S[1, 2] and S[2, 0] == S[2, 1] and S[3, 3] == S[4, 4]


def test_dilute_sphere_against_eshelby_and_hs_bounds():
    """A small centred stiff-matrix / soft-sphere composite lies near the
    Appendix-B non-interaction estimate (Eq. eqN2) and inside the
    Hashin-Shtrikman bounds of its isotropic part.  Uniform kinematic
    conditions make the sample stiffer than the dilute estimate (Sec. 5.1)."""
    n = 21
    K, G = images.single_sphere(n, radius_frac=0.2, inclusion=(5.0, 2.0))
    phi = float(np.mean(K < 10))
    C = apt.solve(K, G, tol=1e-10).C
    C1, C2 = analytic.c_iso(70.0, 30.0), analytic.c_iso(5.0, 2.0)
    H = analytic.h_tensor(C1, C2, analytic.eshelby_sphere_mandel(analytic.poisson(70.0, 30.0)))
    Cd = analytic.dilute_stiffness(C1, H, phi)
    Ki, Gi = analytic.isotropic_projection(C)
    Kd, Gd = analytic.isotropic_projection(Cd)
    assert abs(Ki - Kd) / Kd < 0.02 and abs(Gi - Gd) / Gd < 0.03
    # a finite sample under uniform kinematic conditions may exceed the
    # (infinite-medium) upper bound slightly; allow 1 %
    Kl, Ku, Gl, Gu = analytic.hashin_shtrikman(70.0, 30.0, 5.0, 2.0, phi)
    assert Kl <= Ki <= Ku * 1.01 and Gl <= Gi <= Gu * 1.01


# ------------------------------------------------------------- gradient
def test_adjoint_gradient_matches_finite_differences():
    """dJ/dK_c and dJ/dG_c from the converged fields (self-adjoint operator)
    against central differences of J = sum w_mn C_mn through direct solves."""
    K, G = images.random_moduli((4, 3, 5), seed=31)
    K = K.astype(np.float64)
    G = G.astype(np.float64)
    W = images.adjoint_weights(7)
    d = operator.solve_all(K, G)
    dK, dG = d["op"].grad_C(d["strains"], W)

    def J(Kx, Gx):
        return float(np.sum(W * operator.solve_all(Kx, Gx)["C_energy"]))

    rng = np.random.default_rng(3)
    for _ in range(4):
        c = tuple(int(rng.integers(0, s)) for s in K.shape)
        for arr, g in ((K, dK), (G, dG)):
            h = 1e-4 * arr[c]
            ap, am = arr.copy(), arr.copy()
            ap[c] += h
            am[c] -= h
            fd = (J(ap, G) - J(am, G)) / (2 * h) if arr is K else (J(K, ap) - J(K, am)) / (2 * h)
            assert abs(fd - g[c]) <= 1e-6 * np.abs(g).max() + 1e-7 * abs(g[c]), (c, fd, g[c])


# ----------------------------------------------------------- iterations
def test_iteration_count_is_a_few_times_nx():
    """Sec. 3.1: a heterogeneous 3-D model needs about 5 nx to 10 nx
    pseudo-time iterations; a mildly heterogeneous image must land in a
    loose band around that (soft pin of the numerical parameters)."""
    K, G = images.random_moduli(16, seed=1, kmin=30, kmax=80, gmin=15, gmax=40)
    r = apt.solve(K, G, loads=np.eye(6)[:1], tol=1e-6, n_check=4)
    assert r.cases[0].status == 0
    assert 4 * 16 <= r.cases[0].iters <= 12 * 16
