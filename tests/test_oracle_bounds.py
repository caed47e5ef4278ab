"""Pins of the oracle's bound and projection formulas (oracle/analytic.py)
against results derived here by other routes:

* the Hashin-Shtrikman bulk bound with the stiff phase as coating equals the
  exact bulk modulus of Hashin's coated-sphere assemblage, obtained by
  solving the radial elasticity problem of one composite sphere;
* at f2 -> 0 the slopes of the HS bounds (matrix as reference) are the
  dilute Eshelby results dK/df = (K2 - K1) A_K, dG/df = (G2 - G1) A_G with the
  strain concentration computed from the sphere's Eshelby tensor;
* the end points f2 = 0, 1 and identical phases;
* the Reuss bound's compliance is the volume average of the voxel
  compliances (each inverted numerically), and its isotropic moduli are the
  harmonic means 1/<1/K>, 1/<1/G>; its shear entry equals Backus' C44 for a
  layered stack;
* the isotropic projection returns (K, G) of an isotropic C and the
  Voigt-averaged moduli (C11 + 2 C12)/3, (C11 - C12 + 3 C44)/5 of a cubic C.
Each formula is one a plausible slip (a wrong modulus in a denominator, a
wrong factor on the shear term) would move, and these checks catch it.
"""
import numpy as np
import pytest

from oracle import analytic

PAIRS = [(70.0, 30.0, 2.25, 1e-3), (36.0, 44.0, 10.0, 5.0), (5.0, 2.0, 80.0, 40.0), (70.0, 30.0, 1e-4, 1e-4)]


def coated_sphere_bulk(Kc, Gc, Ki, f_in):
    """Bulk modulus of a composite sphere (inclusion Ki of volume fraction
    f_in, coating Kc, Gc) under a uniform dilatation of its surface: radial
    displacement u = C r in the core, A r + B / r^2 in the coating; continuity
    of u and of the radial stress (3K A - 4G B / r^3 in the coating, 3 Ki C in
    the core) at r = a, u(b) = e b at the surface; K* = sigma_rr(b) / (3 e)."""
    b = 1.0
    a = f_in ** (1.0 / 3.0) * b
    e = 1.0
    # unknowns A, B, C
    M = np.array([[a, 1.0 / a ** 2, -a],
                  [3.0 * Kc, -4.0 * Gc / a ** 3, -3.0 * Ki],
                  [b, 1.0 / b ** 2, 0.0]])
    A, B, _ = np.linalg.solve(M, np.array([0.0, 0.0, e * b]))
    return (3.0 * Kc * A - 4.0 * Gc * B / b ** 3) / (3.0 * e)


@pytest.mark.parametrize("K1,G1,K2,G2", PAIRS)
@pytest.mark.parametrize("f2", [0.05, 0.3, 0.7])
def test_hs_bulk_bound_is_the_coated_sphere_assemblage(K1, G1, K2, G2, f2):
    Kl, Ku, _, _ = analytic.hashin_shtrikman(K1, G1, K2, G2, f2)
    # the bound attained with the phase of larger shear modulus as coating
    if G1 >= G2:
        exact = coated_sphere_bulk(K1, G1, K2, f2)
    else:
        exact = coated_sphere_bulk(K2, G2, K1, 1.0 - f2)
    stiff_coating_is_upper = (K1 - K2) * (G1 - G2) >= 0
    got = Ku if stiff_coating_is_upper else Kl
    assert abs(got - exact) <= 1e-12 * max(K1, K2)


def dilute_concentration(K1, G1, K2, G2):
    """Strain concentration A = [I + s S1 (C2 - C1)]^-1 of a sphere from the
    Eshelby tensor s (Mandel); returns its volumetric and deviatoric
    eigenvalues."""
    nu = analytic.poisson(K1, G1)
    s = analytic.eshelby_sphere_mandel(nu)
    C1 = analytic.voigt_to_mandel_stiffness(analytic.c_iso(K1, G1))
    C2 = analytic.voigt_to_mandel_stiffness(analytic.c_iso(K2, G2))
    A = np.linalg.inv(np.eye(6) + s @ np.linalg.inv(C1) @ (C2 - C1))
    vol = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0]) / np.sqrt(3.0)
    dev = np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    return vol @ A @ vol, dev @ A @ dev


@pytest.mark.parametrize("K1,G1,K2,G2", PAIRS)
def test_hs_slopes_at_the_dilute_limit_are_eshelbys(K1, G1, K2, G2):
    AK, AG = dilute_concentration(K1, G1, K2, G2)
    h = 1e-7
    # the bound whose reference medium is phase 1 (the matrix)
    def hs_matrix(f):
        Kl, Ku, Gl, Gu = analytic.hashin_shtrikman(K1, G1, K2, G2, f)
        Kref = Ku if (K1 - K2) * (G1 - G2) >= 0 and G1 >= G2 else Kl
        Gref = Gu if G1 >= G2 else Gl
        return Kref, Gref
    K0, G0 = hs_matrix(0.0)
    Kh, Gh = hs_matrix(h)
    assert abs(K0 - K1) <= 1e-12 * K1 and abs(G0 - G1) <= 1e-12 * G1
    assert abs((Kh - K0) / h - (K2 - K1) * AK) <= 1e-5 * abs(K2 - K1)
    assert abs((Gh - G0) / h - (G2 - G1) * AG) <= 1e-5 * abs(G2 - G1)


@pytest.mark.parametrize("K1,G1,K2,G2", PAIRS)
def test_hs_end_points_and_identical_phases(K1, G1, K2, G2):
    for f2, (K, G) in ((0.0, (K1, G1)), (1.0, (K2, G2))):
        Kl, Ku, Gl, Gu = analytic.hashin_shtrikman(K1, G1, K2, G2, f2)
        for v, ref in ((Kl, K), (Ku, K), (Gl, G), (Gu, G)):
            assert abs(v - ref) <= 1e-12 * max(K1, K2, G1, G2)
    Kl, Ku, Gl, Gu = analytic.hashin_shtrikman(K1, G1, K1, G1, 0.4)
    assert Kl == Ku == K1 and Gl == Gu == G1


def test_reuss_bound_is_the_averaged_compliance():
    rng = np.random.default_rng(4)
    K = rng.uniform(1.0, 80.0, 37)
    G = rng.uniform(0.5, 40.0, 37)
    S = np.mean([np.linalg.inv(analytic.c_iso(k, g)) for k, g in zip(K, G)], axis=0)
    C = analytic.reuss_bound(K, G)
    assert np.abs(C - np.linalg.inv(S)).max() <= 1e-10 * np.abs(C).max()
    Kr, Gr = analytic.isotropic_projection(C)
    assert abs(Kr - 1.0 / np.mean(1.0 / K)) <= 1e-10 * Kr
    assert abs(Gr - 1.0 / np.mean(1.0 / G)) <= 1e-10 * Gr
    # identical voxels: the single-phase stiffness
    assert np.abs(analytic.reuss_bound([7.0] * 5, [3.0] * 5) - analytic.c_iso(7.0, 3.0)).max() <= 1e-12


def test_reuss_shear_equals_backus_c44_of_layers():
    K = np.array([70.0, 2.25, 36.0])
    G = np.array([30.0, 1.0, 44.0])
    f = np.array([0.2, 0.5, 0.3])
    B = analytic.backus(K, G, f)
    # the Reuss bound of voxels in these proportions
    Kv = np.repeat(K, (f * 10).astype(int))
    Gv = np.repeat(G, (f * 10).astype(int))
    R = analytic.reuss_bound(Kv, Gv)
    assert abs(R[3, 3] - B[3, 3]) <= 1e-12 * B[3, 3]
    assert abs(R[4, 4] - B[4, 4]) <= 1e-12 * B[4, 4]


def test_isotropic_projection_of_isotropic_and_cubic_stiffness():
    for K, G in ((70.0, 30.0), (2.25, 1e-3), (36.0, 44.0)):
        k, g = analytic.isotropic_projection(analytic.c_iso(K, G))
        assert abs(k - K) <= 1e-12 * K and abs(g - G) <= 1e-12 * max(G, 1.0)
    C11, C12, C44 = 168.4, 121.4, 75.4       # a cubic crystal's three constants (GPa)
    C = np.zeros((6, 6))
    C[:3, :3] = C12
    C[[0, 1, 2], [0, 1, 2]] = C11
    C[[3, 4, 5], [3, 4, 5]] = C44
    k, g = analytic.isotropic_projection(C)
    assert abs(k - (C11 + 2 * C12) / 3) <= 1e-12 * k
    assert abs(g - (C11 - C12 + 3 * C44) / 5) <= 1e-12 * g
