"""ORACLE -- test infrastructure only.

Closed forms that pin the numerical oracle from outside:

* isotropic stiffness, Voigt and Reuss averages;
* Backus long-wave averaging of a stack of isotropic layers (Model 1,
  Sec. 4.1; Table 2 prints its values for the Table 1 layers);
* Hashin-Shtrikman bounds of a two-phase isotropic composite;
* the compliance contribution tensor H of an ellipsoidal inhomogeneity,
  Appendix B: H = [(S2 - S1)^-1 + Q]^-1 with Q = C1 : (I4 - s)  (Eqs. eqN21,
  eqN22), equivalently H = (S2 - S1) : Gamma with
  Gamma = [I4 + Q : (S2 - S1)]^-1 (Eq. eqN24), and the non-interaction
  estimate S* = S1 + phi H (Eq. eqN2); here with the textbook Eshelby tensor
  of a sphere;
* the textbook dilute strain concentration of a sphere (Eshelby), used to
  pin the Appendix-B algebra.

Voigt matrices use engineering shear strain; fourth-order tensor algebra is
done in Mandel form (shear rows and columns scaled by sqrt 2) so that double
contraction is a matrix product.
"""
from __future__ import annotations

import numpy as np

_F = np.array([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])


def c_iso(K, G):
    """6x6 Voigt stiffness of an isotropic solid."""
    lam = K - 2.0 * G / 3.0
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[[0, 1, 2], [0, 1, 2]] = lam + 2.0 * G
    C[[3, 4, 5], [3, 4, 5]] = G
    return C


def voigt_to_mandel_stiffness(C):
    return C * np.outer(_F, _F)


def mandel_to_voigt_stiffness(M):
    return M / np.outer(_F, _F)


def voigt_to_mandel_compliance(S):
    return S / np.outer(_F, _F)


def voigt_bound(K, G):
    """<C> for isotropic voxels: C_iso(mean K, mean G)."""
    return c_iso(float(np.mean(np.asarray(K, np.float64))), float(np.mean(np.asarray(G, np.float64))))


def reuss_bound(K, G):
    """<C^-1>^-1 for isotropic voxels."""
    K = np.asarray(K, np.float64).ravel()
    G = np.asarray(G, np.float64).ravel()
    # compliance of an isotropic solid is linear in 1/K and 1/G
    invK = float(np.mean(1.0 / K))
    invG = float(np.mean(1.0 / G))
    S = np.zeros((6, 6))
    # S = (1/9K) 1 1^T + (1/2G)(I - 1/3 1 1^T) on the normal block, 1/G on shear (Voigt)
    S[:3, :3] = invK / 9.0 - invG / 6.0
    S[[0, 1, 2], [0, 1, 2]] = invK / 9.0 + invG / 3.0
    S[[3, 4, 5], [3, 4, 5]] = invG
    return np.linalg.inv(S)


def backus(K, G, frac):
    """Backus long-wave stiffness of isotropic layers normal to z (x3) with
    volume fractions frac; Voigt 6x6."""
    K, G, f = (np.asarray(a, np.float64) for a in (K, G, frac))
    f = f / f.sum()
    M = K + 4.0 * G / 3.0
    lam = K - 2.0 * G / 3.0
    avg = lambda a: float(np.sum(f * a))
    iM = avg(1.0 / M)
    lM = avg(lam / M)
    C = np.zeros((6, 6))
    C33 = 1.0 / iM
    C13 = lM / iM
    C11 = avg(M - lam * lam / M) + lM * lM / iM
    C12 = avg(lam - lam * lam / M) + lM * lM / iM
    C[0, 0] = C[1, 1] = C11
    C[2, 2] = C33
    C[0, 1] = C[1, 0] = C12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = C13
    C[3, 3] = C[4, 4] = 1.0 / avg(1.0 / G)
    C[5, 5] = avg(G)
    return C


def hashin_shtrikman(K1, G1, K2, G2, f2):
    """(K_lower, K_upper, G_lower, G_upper) of a two-phase isotropic composite
    with phase-2 fraction f2 (well-ordered or not: both assignments are
    evaluated and sorted)."""
    f1 = 1.0 - f2

    def hs(Ka, Ga, Kb, Gb, fb):
        fa = 1.0 - fb
        Kh = Ka + fb / (1.0 / (Kb - Ka) + fa / (Ka + 4.0 * Ga / 3.0)) if Kb != Ka else Ka
        Gh = Ga + fb / (1.0 / (Gb - Ga) + 2.0 * fa * (Ka + 2.0 * Ga) / (5.0 * Ga * (Ka + 4.0 * Ga / 3.0))) \
            if Gb != Ga else Ga
        return Kh, Gh

    ka, ga = hs(K1, G1, K2, G2, f2)
    kb, gb = hs(K2, G2, K1, G1, f1)
    return min(ka, kb), max(ka, kb), min(ga, gb), max(ga, gb)


# ------------------------------------------------------- Eshelby / Appendix B
def _vol_dev_mandel():
    one = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    P = np.outer(one, one) / 3.0
    return P, np.eye(6) - P


def eshelby_sphere_mandel(nu):
    """Eshelby tensor of a sphere in an isotropic matrix (Poisson ratio nu):
    s = alpha P_vol + beta P_dev with alpha = (1+nu)/(3(1-nu)) and
    beta = 2(4-5nu)/(15(1-nu))."""
    Pv, Pd = _vol_dev_mandel()
    alpha = (1.0 + nu) / (3.0 * (1.0 - nu))
    beta = 2.0 * (4.0 - 5.0 * nu) / (15.0 * (1.0 - nu))
    return alpha * Pv + beta * Pd


def eshelby_spheroid_mandel(nu, alpha):
    """Eshelby tensor of a spheroid with semi-axes (a, a, alpha a), symmetry
    axis z, in an isotropic matrix of Poisson ratio nu, in Mandel form
    (Voigt order xx, yy, zz, yz, xz, xy).  Closed forms of the spheroid's
    depolarisation integrals (Eshelby 1957, as tabulated for spheroids by Mura
    and by Tandon & Weng) with the shape function
        g = alpha / (1 - alpha^2)^(3/2) (arccos alpha - alpha sqrt(1 - alpha^2))   (oblate)
        g = alpha / (alpha^2 - 1)^(3/2) (alpha sqrt(alpha^2 - 1) - arccosh alpha)  (prolate).
    alpha = 1 is the sphere (use eshelby_sphere_mandel)."""
    a2 = float(alpha) ** 2
    if abs(a2 - 1.0) < 1e-12:
        return eshelby_sphere_mandel(nu)
    if alpha < 1.0:
        g = alpha / (1.0 - a2) ** 1.5 * (np.arccos(alpha) - alpha * np.sqrt(1.0 - a2))
    else:
        g = alpha / (a2 - 1.0) ** 1.5 * (alpha * np.sqrt(a2 - 1.0) - np.arccosh(alpha))
    d = a2 - 1.0
    c2, c4 = 1.0 / (2.0 * (1.0 - nu)), 1.0 / (4.0 * (1.0 - nu))
    m = 1.0 - 2.0 * nu
    s1111 = 3.0 / (8.0 * (1.0 - nu)) * a2 / d + c4 * (m - 9.0 / (4.0 * d)) * g
    s3333 = c2 * (m + (3.0 * a2 - 1.0) / d - (m + 3.0 * a2 / d) * g)
    s1122 = c4 * (a2 / (2.0 * d) - (m + 3.0 / (4.0 * d)) * g)
    s1133 = c2 * (-a2 / d + 0.5 * (3.0 * a2 / d - m) * g)
    s3311 = c2 * (-m - 1.0 / d + (m + 3.0 / (2.0 * d)) * g)
    s1212 = c4 * (a2 / (2.0 * d) + (m - 3.0 / (4.0 * d)) * g)
    s1313 = c4 * (m - (a2 + 1.0) / d - 0.5 * (m - 3.0 * (a2 + 1.0) / d) * g)
    S = np.zeros((6, 6))
    S[0, 0] = S[1, 1] = s1111
    S[0, 1] = S[1, 0] = s1122
    S[0, 2] = S[1, 2] = s1133
    S[2, 0] = S[2, 1] = s3311
    S[2, 2] = s3333
    S[3, 3] = S[4, 4] = 2.0 * s1313      # Mandel shear entries: 2 s_ijij
    S[5, 5] = 2.0 * s1212
    return S


def poisson(K, G):
    return (3.0 * K - 2.0 * G) / (2.0 * (3.0 * K + G))


def h_tensor(C1_voigt, C2_voigt, s_mandel):
    """Compliance contribution tensor (Mandel) via Eqs. eqN21 - eqN22."""
    C1 = voigt_to_mandel_stiffness(C1_voigt)
    C2 = voigt_to_mandel_stiffness(C2_voigt)
    S1, S2 = np.linalg.inv(C1), np.linalg.inv(C2)
    Q = C1 @ (np.eye(6) - s_mandel)
    return np.linalg.inv(np.linalg.inv(S2 - S1) + Q)


def h_tensor_gamma(C1_voigt, C2_voigt, s_mandel):
    """The same tensor through the stress concentration tensor, Eq. eqN24."""
    C1 = voigt_to_mandel_stiffness(C1_voigt)
    C2 = voigt_to_mandel_stiffness(C2_voigt)
    S1, S2 = np.linalg.inv(C1), np.linalg.inv(C2)
    Q = C1 @ (np.eye(6) - s_mandel)
    Gamma = np.linalg.inv(np.eye(6) + Q @ (S2 - S1))
    return (S2 - S1) @ Gamma


def dilute_stiffness(C1_voigt, H_mandel, phi):
    """C* from S* = S1 + phi H (Eq. eqN2), returned in Voigt form."""
    S1 = np.linalg.inv(voigt_to_mandel_stiffness(C1_voigt))
    return mandel_to_voigt_stiffness(np.linalg.inv(S1 + phi * H_mandel))


def sphere_strain_concentration(K1, G1, K2, G2):
    """Textbook dilute strain concentration factors (bulk, shear) of a
    spherical inhomogeneity: eps_in = A : eps_far."""
    AK = (3.0 * K1 + 4.0 * G1) / (3.0 * K2 + 4.0 * G1)
    beta = 6.0 * (K1 + 2.0 * G1) / (5.0 * (3.0 * K1 + 4.0 * G1))
    AG = 1.0 / (1.0 + beta * (G2 - G1) / G1)
    return AK, AG


def isotropic_projection(C):
    """(K, G) of the isotropic part of a Voigt stiffness (Voigt-type average)."""
    K = (C[0, 0] + C[1, 1] + C[2, 2] + 2.0 * (C[0, 1] + C[0, 2] + C[1, 2])) / 9.0
    G = ((C[0, 0] + C[1, 1] + C[2, 2]) - (C[0, 1] + C[0, 2] + C[1, 2])
         + 3.0 * (C[3, 3] + C[4, 4] + C[5, 5])) / 15.0
    return K, G


# ------------------------------------------------ direct tests, Appendix A.3
def direct_offdiag(sig, eps, cdiag):
    """C12, C13, C23 from the combined three-face test of Appendix A.3.

    sig, eps: the volume-averaged normal stresses (<s11>, <s22>, <s33>) and
    normal strains (<e11>, <e22>, <e33>) of the test in which all three
    normal velocities are prescribed on one face each (zero on the opposite
    faces, tangential tractions free); cdiag: (C11, C22, C33) of the three
    normal tests (Appendix A.1).  Eq. D1 removes the diagonal part of Hooke's
    law, sbar_i = s_i - C_ii e_i, Eq. D2 takes ebar_i = e_i, and Eqs. D3-D5
    solve the system D3v1 of the three remaining unknowns."""
    s = np.asarray(sig, np.float64) - np.asarray(cdiag, np.float64) * np.asarray(eps, np.float64)   # Eq. D1
    e = np.asarray(eps, np.float64)                                                                  # Eq. D2
    c12 = (e[0] * s[0] + e[1] * s[1] - e[2] * s[2]) / (2.0 * e[0] * e[1])                            # Eq. D3
    c13 = (e[0] * s[0] - e[1] * s[1] + e[2] * s[2]) / (2.0 * e[0] * e[2])                            # Eq. D4
    c23 = (-e[0] * s[0] + e[1] * s[1] + e[2] * s[2]) / (2.0 * e[1] * e[2])                           # Eq. D5
    return c12, c13, c23
