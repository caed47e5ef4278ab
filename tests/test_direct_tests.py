"""The paper's combined direct test for the off-diagonal stiffnesses
(Appendix A.3, Eqs. D1-D5) in the oracle, pinned by Hooke's law itself and by
the layered medium of Model 1 (Sec. 4.1), where the roller tests are exact and
Table 2 prints the analytic values."""
import json
import os

import numpy as np
import pytest

from oracle import analytic, apt
from paper_2410_20441_gb300 import images

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ROLLER_LOADS = np.array([[1, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0], [0, 0, 1, 0, 0, 0], [1, 1, 1, 0, 0, 0]], float)


def test_d3_d5_invert_hookes_law_of_an_orthorhombic_medium():
    """For any orthorhombic C and any three nonzero normal strains, the
    averages s = C e fed through Eqs. D1-D5 return C12, C13, C23 exactly."""
    rng = np.random.default_rng(12)
    for _ in range(20):
        A = rng.normal(size=(3, 3))
        Cn = A @ A.T + 3 * np.eye(3)          # a positive definite normal block
        e = rng.uniform(0.2, 2.0, 3) * rng.choice([-1, 1], 3)
        s = Cn @ e
        c12, c13, c23 = analytic.direct_offdiag(s, e, np.diag(Cn))
        assert np.allclose([c12, c13, c23], [Cn[0, 1], Cn[0, 2], Cn[1, 2]], rtol=1e-12, atol=1e-12)


def roller_direct(K, G, tol=1e-12):
    r = apt.solve(K, G, loads=ROLLER_LOADS, tol=tol, bc=1, max_iter=400000)
    assert all(c.status == 0 for c in r.cases)
    cdiag = [r.S[q, q] / r.E[q, q] for q in range(3)]                # Eq. eq:4 for C11, C22, C33
    comb = r.cases[3]
    c12, c13, c23 = analytic.direct_offdiag(comb.sig[:3], comb.eps[:3], cdiag)
    return np.array(cdiag + [c12, c13, c23]), r


def test_combined_test_on_the_layered_medium_is_backus():
    """Layers of Table 1 normal to z (15-voxel layers, 191 along z): the
    roller tests reproduce the Backus normal block exactly, so Eqs. D3-D5
    give Backus' C12 and C13 = C23, and round to Table 2's analytic column."""
    gold = json.load(open(os.path.join(GOLDEN, "table2_backus.json")))
    K, G = images.laminate((3, 3, 191))
    Cd, r = roller_direct(K, G)
    B = analytic.backus([7.2, 36.0], [8.8, 44.0], [101, 90])
    ref = [B[0, 0], B[1, 1], B[2, 2], B[0, 1], B[0, 2], B[1, 2]]
    assert np.abs(Cd - ref).max() <= 1e-7 * B.max()
    for v, name in zip(Cd, ("C11", "C22", "C33", "C12", "C13", "C23")):
        assert round(v, 3) == pytest.approx(gold[name], abs=1.5e-3), name
    # the combined test's strains are those prescribed (rollers: <e_ii> = 1)
    assert np.allclose(r.cases[3].eps[:3], 1.0, atol=1e-12)


def test_combined_test_agrees_with_the_six_case_stiffness_under_rollers():
    """On a heterogeneous image the roller normal block from three single-axis
    tests and the combined test (Eqs. D1-D5) is the same linear map: the
    combined test's averages are the sum of the three single tests', so
    D3-D5 return the off-diagonal entries of S E^-1 of the normal tests."""
    K, G = images.random_moduli((7, 6, 8), seed=21)
    Cd, r = roller_direct(K, G)
    Cn = r.S[:3, :3] @ np.linalg.inv(r.E[:3, :3])
    ref = [Cn[0, 0], Cn[1, 1], Cn[2, 2], 0.5 * (Cn[0, 1] + Cn[1, 0]), 0.5 * (Cn[0, 2] + Cn[2, 0]),
           0.5 * (Cn[1, 2] + Cn[2, 1])]
    assert np.abs(Cd - ref).max() <= 1e-9 * np.abs(Cn).max()


# ------------------------------------------------ simple shear, Appendix A.2
SHEAR = {2: 3, 3: 4, 4: 5}      # boundary mode -> its Voigt shear component (yz, xz, xy)


@pytest.mark.parametrize("bc", [2, 3, 4])
def test_simple_shear_tests_two_oracle_routes_agree(bc):
    """The simple shear tests (Appendix A.2, bc 2-4) written twice: the APT
    iteration of the C oracle and the direct solve of the assembled operator
    (oracle/operator.py), each with its own statement of which boundary edges
    are traction-free, agree on the averages to the direct solve's precision."""
    from oracle import operator
    K, G = images.random_moduli((6, 7, 5), seed=40 + bc)
    e = np.eye(6)[SHEAR[bc]]
    r = apt.solve(K, G, loads=e[None], tol=1e-12, bc=bc, max_iter=400000)
    assert r.cases[0].status == 0
    d = operator.solve_all(K, G, loads=e[None], bc=bc)
    scale = np.abs(d["S"]).max()
    assert np.abs(r.S[:, 0] - d["S"][:, 0]).max() <= 1e-9 * scale
    assert np.abs(r.E[:, 0] - d["E"][:, 0]).max() <= 1e-9
    # the test's stiffness is C_kk = <sigma_k> / <gamma_k> of its component
    k = SHEAR[bc]
    assert d["S"][k, 0] / d["E"][k, 0] > 0


def test_simple_shear_tests_follow_the_axes():
    """Exchanging the image's x and y axes exchanges the yz and xz tests
    (bc 2 <-> 3): C44 of one image is C55 of its transpose, exactly."""
    K, G = images.random_moduli((6, 5, 7), seed=9)          # (nz, ny, nx)
    Kt, Gt = np.ascontiguousarray(K.transpose(0, 2, 1)), np.ascontiguousarray(G.transpose(0, 2, 1))
    a = apt.solve(K, G, loads=np.eye(6)[3][None], tol=1e-12, bc=2, max_iter=400000)
    b = apt.solve(Kt, Gt, loads=np.eye(6)[4][None], tol=1e-12, bc=3, max_iter=400000)
    ca = a.S[3, 0] / a.E[3, 0]
    cb = b.S[4, 0] / b.E[4, 0]
    assert abs(ca - cb) <= 1e-10 * abs(ca)


def test_simple_shear_of_a_thin_wide_homogeneous_slab_tends_to_g():
    """The free lateral faces disturb the shear only within a layer of about
    the sheared thickness: for a homogeneous slab 40 x 40 x 4 the xz test
    gives C55 within a few percent of G, and it gets closer as the slab
    widens (a homogeneous cube is not exact under these conditions)."""
    vals = []
    for n in (12, 24, 40):
        K = np.full((4, n, n), 70.0)
        G = np.full((4, n, n), 30.0)
        r = apt.solve(K, G, loads=np.eye(6)[4][None], tol=1e-10, bc=3, max_iter=400000)
        vals.append(r.S[4, 0] / r.E[4, 0])
    errs = [abs(v - 30.0) / 30.0 for v in vals]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.05, vals
