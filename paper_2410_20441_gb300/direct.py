"""The paper's full set of direct tests for an orthorhombic medium (Sec. 3.4,
Appendix A), each a solve on the GPU through the C-ABI:

* three normal tests and the combined three-face test under rollers
  (Appendix A.1, A.3): C11, C22, C33 by Eq. eq:4 and C12, C13, C23 by
  Eqs. D1-D5 (ce_direct_tests);
* three simple shear tests (Appendix A.2): C44, C55, C66 = <sigma_k> /
  <gamma_k> of the unit shear k.  The appendix's text is garbled; read
  literally (the sheared component prescribed on its driven face pair, the
  lateral faces traction-free: CE_BC_SHEAR_YZ, _XZ, _XY, shear="literal")
  the tests give the layered medium of Model 1 C44 = 8.8 and C66 = 15.8 GPa,
  far below Table 2's numerical column (15.307, 25.376), while the same
  shears under uniform kinematic conditions (shear="kubc", the default) give
  15.6 and <G> = 25.386, as the paper's numbers do.

That is the paper's seven solves; `ceff` (six cases under uniform kinematic
conditions, C = S E^-1) is the library's default route to the whole C.
"""
from __future__ import annotations

import numpy as np

from . import ce

SHEAR_TESTS = (("shear_yz", 3), ("shear_xz", 4), ("shear_xy", 5))


def paper_direct_tests(K, G, tol=1e-6, max_iter=1_000_000, shear="kubc", **ctx_kw):
    """The nine orthorhombic constants of the paper's direct tests, as a dict
    C11 ... C66 (GPa); shear: "kubc" or "literal" (see the module text)."""
    out = {}
    with ce.Context(K, G, bc="roller", **ctx_kw) as c:
        c.solve(ce.DIRECT_LOADS, tol=tol, max_iter=max_iter)
        for name, v in zip(("C11", "C22", "C33", "C12", "C13", "C23"), c.direct_tests()):
            out[name] = float(v)
    for bc, k in SHEAR_TESTS:
        with ce.Context(K, G, bc=bc if shear == "literal" else "kubc", **ctx_kw) as c:
            c.solve(np.eye(6)[k][None], tol=tol, max_iter=max_iter)
            sig, eps = c.averages()
            out[f"C{k + 1}{k + 1}"] = float(sig[0, k] / eps[0, k])
    return out
