"""The allocation-free residual check (ce_residual_noalloc) against the
residual the solver reports for the same state and against the FP64 oracle's
residual of that state.

The entry point serves callers that cannot allocate device memory (a host
framework that owns all GPU memory, code running under CUDA-graph capture,
real-time loops); its scratch is a static device array shared by all calls.
Two calls in a row must both agree with the solver: the second one sees the
first call's leftovers in that array.  This file is collected last on
purpose, so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

from oracle import apt
from paper_2410_20441_gb300 import images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_20441_gb300 import ce
    return torch, ce, ce.load()


def _call(L, ce, torch, shape, Kt, Gt, wt, e6, out, bc=0):
    g = ce.Grid(*shape)
    e = np.ascontiguousarray(e6, dtype=np.float64)
    return L.ce_residual_noalloc(ctypes.byref(g), Kt.data_ptr(), Gt.data_ptr(), wt.data_ptr(),
                                 e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bc, out.data_ptr(),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("bc", [0, 1])
def test_noalloc_residual_matches_solver_on_two_calls(env, bc):
    torch, ce, L = env
    nx, ny, nz = 21, 17, 19
    K, G = images.two_phase_random((nx, ny, nz), seed=5, frac=0.3, inclusion=(5.0, 2.0))
    e6 = np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.2]) if bc == 0 else np.array([0.3, -0.2, 0.5, 0, 0, 0])
    # the existing path: FP32 plain kernels, residual of the state after 37 sweeps
    with ce.Context(K, G, prec="fp32", kernel="plain", bc=("kubc", "roller")[bc]) as c:
        c.solve(e6[None], tol=0.0, max_iter=37, check=False)
        r0 = c.info["res0"][0]
        rw = c.info["rel_res"][0] * r0
        w = np.stack([c.field(0, f) for f in ("w_x", "w_y", "w_z")])
    # the oracle's residual of the same w (FP64 stresses and sums)
    st = np.zeros(apt.state_shape(nx, ny, nz))
    st[6:9] = w.astype(np.float32)
    ro_w = apt.residual_norm(K, G, e6, st, bc=bc)
    ro_0 = apt.residual_norm(K, G, e6, np.zeros_like(st), bc=bc)
    Kt = torch.tensor(K, device="cuda")
    Gt = torch.tensor(G, device="cuda")
    wt = torch.tensor(w.astype(np.float32), device="cuda")      # exact: the values are FP32
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        rc = _call(L, ce, torch, (nx, ny, nz), Kt, Gt, wt, e6, out, bc)
        assert rc == ce.CE_OK, L.ce_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - rw) <= 1e-5 * rw, (got, rw)
        assert abs(got[1] - r0) <= 1e-5 * r0, (got, r0)
        # FP32 stresses against FP64 ones: single roundings of O(100) terms
        assert abs(got[0] - ro_w) <= 1e-5 * ro_w, (got, ro_w)
        assert abs(got[1] - ro_0) <= 1e-5 * ro_0, (got, ro_0)


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, ce, L = env
    Kt = torch.ones(8, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = _call(L, ce, torch, (32 * 300, 8 * 200, 2), Kt, Kt, Kt, np.zeros(6), out)
    assert st == ce.CE_EINVAL
    assert b"static scratch" in L.ce_last_error(None)
