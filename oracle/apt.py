"""ORACLE -- test infrastructure only (tests, the smoke check and the CPU
baseline of the benchmark use it; the product path never does).

FP64 route R1 of the oracle: the accelerated pseudo-transient iteration of the
paper, run by the plain C code in ``apt_oracle.c`` (loaded with ctypes), plus
the host-side pieces written out in the paper's notation:

* numerical parameters, Eqs. PT1_1t2 - PT24q (Sec. 3.1):
    dt~ = C~ dx / Vp~,  Vp~ = sqrt(H~/rho~),  St = Lx / (Vp~ dt),
    dt~/rho~ = C~ dx Lx / (St H~ dt),  H~ dt~ = (Vp~ dt~)^2 (dt~/rho~)^-1,
    G~ dt~ = H~ dt~ / (K_G + 4/3),  K~ dt~ = K_G G~ dt~,  St_opt times sqrt 3;
  with K~ = K and G~ = G (Sec. 3.1) taken locally, the pseudo step
  dt~ = C~ dx St dt / Lx is uniform, K~ dt~ and G~ dt~ follow each stress
  point's own modulus, and dt~/rho~ follows H~ at each velocity node (the C
  code forms H~ there); this module supplies dt~ and C~ dx Lx / (St dt);
* the effective stiffness from volume averages, Eqs. BC:1 - BC:3 and eq:4:
    <sigma>^m = C <eps>^m for the load cases m, i.e. C = S E^-1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apt_oracle.c")
_LIB = os.path.join(_HERE, "libapt_oracle.so")

# readings of the paper (listed with their reasons in the design notes)
ST_3D = 2.0 * np.pi * np.sqrt(3.0)       # St_opt times sqrt(3) in 3-D (Sec. 3.1, Eq. PT24q)
ST_POROUS = 0.35 * ST_3D                 # faster tail for near-void pores (numerical choice)
CFL_3D = 0.95 / np.sqrt(3.0)             # C~ below the 3-D staggered-grid limit 1/sqrt(3)
FIELDS = ("p", "tau_xx", "tau_yy", "tau_xy", "tau_xz", "tau_yz", "w_x", "w_y", "w_z")
STATUS = {0: "converged", 4: "not converged", 5: "diverged"}


def build(force: bool = False) -> str:
    """Compile the C oracle (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i, d = ctypes.c_int, ctypes.c_double
        L.oracle_solve.argtypes = [i, i, i, i, d, d, d, dp, dp, dp, d, i, i, i, dp, dp, i, ip,
                                   ip, dp, dp]
        L.oracle_solve.restype = i
        L.oracle_init.argtypes = [i, i, i, i, dp, dp, dp, dp]
        L.oracle_sweeps.argtypes = [i, i, i, i, d, d, d, dp, dp, dp, dp, i]
        L.oracle_node_moduli.argtypes = [i, i, i, dp, dp, dp]
        L.oracle_residual2.argtypes = [i, i, i, i, dp, dp, dp, dp]
        L.oracle_residual2.restype = d
        L.oracle_elastic_stress.argtypes = [i, i, i, i, dp, dp, dp, dp, dp]
        L.oracle_average.argtypes = [i, i, i, dp, dp, dp, dp]
        L.oracle_num_threads.restype = i
        L.oracle_stress_planes.argtypes = [i, i, i, i, d, d, dp, dp, dp, dp, i, i]
        L.oracle_velocity_planes.argtypes = [i, i, i, d, dp, dp, i, i]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ------------------------------------------------------------------ scalars
@dataclass
class Params:
    dtt: float      # pseudo-time step dt~
    cdr: float      # C~ dx Lx / (St dt); dt~/rho~ = cdr / H~ at a velocity node
    dt: float = 1.0
    St: float = ST_3D
    Ct: float = CFL_3D
    L: float = 0.0


def numerical_parameters(shape, Ct=CFL_3D, St=ST_3D, dx=1.0, dt=1.0):
    """The paper's numerical parameters (Sec. 3.1) with Lx = max extent."""
    nx, ny, nz = shape
    Lx = max(nx, ny, nz) * dx
    Vp = Lx / (St * dt)                 # St = Lx / (Vp~ dt)
    dtt = Ct * dx / Vp                  # dt~ = C~ dx / Vp~
    cdr = Ct * dx * Lx / (St * dt)      # dt~/rho~ times H~ (Eq. PT1_1t31222)
    return Params(dtt=dtt, cdr=cdr, dt=dt, St=St, Ct=Ct, L=Lx)


# -------------------------------------------------------------------- state
def _grid(K):
    nz, ny, nx = K.shape
    return nx, ny, nz


def state_shape(nx, ny, nz):
    return (len(FIELDS), nz + 1, ny + 1, nx + 1)


def init_state(K, G, e6, bc=0):
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nx, ny, nz = _grid(K)
    st = np.zeros(state_shape(nx, ny, nz))
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    lib().oracle_init(nx, ny, nz, bc, _p(K), _p(G), _p(e6), _p(st))
    return st


def sweeps(K, G, e6, state, n, par: Params, bc=0):
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nx, ny, nz = _grid(K)
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    assert state.flags.c_contiguous and state.shape == state_shape(nx, ny, nz)
    lib().oracle_sweeps(nx, ny, nz, bc, par.dtt, par.cdr, par.dt, _p(K), _p(G), _p(e6),
                        _p(state), int(n))
    return state


def residual_norm(K, G, e6, state, bc=0):
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nx, ny, nz = _grid(K)
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    st = np.ascontiguousarray(state, dtype=np.float64)
    return float(np.sqrt(lib().oracle_residual2(nx, ny, nz, bc, _p(K), _p(G), _p(e6), _p(st))))


def elastic_stress(K, G, e6, state, bc=0):
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nx, ny, nz = _grid(K)
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    st = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros((6, nz + 1, ny + 1, nx + 1))
    lib().oracle_elastic_stress(nx, ny, nz, bc, _p(K), _p(G), _p(e6), _p(st), _p(out))
    return out


def node_moduli(K, G):
    """H~ at every interior velocity node (3 index-grid arrays)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nx, ny, nz = _grid(K)
    out = np.zeros((3, nz + 1, ny + 1, nx + 1))
    lib().oracle_node_moduli(nx, ny, nz, _p(K), _p(G), _p(out))
    return out


def average(e6, state):
    nx, ny, nz = state.shape[3] - 1, state.shape[2] - 1, state.shape[1] - 1
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    st = np.ascontiguousarray(state, dtype=np.float64)
    sig = np.zeros(6)
    eps = np.zeros(6)
    lib().oracle_average(nx, ny, nz, _p(e6), _p(st), _p(sig), _p(eps))
    return sig, eps


# -------------------------------------------------------------------- solve
@dataclass
class CaseResult:
    status: int
    iters: int
    rel: float
    r0: float
    hist: np.ndarray
    sig: np.ndarray
    eps: np.ndarray
    state: np.ndarray | None = None


@dataclass
class Result:
    C: np.ndarray
    S: np.ndarray           # columns <sigma>^m
    E: np.ndarray           # columns <eps>^m
    cases: list = field(default_factory=list)
    par: Params | None = None


def solve_case(K, G, e6, par: Params, tol=1e-8, max_iter=100000, n_check=16, bc=0,
               state=None, keep_state=False):
    K = np.ascontiguousarray(K, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    nx, ny, nz = _grid(K)
    e6 = np.ascontiguousarray(e6, dtype=np.float64)
    init = 0
    if state is None:
        state = np.zeros(state_shape(nx, ny, nz))
        init = 1
    cap = max_iter // max(n_check, 1) + 4
    hist = np.zeros(cap)
    nh, it = ctypes.c_int(0), ctypes.c_int(0)
    rel, r0 = ctypes.c_double(0), ctypes.c_double(0)
    st = lib().oracle_solve(nx, ny, nz, bc, par.dtt, par.cdr, par.dt, _p(K), _p(G),
                            _p(e6), float(tol), int(max_iter), int(n_check), init, _p(state),
                            _p(hist), cap, ctypes.byref(nh), ctypes.byref(it), ctypes.byref(rel),
                            ctypes.byref(r0))
    sig, eps = average(e6, state)
    return CaseResult(status=st, iters=it.value, rel=rel.value, r0=r0.value,
                      hist=hist[:nh.value].copy(), sig=sig, eps=eps,
                      state=state if keep_state else None)


def stiffness_from_averages(S, E):
    """C with <sigma>^m = C <eps>^m for every column m (Eq. BC:3)."""
    return S @ np.linalg.inv(E)


def solve(K, G, loads=None, tol=1e-8, max_iter=100000, n_check=16, bc=0, Ct=CFL_3D, St=ST_3D,
          keep_state=False):
    """Six (or the given) load cases, one at a time, then C = S E^-1."""
    loads = np.eye(6) if loads is None else np.asarray(loads, dtype=np.float64)
    par = numerical_parameters(_grid(np.asarray(K)), Ct=Ct, St=St)
    cases = [solve_case(K, G, loads[m], par, tol, max_iter, n_check, bc, keep_state=keep_state)
             for m in range(loads.shape[0])]
    S = np.stack([c.sig for c in cases], axis=1)
    E = np.stack([c.eps for c in cases], axis=1)
    C = stiffness_from_averages(S, E) if loads.shape[0] == 6 else None
    return Result(C=C, S=S, E=E, cases=cases, par=par)
