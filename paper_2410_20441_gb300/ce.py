"""ctypes binding of libce (include/ce.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module
passes pointers, sizes and the current torch stream, and lets the torch
caching allocator serve the library's device memory.  If the compiled
library is missing it is built (nvcc); if that fails, an error is raised --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CE_MAX_CASES = 6
STATUS = ["ok", "invalid argument", "out of device memory", "CUDA error", "not converged", "diverged",
          "call out of order", "not implemented"]
CE_OK, CE_EINVAL, CE_ENOMEM, CE_ECUDA, CE_ENOTCONV, CE_EDIVERGED, CE_ESTATE, CE_ENOTIMPL = range(8)
PREC = {"fp32": 0, "fp64": 1}
BC = {"kubc": 0, "roller": 1, "shear_yz": 2, "shear_xz": 3, "shear_xy": 4}
KERNEL = {"auto": 0, "plain": 1, "fused": 2, "fused_lsu": 3}
FIELDS = ("p", "tau_xx", "tau_yy", "tau_xy", "tau_xz", "tau_yz", "w_x", "w_y", "w_z", "u_x", "u_y", "u_z")
WARM_START = 1
NO_REFINE = 2
REFINE_EACH_CHECK = 4
EXPORTS = ("ce_default_opts", "ce_create", "ce_solve", "ce_ceff", "ce_averages", "ce_grad", "ce_get_field",
           "ce_destroy", "ce_status_str", "ce_last_error", "ce_create_batch", "ce_solve_batch", "ce_ceff_batch",
           "ce_residual_noalloc", "ce_autotune", "ce_set_tile", "ce_set_moduli", "ce_slab_cells",
           "ce_create_slab", "ce_slab_start", "ce_slab_sweep", "ce_slab_residual", "ce_slab_halo_bytes",
           "ce_slab_pack", "ce_slab_unpack", "ce_slab_sums", "ce_direct_tests", "ce_ceff_from_sums",
           "ce_slab_sweep_part", "ce_autotune_for", "ce_sweep_chunk")
# what a tuned launch shape serves (ce_autotune_for)
TUNE = {"auto": 0, "plain": 1, "refined": 2}
# the four loads of the paper's direct tests (Appendix A.1, A.3): e1, e2, e3, e1 + e2 + e3
DIRECT_LOADS = np.array([[1, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0], [0, 0, 1, 0, 0, 0], [1, 1, 1, 0, 0, 0]],
                        dtype=np.float64)


class CeError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("bc", ctypes.c_int), ("kernel", ctypes.c_int), ("St", ctypes.c_double),
                ("Ct", ctypes.c_double), ("n_check", ctypes.c_int), ("tile", ctypes.c_int * 4),
                ("St_first", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("n_cases", ctypes.c_int), ("iters", ctypes.c_int * CE_MAX_CASES),
                ("rel_res", ctypes.c_double * CE_MAX_CASES), ("res0", ctypes.c_double * CE_MAX_CASES),
                ("status", ctypes.c_int * CE_MAX_CASES), ("sweeps", ctypes.c_int), ("checks", ctypes.c_int),
                ("case_sweeps", ctypes.c_longlong), ("launches", ctypes.c_int), ("sweep_ms", ctypes.c_double),
                ("check_ms", ctypes.c_double), ("seconds", ctypes.c_double), ("teff_gbs", ctypes.c_double),
                ("rebases", ctypes.c_int), ("sweeps_corr", ctypes.c_int), ("case_sweeps_corr", ctypes.c_longlong),
                ("sweep_ms_corr", ctypes.c_double)]

    def as_dict(self):
        n = self.n_cases
        return {"n_cases": n, "iters": list(self.iters)[:n], "rel_res": list(self.rel_res)[:n],
                "res0": list(self.res0)[:n], "status": list(self.status)[:n], "sweeps": self.sweeps,
                "checks": self.checks, "case_sweeps": self.case_sweeps, "launches": self.launches,
                "sweep_ms": self.sweep_ms, "check_ms": self.check_ms, "seconds": self.seconds,
                "teff_gbs": self.teff_gbs, "rebases": self.rebases, "sweeps_corr": self.sweeps_corr,
                "case_sweeps_corr": self.case_sweeps_corr, "sweep_ms_corr": self.sweep_ms_corr}


_lib = None


def load(path: str | None = None):
    """Load libce.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    if not os.path.exists(path):
        raise CeError(CE_ECUDA, f"libce not found at {path}")
    L = ctypes.CDLL(path)
    vp, ip, dp, fp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    L.ce_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.ce_default_opts.restype = None
    L.ce_create.argtypes = [ctypes.POINTER(Grid), fp, fp, ip, ctypes.POINTER(Opts), ctypes.POINTER(Allocator), vp,
                            ctypes.POINTER(vp)]
    L.ce_solve.argtypes = [vp, dp, ip, ctypes.c_double, ip, ctypes.c_uint, ctypes.POINTER(SolveInfo)]
    L.ce_ceff.argtypes = [vp, dp]
    L.ce_averages.argtypes = [vp, dp, dp]
    L.ce_direct_tests.argtypes = [vp, dp]
    L.ce_ceff_from_sums.argtypes = [dp, ip, ctypes.POINTER(Grid), dp]
    L.ce_grad.argtypes = [vp, dp, fp, fp, ip]
    L.ce_get_field.argtypes = [vp, ip, ip, dp]
    L.ce_destroy.argtypes = [vp]
    L.ce_destroy.restype = None
    L.ce_status_str.argtypes = [ip]
    L.ce_status_str.restype = ctypes.c_char_p
    L.ce_last_error.argtypes = [vp]
    L.ce_last_error.restype = ctypes.c_char_p
    L.ce_create_batch.argtypes = [ip, ctypes.POINTER(Grid), ctypes.POINTER(vp), ctypes.POINTER(vp), ip,
                                  ctypes.POINTER(Opts), ctypes.POINTER(Allocator), vp, ctypes.POINTER(vp)]
    L.ce_solve_batch.argtypes = [vp, ctypes.c_double, ip, ctypes.POINTER(ctypes.c_int)]
    L.ce_ceff_batch.argtypes = [vp, dp]
    L.ce_residual_noalloc.argtypes = [ctypes.POINTER(Grid), fp, fp, fp, dp, ip, fp, vp]
    L.ce_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), dp]
    L.ce_autotune_for.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_int), dp]
    L.ce_sweep_chunk.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_int), ip, ip, ctypes.POINTER(ctypes.c_int)]
    L.ce_set_tile.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.ce_set_moduli.argtypes = [vp, fp, fp, ip]
    ipp = ctypes.POINTER(ctypes.c_int)
    L.ce_slab_cells.argtypes = [ctypes.POINTER(Grid), ip, ip, ipp, ipp]
    L.ce_create_slab.argtypes = [ctypes.POINTER(Grid), ip, ip, fp, fp, ip, ctypes.POINTER(Opts),
                                 ctypes.POINTER(Allocator), vp, ctypes.POINTER(vp)]
    L.ce_slab_start.argtypes = [vp, dp, ip, dp]
    L.ce_slab_sweep.argtypes = [vp, ipp, ip, ip, ip]
    L.ce_slab_residual.argtypes = [vp, dp]
    L.ce_slab_sweep_part.argtypes = [vp, ipp, ip, ip]
    L.ce_slab_halo_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.ce_slab_pack.argtypes = [vp, ip, vp]
    L.ce_slab_unpack.argtypes = [vp, ip, vp]
    L.ce_slab_sums.argtypes = [vp, dp]
    for name in ("ce_create", "ce_solve", "ce_ceff", "ce_averages", "ce_direct_tests", "ce_ceff_from_sums", "ce_grad", "ce_get_field", "ce_create_batch",
                 "ce_solve_batch", "ce_ceff_batch", "ce_residual_noalloc", "ce_autotune", "ce_set_tile",
                 "ce_set_moduli", "ce_slab_cells", "ce_create_slab", "ce_slab_start", "ce_slab_sweep",
                 "ce_slab_residual", "ce_slab_halo_bytes", "ce_slab_pack", "ce_slab_unpack", "ce_slab_sums",
                 "ce_slab_sweep_part", "ce_autotune_for", "ce_sweep_chunk"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_opts(prec="fp32", bc="kubc", kernel="auto", St=None, Ct=None, n_check=0, tile=(0, 0, 0, 0),
              St_first=None):
    L = load()
    o = Opts()
    L.ce_default_opts(ctypes.byref(o))
    o.prec = PREC[prec]
    o.bc = BC[bc]
    o.kernel = KERNEL[kernel]
    if St is not None:
        o.St = float(St)
    if Ct is not None:
        o.Ct = float(Ct)
    o.n_check = int(n_check)
    if St_first is not None:
        o.St_first = float(St_first)
    tile = tuple(tile) + (0,) * (4 - len(tile))
    for q in range(4):
        o.tile[q] = int(tile[q])
    return o


class _TorchAllocator:
    """Serves libce allocations from the torch caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Context:
    """One image on one GPU: ce_create ... ce_destroy."""

    def __init__(self, K, G, prec="fp32", bc="kubc", kernel="auto", St=None, Ct=None, n_check=0,
                 tile=(0, 0, 0), stream=None, allocator="torch", St_first=None):
        L = load()
        self._L = L
        self._keep = []
        if _is_torch(K) and not K.is_cuda:
            # host tensors (e.g. pinned): pass their host pointers
            import torch
            K = K.detach().to(torch.float32).contiguous()
            G = G.detach().to(torch.float32).contiguous()
            self._keep += [K, G]
            nz, ny, nx = K.shape
            kp, gp, on_dev = K.data_ptr(), G.data_ptr(), 0
            device = None
        elif _is_torch(K):
            import torch
            if not (K.is_cuda and G.is_cuda):
                raise CeError(CE_EINVAL, "torch moduli must both be CUDA or both host tensors")
            K = K.detach().to(torch.float32).contiguous()
            G = G.detach().to(torch.float32).contiguous()
            self._keep += [K, G]
            nz, ny, nx = K.shape
            kp, gp, on_dev = K.data_ptr(), G.data_ptr(), 1
            device = K.device.index
        else:
            K = np.ascontiguousarray(K, dtype=np.float32)
            G = np.ascontiguousarray(G, dtype=np.float32)
            self._keep += [K, G]
            nz, ny, nx = K.shape
            kp, gp, on_dev = K.ctypes.data, G.ctypes.data, 0
            device = None
        if G.shape != K.shape:
            raise CeError(CE_EINVAL, "K and G shapes differ")
        self.shape = (nx, ny, nz)
        self.prec = prec
        alloc_ptr = None
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
                    device = torch.cuda.current_device() if device is None else device
            except ImportError:
                stream = 0
        self.stream = stream or 0
        if allocator == "torch":
            try:
                import torch
                if torch.cuda.is_available():
                    self._alloc = _TorchAllocator(device if device is not None else torch.cuda.current_device())
                    alloc_ptr = ctypes.byref(self._alloc.struct)
            except ImportError:
                pass
        self.bc = bc
        auto = isinstance(tile, str)
        if auto and tile != "auto":
            raise CeError(CE_EINVAL, "tile must be ints (stages, rows, planes, columns) or 'auto'")
        self.opts = make_opts(prec, bc, kernel, St, Ct, n_check, (0, 0, 0) if auto else tile, St_first)
        g = Grid(nx, ny, nz)
        h = ctypes.c_void_p()
        st = L.ce_create(ctypes.byref(g), kp, gp, on_dev, ctypes.byref(self.opts), alloc_ptr,
                         ctypes.c_void_p(self.stream), ctypes.byref(h))
        if st != CE_OK:
            raise CeError(st, "ce_create failed")
        self._h = h
        self.info = None
        self.tile = tuple(self.opts.tile)
        if auto and prec == "fp32" and kernel in ("auto", "fused"):
            from . import autotune
            autotune.tune_context(self)

    # ------------------------------------------------------------------
    def autotune(self, sweeps=6, solves="auto"):
        """Search the TMA sweep's launch shape on this image (ce_autotune_for)
        for the solves it will serve: "auto" (refined solves when the context
        runs them), "plain" (unrefined solves, batches, slabs) or "refined";
        returns (tile, ms per sweep)."""
        if solves not in TUNE:
            raise CeError(CE_EINVAL, "solves must be 'auto', 'plain' or 'refined'")
        t = (ctypes.c_int * 4)()
        ms = ctypes.c_double()
        st = self._L.ce_autotune_for(self._h, int(sweeps), TUNE[solves], t, ctypes.byref(ms))
        if st != CE_OK:
            raise CeError(st, self._err())
        self.tile = tuple(t)
        return self.tile, ms.value

    def set_moduli(self, K, G):
        """Replace the moduli (same shape); the fields stay for a warm start."""
        if _is_torch(K):
            import torch
            K = K.detach().to(torch.float32).contiguous()
            G = G.detach().to(torch.float32).contiguous()
            self._keep_mod = (K, G)
            st = self._L.ce_set_moduli(self._h, K.data_ptr(), G.data_ptr(), 1 if K.is_cuda else 0)
        else:
            K = np.ascontiguousarray(K, dtype=np.float32)
            G = np.ascontiguousarray(G, dtype=np.float32)
            if K.shape != tuple(reversed(self.shape)) or G.shape != K.shape:
                raise CeError(CE_EINVAL, "moduli shape differs from the context's grid")
            st = self._L.ce_set_moduli(self._h, K.ctypes.data, G.ctypes.data, 0)
        if st != CE_OK:
            raise CeError(st, self._err())

    def set_tile(self, tile):
        tile = tuple(int(v) for v in tile) + (0,) * (4 - len(tile))
        t = (ctypes.c_int * 4)(*tile)
        st = self._L.ce_set_tile(self._h, t)
        if st != CE_OK:
            raise CeError(st, self._err())
        self.tile = tuple(t)
    def _err(self):
        return self._L.ce_last_error(self._h).decode()

    def solve(self, loads=None, tol=1e-6, max_iter=1_000_000, warm=False, check=True, refine="auto"):
        """Solve the load cases (rows of `loads`, Voigt, engineering shear;
        None = the six unit cases).  refine: "auto" (defect correction where
        the context supports it), "off" (CE_NO_REFINE) or "each" (rebase at
        every check, CE_REFINE_EACH_CHECK).  Returns the status; raises
        CeError on argument or CUDA errors (and on non-convergence when
        check=True)."""
        if loads is None:
            n, lp = 6, None
        else:
            loads = np.ascontiguousarray(np.atleast_2d(loads), dtype=np.float64)
            n, lp = loads.shape[0], _dp(loads)
        info = SolveInfo()
        flags = (WARM_START if warm else 0) | {"auto": 0, "off": NO_REFINE, "each": REFINE_EACH_CHECK}[refine]
        st = self._L.ce_solve(self._h, lp, n, float(tol), int(max_iter), flags, ctypes.byref(info))
        self.info = info.as_dict()
        if st in (CE_EINVAL, CE_ENOMEM, CE_ECUDA, CE_ESTATE, CE_ENOTIMPL) or (check and st != CE_OK):
            raise CeError(st, self._err())
        return st

    def ceff(self):
        C = np.zeros(36)
        st = self._L.ce_ceff(self._h, _dp(C))
        if st != CE_OK:
            raise CeError(st, self._err())
        return C.reshape(6, 6)

    def direct_tests(self):
        """(C11, C22, C33, C12, C13, C23) of the paper's direct tests from the
        last solve of DIRECT_LOADS (ce_direct_tests; Appendix A, Eqs. D1-D5)."""
        out = np.zeros(6)
        st = self._L.ce_direct_tests(self._h, _dp(out))
        if st != CE_OK:
            raise CeError(st, self._err())
        return out

    def averages(self):
        n = self.info["n_cases"] if self.info else 6
        s = np.zeros(6 * n)
        e = np.zeros(6 * n)
        st = self._L.ce_averages(self._h, _dp(s), _dp(e))
        if st != CE_OK:
            raise CeError(st, self._err())
        return s.reshape(n, 6), e.reshape(n, 6)

    def grad(self, w, dK=None, dG=None):
        """dJ/dK, dJ/dG of J = sum w_mn C_mn.  With torch CUDA tensors dK, dG
        the result is written on the device; otherwise numpy arrays return."""
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(36)
        nx, ny, nz = self.shape
        if dK is not None:
            st = self._L.ce_grad(self._h, _dp(w), dK.data_ptr(), dG.data_ptr(), 1)
            if st != CE_OK:
                raise CeError(st, self._err())
            return dK, dG
        hk = np.zeros((nz, ny, nx), np.float32)
        hg = np.zeros((nz, ny, nx), np.float32)
        st = self._L.ce_grad(self._h, _dp(w), hk.ctypes.data, hg.ctypes.data, 0)
        if st != CE_OK:
            raise CeError(st, self._err())
        return hk, hg

    def field(self, case, name):
        f = FIELDS.index(name) if isinstance(name, str) else int(name)
        nx, ny, nz = self.shape
        out = np.zeros((nz + 1, ny + 1, nx + 1))
        st = self._L.ce_get_field(self._h, int(case), f, _dp(out))
        if st != CE_OK:
            raise CeError(st, self._err())
        return out

    def state(self, case):
        """The nine paper fields (p, tau, w) of one case."""
        return np.stack([self.field(case, f) for f in range(9)])

    def close(self):
        if getattr(self, "_h", None):
            self._L.ce_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchContext:
    """Many images of uneven size solved together (ce_create_batch): one CUDA
    graph whose WHILE loop runs the batched sweep over every active sample."""

    def __init__(self, images, St=None, Ct=None, n_check=0, tile=(0, 0, 0), stream=None, allocator="torch"):
        L = load()
        self._L = L
        self._keep = []
        n = len(images)
        grids = (Grid * n)()
        Kp = (ctypes.c_void_p * n)()
        Gp = (ctypes.c_void_p * n)()
        self.shapes = []
        for s, (K, G) in enumerate(images):
            K = np.ascontiguousarray(K, dtype=np.float32)
            G = np.ascontiguousarray(G, dtype=np.float32)
            self._keep += [K, G]
            nz, ny, nx = K.shape
            grids[s] = Grid(nx, ny, nz)
            Kp[s] = K.ctypes.data
            Gp[s] = G.ctypes.data
            self.shapes.append((nx, ny, nz))
        alloc_ptr = None
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        if allocator == "torch":
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            alloc_ptr = ctypes.byref(self._alloc.struct)
        if isinstance(tile, str):
            if tile != "auto":
                raise CeError(CE_EINVAL, "tile must be ints (stages, rows, planes, columns) or 'auto'")
            # one launch shape for the whole batch, tuned on its largest sample
            # for the double-word sweep the batch runs
            from . import autotune
            big = max(range(n), key=lambda s: self.shapes[s][0] * self.shapes[s][1] * self.shapes[s][2])
            with Context(images[big][0], images[big][1], prec="fp32", kernel="fused", St=St, Ct=Ct,
                         n_check=n_check) as probe:
                tile, _ = autotune.tune_context(probe, solves="plain")
        self.tile = tuple(int(v) for v in tile) + (0,) * (4 - len(tuple(tile)))
        self.opts = make_opts("fp32", "kubc", "fused", St, Ct, n_check, self.tile)
        h = ctypes.c_void_p()
        st = L.ce_create_batch(n, grids, Kp, Gp, 0, ctypes.byref(self.opts), alloc_ptr, ctypes.c_void_p(stream),
                               ctypes.byref(h))
        if st != CE_OK:
            raise CeError(st, "ce_create_batch failed: " + L.ce_last_error(None).decode())
        self._h = h
        self.n = n
        self.iters = None

    def solve(self, tol=1e-5, max_iter=100_000, check=True):
        it = (ctypes.c_int * self.n)()
        st = self._L.ce_solve_batch(self._h, float(tol), int(max_iter), it)
        self.iters = list(it)
        if st in (CE_EINVAL, CE_ENOMEM, CE_ECUDA, CE_ESTATE, CE_ENOTIMPL) or (check and st != CE_OK):
            raise CeError(st, self._L.ce_last_error(self._h).decode())
        return st

    def ceff(self):
        C = np.zeros(36 * self.n)
        st = self._L.ce_ceff_batch(self._h, _dp(C))
        if st != CE_OK:
            raise CeError(st, self._L.ce_last_error(self._h).decode())
        return C.reshape(self.n, 6, 6)

    def close(self):
        if getattr(self, "_h", None):
            self._L.ce_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def ceff_from_sums(sums, shape):
    """C = S E^-1 (ce_ceff_from_sums) from the per-case sums (6 x 12: sigma
    then engineering strain, Voigt) added over the parts of a grid of shape
    (nx, ny, nz); averages pass as sums over shape (1, 1, 1)."""
    L = load()
    s = np.ascontiguousarray(sums, dtype=np.float64).reshape(6, 12)
    C = np.zeros(36)
    st = L.ce_ceff_from_sums(_dp(s), 6, ctypes.byref(Grid(*[int(v) for v in shape])), _dp(C))
    if st != CE_OK:
        raise CeError(st, L.ce_last_error(None).decode())
    return C.reshape(6, 6)


def sweep_chunk(shape, tile, n_cases, n_sm):
    """z-planes per block of the FP32 TMA sweep over n_cases of the six load
    cases on a device with n_sm SMs (ce_sweep_chunk; host only)."""
    L = load()
    nz, ny, nx = shape
    g = Grid(nx, ny, nz)
    t = (ctypes.c_int * 4)(*(tuple(int(v) for v in tile) + (0,) * (4 - len(tile))))
    out = ctypes.c_int()
    st = L.ce_sweep_chunk(ctypes.byref(g), t, int(n_cases), int(n_sm), ctypes.byref(out))
    if st != CE_OK:
        raise CeError(st, L.ce_last_error(None).decode())
    return out.value


def slab_cells(shape, z0, z1):
    """Cell layers [c0, c1) along z that the slab owning the index planes
    [z0, z1) of a grid of shape (nx, ny, nz) reads (ce_slab_cells)."""
    L = load()
    c0, c1 = ctypes.c_int(), ctypes.c_int()
    g = Grid(*shape)
    st = L.ce_slab_cells(ctypes.byref(g), int(z0), int(z1), ctypes.byref(c0), ctypes.byref(c1))
    if st != CE_OK:
        raise CeError(st, f"no slab window for planes [{z0}, {z1}) of nz = {shape[2]}")
    return c0.value, c1.value


class Slab:
    """One z-slab of a grid (ce_create_slab ... ce_destroy): it owns the index
    planes [z0, z1) and holds one ghost plane on each side with a neighbour.
    K, G are the whole grid's moduli, shape (nz, ny, nx), numpy or torch (host
    or CUDA); only the slab's cell layers are passed to the library."""

    def __init__(self, K, G, z0, z1, bc="kubc", St=None, Ct=None, n_check=0, tile=(0, 0, 0, 0), stream=None,
                 allocator="torch"):
        L = load()
        self._L = L
        nz, ny, nx = K.shape
        self.shape = (nx, ny, nz)
        self.z0, self.z1 = int(z0), int(z1)
        self.c0, self.c1 = slab_cells(self.shape, z0, z1)
        Ks, Gs = K[self.c0:self.c1], G[self.c0:self.c1]
        if _is_torch(Ks):
            import torch
            Ks = Ks.detach().to(torch.float32).contiguous()
            Gs = Gs.detach().to(torch.float32).contiguous()
            kp, gp, on_dev = Ks.data_ptr(), Gs.data_ptr(), int(Ks.is_cuda)
        else:
            Ks = np.ascontiguousarray(Ks, dtype=np.float32)
            Gs = np.ascontiguousarray(Gs, dtype=np.float32)
            kp, gp, on_dev = Ks.ctypes.data, Gs.ctypes.data, 0
        self._keep = [Ks, Gs]
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        alloc_ptr = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            alloc_ptr = ctypes.byref(self._alloc.struct)
        self.opts = make_opts("fp32", bc, "fused", St, Ct, n_check, tile)
        h = ctypes.c_void_p()
        st = L.ce_create_slab(ctypes.byref(Grid(nx, ny, nz)), self.z0, self.z1, kp, gp, on_dev,
                              ctypes.byref(self.opts), alloc_ptr, ctypes.c_void_p(self.stream), ctypes.byref(h))
        if st != CE_OK:
            raise CeError(st, "ce_create_slab failed")
        self._h = h
        self.n_cases = 0
        self.lower = self.z0 > 0              # a neighbour below
        self.upper = self.z1 < nz + 1         # a neighbour above

    def _err(self):
        return self._L.ce_last_error(self._h).decode()

    def _ok(self, st):
        if st != CE_OK:
            raise CeError(st, self._err())

    def start(self, loads=None):
        """Initial state; returns this slab's share of ||div sigma(0)||^2 per case."""
        if loads is None:
            n, lp = 6, None
        else:
            loads = np.ascontiguousarray(np.atleast_2d(loads), dtype=np.float64)
            n, lp = loads.shape[0], _dp(loads)
        b2 = np.zeros(n)
        self._ok(self._L.ce_slab_start(self._h, lp, n, _dp(b2)))
        self.n_cases = n
        return b2

    def sweep(self, cases=None, n_sweeps=1, check=False):
        if cases is None:
            cp, n = None, 0
        else:
            arr = (ctypes.c_int * len(cases))(*[int(m) for m in cases])
            cp, n = arr, len(cases)
        self._ok(self._L.ce_slab_sweep(self._h, cp, n, int(n_sweeps), int(bool(check))))

    def sweep_part(self, cases=None, part=1):
        """Half of one sweep (ce_slab_sweep_part): part 1 the boundary planes,
        part 2 the interior; pack between them to overlap the exchange."""
        if cases is None:
            cp, n = None, 0
        else:
            arr = (ctypes.c_int * len(cases))(*[int(m) for m in cases])
            cp, n = arr, len(cases)
        self._ok(self._L.ce_slab_sweep_part(self._h, cp, n, int(part)))

    def residual(self, n):
        r2 = np.zeros(n)
        self._ok(self._L.ce_slab_residual(self._h, _dp(r2)))
        return r2

    def halo_bytes(self):
        b = ctypes.c_size_t()
        self._ok(self._L.ce_slab_halo_bytes(self._h, ctypes.byref(b)))
        return b.value

    def pack(self, side, msg):
        """msg: a CUDA tensor or a device address, ce_slab_halo_bytes long."""
        ptr = msg.data_ptr() if hasattr(msg, "data_ptr") else int(msg)
        self._ok(self._L.ce_slab_pack(self._h, int(side), ctypes.c_void_p(ptr)))

    def unpack(self, side, msg):
        ptr = msg.data_ptr() if hasattr(msg, "data_ptr") else int(msg)
        self._ok(self._L.ce_slab_unpack(self._h, int(side), ctypes.c_void_p(ptr)))

    def sums(self):
        s = np.zeros(12 * self.n_cases)
        self._ok(self._L.ce_slab_sums(self._h, _dp(s)))
        return s.reshape(self.n_cases, 12)

    def field(self, case, name):
        """A field on the slab's local index planes (global plane = local + c0)."""
        f = FIELDS.index(name) if isinstance(name, str) else int(name)
        nx, ny, _ = self.shape
        out = np.zeros((self.c1 - self.c0 + 1, ny + 1, nx + 1))
        self._ok(self._L.ce_get_field(self._h, int(case), f, _dp(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._L.ce_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def effective_stiffness(K, G, tol=1e-6, max_iter=1_000_000, **kw):
    """One-call convenience: C_eff (6x6, GPa) of an image."""
    with Context(K, G, **kw) as c:
        c.solve(None, tol=tol, max_iter=max_iter)
        return c.ceff()
