"""The C-ABI library builds, loads and exports every symbol include/ce.h
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2410_20441_gb300 import build as cebuild
from paper_2410_20441_gb300 import ce

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ce.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ce_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ce_create", "ce_solve", "ce_ceff", "ce_grad", "ce_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    L = ce.load(cebuild.build())
    for s in declared_symbols():
        assert hasattr(L, s), s
    assert set(declared_symbols()) <= set(ce.EXPORTS)


def test_status_strings_and_defaults_without_gpu():
    L = ce.load()
    assert L.ce_status_str(0) == b"ok"
    assert L.ce_status_str(4) == b"not converged"
    o = ce.Opts()
    L.ce_default_opts(ctypes.byref(o))
    assert o.prec == 0 and o.bc == 0 and o.kernel == 0
    assert abs(o.St - 2 * 3.141592653589793 * 3 ** 0.5) < 1e-12
    assert abs(o.Ct - 0.95 / 3 ** 0.5) < 1e-12


def test_create_rejects_bad_grids_before_touching_the_device():
    L = ce.load()
    h = ctypes.c_void_p()
    import numpy as np
    K = np.ones(8, np.float32)
    # too small, and too large for 32-bit index-grid offsets ((n+1)^3 >= 2^31)
    for dims in ((1, 2, 2), (2, 0, 2), (2, 2, -3), (1290, 1290, 1290), (4000, 4000, 200)):
        g = ce.Grid(*dims)
        st = L.ce_create(ctypes.byref(g), K.ctypes.data, K.ctypes.data, 0, None, None, None, ctypes.byref(h))
        assert st == ce.CE_EINVAL
        assert L.ce_last_error(None)           # the context-free message says why
    assert b"32-bit" in L.ce_last_error(None)
    g = ce.Grid(2, 2, 2)
    assert L.ce_create(ctypes.byref(g), None, K.ctypes.data, 0, None, None, None, ctypes.byref(h)) == ce.CE_EINVAL
    assert b"NULL" in L.ce_last_error(None)
    assert L.ce_create(ctypes.byref(g), K.ctypes.data, K.ctypes.data, 0, None, None, None, None) == ce.CE_EINVAL
    c0, c1 = ctypes.c_int(), ctypes.c_int()
    assert L.ce_slab_cells(ctypes.byref(g), 0, 9, ctypes.byref(c0), ctypes.byref(c1)) == ce.CE_EINVAL
    assert b"slab_cells" in L.ce_last_error(None)


def test_sources_target_sm103a_only():
    assert cebuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2410_20441_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "apt_oracle" not in txt, f


def test_binding_structs_match_the_header(tmp_path):
    """sizeof and field offsets of the public structs, as gcc lays them out
    from include/ce.h, equal those of the ctypes mirrors in ce.py."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"ce_grid": (ce.Grid, ("nx", "ny", "nz")),
              "ce_opts": (ce.Opts, ("prec", "bc", "kernel", "St", "Ct", "n_check", "tile")),
              "ce_allocator": (ce.Allocator, ("alloc", "free", "user")),
              "ce_solve_info": (ce.SolveInfo, ("n_cases", "iters", "rel_res", "res0", "status", "sweeps", "checks",
                                               "case_sweeps", "launches", "sweep_ms", "check_ms", "seconds",
                                               "teff_gbs", "rebases", "sweeps_corr", "case_sweeps_corr",
                                               "sweep_ms_corr"))}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ce.h"', "int main(void) {"]
    for st, (_, names) in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for n in names:
            lines.append(f'printf("{st} {n} %zu\\n", offsetof({st}, {n}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st, (cls, names) in fields.items():
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for n in names:
            assert got[(st, n)] == getattr(cls, n).offset, (st, n)
