"""Launch-shape autotuning of the FP32 TMA sweep, with a JSON cache.

The search itself runs in the library (ce_autotune: copy stages x rows per
block x z-planes per block, timed on the device).  This module keys its
result by grid shape, precision, number of load cases, boundary condition,
GPU model and library build, and keeps it in a JSON file so that a shape is
tuned once per machine:

    {"<key>": {"tile": [stages, rows, planes, columns], "ms_per_sweep": t, "when": ...}}

The cache file is ``$CE_TUNE_CACHE`` when set, else
``~/.cache/paper_2410_20441_gb300/tune.json``.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import ce as _ce


def cache_path() -> str:
    p = os.environ.get("CE_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2410_20441_gb300", "tune.json")


def _library_tag() -> str:
    L = _ce.load()
    path = getattr(L, "_name", None)
    if path and os.path.exists(path):
        st = os.stat(path)
        return hashlib.sha256(f"{st.st_size}:{int(st.st_mtime)}".encode()).hexdigest()[:12]
    return "unknown"


def gpu_tag() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            p = torch.cuda.get_device_properties(torch.cuda.current_device())
            return f"{p.name}|sm{p.multi_processor_count}"
    except ImportError:
        pass
    return "cpu"


def key(shape, prec="fp32", n_cases=6, bc="kubc", gpu=None, lib=None) -> str:
    nx, ny, nz = shape
    return f"{nx}x{ny}x{nz}|{prec}|{n_cases}|{bc}|{gpu or gpu_tag()}|{lib or _library_tag()}"


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(k: str, tile, ms: float, path=None) -> None:
    """Add one entry; the file is replaced atomically (write, then rename)."""
    path = path or cache_path()
    d = load_cache(path)
    d[k] = {"tile": [int(t) for t in tile], "ms_per_sweep": float(ms),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(k: str, path=None):
    e = load_cache(path).get(k)
    if not e or len(e.get("tile", [])) != 4:
        return None
    return tuple(int(t) for t in e["tile"])


def tune_context(ctx, sweeps: int = 6, path=None, force: bool = False, solves: str = "auto"):
    """Give a single-image FP32 context its cached tile, or search and cache
    one, for the solves it will serve ("auto", "plain" or "refined", as
    Context.autotune).  Returns (tile, ms_per_sweep or None when taken from
    the cache)."""
    k = key(ctx.shape, ctx.prec, 6, ctx.bc)
    if solves != "auto":
        k += "|" + solves
    if not force:
        t = lookup(k, path)
        if t is not None:
            ctx.set_tile(t)
            return t, None
    tile, ms = ctx.autotune(sweeps, solves=solves)
    store(k, tile, ms, path)
    return tile, ms
