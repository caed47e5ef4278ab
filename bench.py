#!/usr/bin/env python
"""Benchmark: seconds to a converged 6x6 C_eff of a synthetic porous image.

Workload (default ``porous191``): 191^3 calcite-like matrix (K = 70, G = 30
GPa) with random overlapping spherical pores (radius 3-10 voxels, seeded) to
10 % porosity, pores K = G = 1e-4 GPa; six unit load cases fused in one FP32
sweep per pseudo-time step, FP64 reductions and FP64 defect correction,
relative residual 1e-6.

One step = ce_solve (init, pseudo-time loop with residual checks and
rebases, volume averages) + ce_ceff, with the moduli already resident in
HBM.  The state (3 GB) is far larger than L2, so no flush is needed between
steps.

Printed JSON line (rank 0): value = seconds per C_eff over the whole job
(timed region / (steps * ranks)); `roofline` for the fused sweep kernel:
achieved = the method's algorithmic bytes per sweep (9 state fields per load
case read and written, 72 B per voxel and case, plus 8 B of K, G per voxel)
over the mean launch time, with the velocity-form state the kernel actually
keeps (60 B per voxel and case) beside it; `cpu_baseline` = the FP64 CPU
oracle on a bounded sample; `e2e` = the same metric through the public API
from pinned host buffers; `fp64_plain` = the plain FP64 GPU path with the
load cases solved one after another (a whole solve up to 16 M voxels, a
bounded sample above); `C_vs_oracle` = the C's largest difference from the
FP64 oracle's C of the same image (tests/golden, where stored); `secondary` =
the same measurement on the 479^3 cracked image (the metric's second size),
one timed step.

Multi-GPU (torchrun): every rank solves its own seeded image (weak scaling,
no data-path collective); the barrier and max-over-ranks timing bracket the
timed region.  ``--impl reference`` times the CPU oracle instead (rank 0).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2410_20441_gb300 import images  # noqa: E402

METRIC = "seconds to converged 6x6 C_eff at 191^3/479^3; HBM GB/s per iteration vs peak"
ST_3D = 2.0 * np.pi * np.sqrt(3.0)              # the paper's Strouhal number in 3-D (Eq. PT24q)
ST_POROUS = 0.35 * ST_3D                         # faster for near-void pores on small grids (<= 64^3)
# algorithmic bytes of one sweep of the method: the nine FP32 state fields of
# a load case (p, tau_xx, tau_yy, tau_xy, tau_xz, tau_yz, v_x, v_y, v_z;
# tau_zz = -tau_xx - tau_yy is not stored), each read once and written once,
# plus K and G read once per voxel
BYTES_PER_VOXEL_CASE = 2 * 9 * 4
BYTES_PER_VOXEL_MAT = 2 * 4
# the velocity-form state the fused kernel keeps instead: u (3 x FP32), w high
# part (3 x FP32), w low part (3 x BF16; in the correction phase the FP32
# right-hand side, read only, takes its place at the same byte count)
VFORM_BYTES_PER_VOXEL_CASE = 2 * (3 * 4 + 3 * 4 + 3 * 2)

WORKLOADS = {
    "porous191": dict(n=191, phi=0.10, tol=1e-6, St=0.7 * ST_3D,
                      desc="191^3 matrix K=70 G=30 GPa, overlapping spherical pores r 3-10 to 10% porosity "
                           "(K=G=1e-4 GPa), seed 1+rank; 6 unit load cases fused; tol 1e-6 (FP32 fields, FP64 "
                           "defect correction decides convergence); St = 0.7 x 2 pi sqrt 3 (fastest of 0.4-1.5 x "
                           "the paper's value at this tol)"),
    "porous96": dict(n=96, phi=0.10, tol=1e-6,
                     desc="96^3 matrix with spherical pores to 10% porosity (small profiling case, state 0.4 GB)"),
    "porous127": dict(n=127, phi=0.15, tol=1e-6,
                      desc="127^3 matrix with spherical pores to 15% porosity (adjoint workload size)"),
    "porous479": dict(n=479, phi=0.10, tol=1e-6, St=ST_3D,
                      desc="479^3 matrix with spherical pores to 10% porosity; 6 cases fused; tol 1e-6"),
    "cracked703": dict(n=703, crack=True, tol=1e-6, St=ST_3D, max_iter=20000,
                       desc="703^3 matrix K=70 G=30 GPa with randomly oriented oblate-spheroid cracks (aspect "
                            "0.02-0.05, radius 8-25 voxels, crack density 0.1, crack voxels K=G=1e-4 GPa); 6 unit "
                            "load cases fused; tol 1e-6 (FP64 defect correction); St = 2 pi sqrt 3"),
    "cracked479": dict(n=479, crack=True, tol=1e-6, St=ST_3D,
                       desc="479^3 matrix K=70 G=30 GPa with randomly oriented oblate-spheroid cracks (aspect "
                            "0.02-0.05, radius 8-25 voxels, crack density sum(a^3)/V = 0.1, crack voxels "
                            "K=G=1e-4 GPa), seed 1+rank; 6 unit load cases fused; tol 1e-6 (FP64 defect "
                            "correction); St = 2 pi sqrt 3"),
}
# case-sweeps (sum over sweeps of the active load cases) of the last GPU run
# of each workload, written by `bench.py --record-case-sweeps`; they scale the
# reference arm's bounded oracle sample to a whole solve (the oracle runs the
# same iteration, so it needs the same sweeps)
CASE_SWEEPS_FILE = os.path.join(ROOT, "profiles", "case_sweeps.json")
# the FP64 comparison is a whole solve up to this size (191^3: about 18 s on a
# GB300), a bounded sample above it
FP64_SOLVE_MAX_VOXELS = 16_000_000


def recorded_case_sweeps(workload, tol):
    """The record of `workload` if it was taken at this tolerance and Strouhal number."""
    if not os.path.exists(CASE_SWEEPS_FILE):
        return None
    d = json.load(open(CASE_SWEEPS_FILE)).get(workload)
    St = WORKLOADS[workload].get("St", ST_POROUS)
    if not d or d.get("tol") != tol or abs(d.get("St", 0.0) - St) > 1e-9 * St:
        return None
    return d


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def config_of(workload, world):
    """The `config` object of both arms: the workload and its solve settings."""
    w = WORKLOADS[workload]
    n = w["n"]
    return {"workload": workload, "desc": w["desc"], "voxels": n ** 3, "load_cases": 6, "tol": w["tol"],
            "St": w.get("St", ST_POROUS), "Ct": 0.95 / np.sqrt(3.0),
            "l2": f"inputs larger than L2 (state {2 * 54 * n ** 3 * 4 / 1e9:.1f} GB ping-pong)",
            "parallelism": f"images x{world}"}


def make_image(name, seed):
    w = WORKLOADS[name]
    if w.get("crack"):
        return images.cracked(w["n"], seed=seed)
    return images.random_spheres(w["n"], w["phi"], seed=seed)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    """Hash of the TMA sweep kernels' code (single- and paired-column), with
    comments and blank space removed, so that only a change of the code
    itself makes a committed capture stale."""
    import re
    h = hashlib.sha256()
    for f in ("k_fused.cu", "k_pair.cu", "tma_util.cuh"):
        src = open(os.path.join(ROOT, "paper_2410_20441_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(workload, tile, mode):
    """DRAM bytes of one six-case launch of the sweep in `mode` (dw, f32,
    rhs) from the committed ncu summary, or None when absent, taken on a
    different kernel code or another tile."""
    p = os.path.join(ROOT, "profiles", f"fused_sweep_{workload}.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_sha256_16") != kernel_hash():
        return None
    for cap in d.get("captures", []):
        if list(cap.get("tile", [])) == list(tile) and cap.get("mode") == mode:
            return cap.get("dram_bytes_per_launch")
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                mx.append(float(row[2]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def oracle_sample(K, G, case_sweeps, seconds_budget=20.0):
    """Time the CPU oracle on a bounded sample of the workload: init + a few
    sweeps of load case xx at full size; scale per case-sweep."""
    from oracle import apt
    nz, ny, nx = K.shape
    par = apt.numerical_parameters((nx, ny, nz), St=ST_POROUS)
    e6 = np.eye(6)[0]
    t0 = time.perf_counter()
    st = apt.init_state(K, G, e6)
    apt.sweeps(K, G, e6, st, 1, par)
    t1 = time.perf_counter()
    n = max(1, min(20, int(seconds_budget / max(t1 - t0, 1e-3))))
    t2 = time.perf_counter()
    apt.sweeps(K, G, e6, st, n, par)
    t3 = time.perf_counter()
    per = (t3 - t2) / n
    return {"per_case_sweep_s": per, "sweeps": n + 1, "threads": apt.num_threads(),
            "value": per * case_sweeps if case_sweeps else None, "sample_seconds": t3 - t0}


def run_batch(args, rank, world):
    """--batch: sixteen seeded random-sphere samples of uneven size (64^3 to
    160^3, porosity 5-20 %), six unit load cases each, solved together by
    one CUDA graph (ce_solve_batch); value = seconds per batch of C_eff."""
    import torch
    from paper_2410_20441_gb300 import ce

    smp = images.batch_samples(seeds=range(100 + 16 * rank, 116 + 16 * rank))
    imgs = [(K, G) for (_, _, K, G) in smp]
    vox = [n ** 3 for (n, _, _, _) in smp]
    tol = 1e-5
    tile = args.tile if args.tile == "auto" else tuple(int(t) for t in args.tile.split(","))
    St = args.batch_st * ST_3D
    b = ce.BatchContext(imgs, St=St, n_check=32, tile=tile)
    tile = b.tile
    for _ in range(max(args.warmup, 0)):
        b.solve(tol=tol, max_iter=60000)
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.solve(tol=tol, max_iter=60000)
        C = b.ceff()
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    iters = list(b.iters)
    b.close()
    alg = sum((BYTES_PER_VOXEL_CASE * 6 + BYTES_PER_VOXEL_MAT) * v * it for v, it in zip(vox, iters))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with ce.BatchContext(imgs, St=St, n_check=32, tile=tile) as b2:
        b2.solve(tol=tol, max_iter=60000)
        C2 = b2.ceff()
    torch.cuda.synchronize()
    e2e = time.perf_counter() - t0
    if rank != 0:
        return
    peak, peak_kind = peaks()
    per = t_ms / 1000.0 / args.steps
    line = {"metric": METRIC, "value": per / world, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch16", "desc": "16 random-sphere samples n ~ U{64..160}, porosity "
                       "U[0.05, 0.20], 6 unit load cases each, one CUDA graph per solve; tol 1e-5; value = "
                       "seconds per batch of 16 C_eff", "sizes": [n for (n, _, _, _) in smp],
                       "voxels": sum(vox), "l2": "inputs larger than L2", "tile": list(tile)},
            "iterations": iters,
            "roofline": {"bound": "hbm", "kernel": "k_sweep_tma_batch (whole graph, average)",
                         "achieved": alg / (per * 1e9), "peak": peak, "unit": "GB/s",
                         "frac": alg / (per * 1e9) / peak, "peak_kind": peak_kind, "traffic": None,
                         "note": "algorithmic bytes of all sweeps / whole solve time (includes init, "
                                 "control kernels and averages)"},
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 8 * sum(vox),
                    "d2h_bytes_per_step": 36 * 8 * len(vox),
                    "includes": "ce_create_batch from host moduli, solve, ceff, destroy",
                    "C_matches_device_run": bool(np.abs(C2 - C).max() <= 1e-6 * np.abs(C).max())},
            "clocks": ck}
    print(json.dumps(line), flush=True)


def run_split(args, rank, world, local, dev):
    """--split cases|slab: one image over the ranks (strong scaling).  cases:
    load case m on rank m mod N, the volume averages gathered, C = S E^-1 on
    every rank.  slab: the z-slab decomposition (slab.DistSlab over NCCL), one
    slab per rank, a one-plane halo exchange after every sweep; slabs keep the
    double-word state without defect correction, so this mode solves to the
    tolerance that state reaches (1e-5)."""
    import torch
    import torch.distributed as dist
    from paper_2410_20441_gb300 import ce, shard, slab

    w = WORKLOADS[args.workload]
    K, G = make_image(args.workload, 1)          # the same image on every rank
    nz, ny, nx = K.shape
    N = nx * ny * nz
    St = w.get("St", ST_POROUS)
    tile = args.tile if args.tile == "auto" else tuple(int(t) for t in args.tile.split(","))
    max_iter = w.get("max_iter", 50000)
    tol = w["tol"] if args.split == "cases" else max(w["tol"], 1e-5)
    Kd, Gd = torch.tensor(K, device=dev), torch.tensor(G, device=dev)
    infos = []
    if args.split == "cases":
        ctx = ce.Context(Kd, Gd, prec="fp32", St=St, tile=tile)
        tile = ctx.tile

        def step():
            mine = [m for m in range(6) if shard.case_owner(m, world) == rank]
            ctx.solve(np.eye(6)[mine], tol=tol, max_iter=max_iter)
            infos.append(dict(ctx.info))
            sig, eps = ctx.averages()
            got = shard.gather({m: (sig[q].tolist(), eps[q].tolist()) for q, m in enumerate(mine)})
            sums = np.array([got[m][0] + got[m][1] for m in range(6)])
            return ce.ceff_from_sums(sums, (1, 1, 1))
        close = ctx.close
    else:
        z0, z1 = slab.plane_ranges(nz, world)[rank]
        t = (3, 16, 64, 1) if tile == "auto" else tile
        sl = ce.Slab(Kd, Gd, z0, z1, St=St, tile=t)
        d = slab.DistSlab(sl, device=dev)
        tile = t

        def step():
            it, rel, st = d.solve(None, tol=tol, max_iter=max_iter)
            infos.append({"iters": [int(v) for v in it], "rel_res": [float(v) for v in rel]})
            return d.ceff()
        close = sl.close
    for _ in range(max(args.warmup, 0)):
        step()
    infos.clear()
    clocks = Clocks(local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        C = step()
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    ck = clocks.stop()
    t_ms = shard.max_over_ranks(e0.elapsed_time(e1), device=dev)
    wall = shard.max_over_ranks(time.perf_counter() - t0, device=dev)
    close()
    # end to end: this rank's share from pinned host moduli (create, solve, C, destroy)
    Kp, Gp = torch.from_numpy(K).pin_memory(), torch.from_numpy(G).pin_memory()
    dist.barrier()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    if args.split == "cases":
        with ce.Context(Kp, Gp, prec="fp32", St=St, tile=tile) as c2:
            mine = [m for m in range(6) if shard.case_owner(m, world) == rank]
            c2.solve(np.eye(6)[mine], tol=tol, max_iter=max_iter)
            sig, eps = c2.averages()
        got = shard.gather({m: (sig[q].tolist(), eps[q].tolist()) for q, m in enumerate(mine)})
        C2 = ce.ceff_from_sums(np.array([got[m][0] + got[m][1] for m in range(6)]), (1, 1, 1))
    else:
        sl2 = ce.Slab(Kp, Gp, z0, z1, St=St, tile=tile)
        d2 = slab.DistSlab(sl2, device=dev)
        d2.solve(None, tol=tol, max_iter=max_iter)
        C2 = d2.ceff()
        sl2.close()
    torch.cuda.synchronize()
    e2e = shard.max_over_ranks(time.perf_counter() - t1, device=dev)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": t_ms / 1000.0 / args.steps, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(config_of(args.workload, world), tol=tol,
                           parallelism=f"{'load cases' if args.split == 'cases' else 'z-slabs'} x{world}",
                           split=args.split,
                           **({"desc": WORKLOADS[args.workload]["desc"].replace("tol 1e-6 (FP32 fields, FP64 defect "
                                                                               "correction decides convergence)",
                                                                               "tol 1e-5 (slabs keep the double-word "
                                                                               "state without defect correction)")}
                              if args.split == "slab" else {})),
            "tile": list(tile), "wall_s_per_step": wall / args.steps,
            "iterations": infos[-1]["iters"], "rel_res": infos[-1]["rel_res"],
            "C_diag": [float(C[q, q]) for q in range(6)],
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 36 * 8,
                    "includes": "create from pinned host moduli, solve, gather, C, destroy (per rank, max)",
                    "C_matches_device_run": bool(np.abs(C2 - C).max() <= 1e-6 * np.abs(C).max())},
            "clocks": ck}
    print(json.dumps(line), flush=True)


def run_reference(args, rank):
    """--impl reference: the CPU oracle as it stands, bounded samples."""
    if rank != 0:
        return
    K, G = make_image(args.workload, 1)
    w = WORKLOADS[args.workload]
    rec = recorded_case_sweeps(args.workload, w["tol"])
    if rec is None:
        cs = 6 * 10 * w["n"]          # paper's upper rule of thumb, 10 nx per load case (Sec. 3.1)
        how = "10 nx sweeps per load case (Sec. 3.1 rule), 6 cases"
    else:
        cs = rec["case_sweeps"]
        how = (f"case-sweeps of the GPU solve of this workload and tol recorded in profiles/case_sweeps.json "
               f"({rec.get('when', '')}, {rec.get('source', '')})")
    vals = []
    for _ in range(args.warmup):
        oracle_sample(K, G, cs, seconds_budget=5.0)
    samples = []
    for _ in range(args.steps):
        s = oracle_sample(K, G, cs, seconds_budget=10.0)
        samples.append(s)
        vals.append(s["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.median(
                [s["sample_seconds"] for s in samples]), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, args.gpus),
            "cpu_baseline": {"value": v, "unit": "s", "cores": samples[0]["threads"], "kind": "oracle",
                             "sample": f"init + {samples[0]['sweeps']} sweeps of load case xx at full size; "
                                       f"seconds per case-sweep x {cs} case-sweeps ({how})"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """A short fixed run of the fused sweep for ncu: no oracle, no tuning."""
    import torch
    from paper_2410_20441_gb300 import ce
    if args.tile == "auto":
        raise SystemExit("--profile-sweeps needs an explicit --tile")
    tile = tuple(int(t) for t in args.tile.split(","))
    w = WORKLOADS[args.workload]
    K, G = make_image(args.workload, 1)
    n = args.profile_sweeps
    with ce.Context(torch.tensor(K, device="cuda"), torch.tensor(G, device="cuda"), prec="fp32", kernel="fused",
                    St=w.get("St", ST_POROUS), n_check=n, tile=tile) as c:
        if args.profile_mode == "rhs":
            # one sweep and a rebase, then n sweeps of the correction phase
            # (the warm start rebases at once): launches 2 .. n + 1
            c.solve(None, tol=0.0, max_iter=1, check=False, refine="each")
            c.solve(None, tol=0.0, max_iter=n, check=False, warm=True)
        else:
            # dw: the double-word state of unrefined solves; f32: the first
            # phase of a refined solve (no rebase within n sweeps)
            c.solve(None, tol=0.0, max_iter=n, check=False, refine="off" if args.profile_mode == "dw" else "auto")
        print(json.dumps({"workload": args.workload, "tile": list(tile), "mode": args.profile_mode,
                          "sweeps": c.info["sweeps"], "rebases": c.info["rebases"],
                          "ms_per_sweep": c.info["sweep_ms"] / max(c.info["sweeps"], 1)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="porous191", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain GPU sample")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 479^3 cracked secondary measurement")
    ap.add_argument("--record-case-sweeps", action="store_true",
                    help="write this run's case-sweeps per solve to profiles/case_sweeps.json (they scale the "
                         "reference arm's oracle sample)")
    ap.add_argument("--tile", default="auto", help="stages,rows,planes of the TMA sweep, or auto (tuned and "
                                                    "cached before the timed region)")
    ap.add_argument("--batch-st", type=float, default=0.7,
                    help="Strouhal number of the batch as a multiple of 2 pi sqrt 3")
    ap.add_argument("--split", default="none", choices=["none", "cases", "slab"],
                    help="split one image over the torchrun ranks: its load cases, or z-slabs with a halo "
                         "exchange (strong scaling); default: every rank solves its own image (weak scaling)")
    ap.add_argument("--batch", action="store_true",
                    help="time the batched solve of 16 uneven samples (64^3-160^3) instead")
    ap.add_argument("--profile-mode", default="f32", choices=["dw", "f32", "rhs"],
                    help="state of the profiled sweeps: dw (double-word w), f32 (first phase of a refined "
                         "solve) or rhs (correction phase)")
    ap.add_argument("--profile-sweeps", type=int, default=0, metavar="N",
                    help="profiling case instead of the benchmark: N fixed sweeps of the six cases of the "
                         "workload with --tile (no tuning; the last sweep measures the residual), then exit")
    args = ap.parse_args()
    if args.profile_sweeps > 0:
        run_profile_case(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2410_20441_gb300 import ce

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if args.split != "none":
        if world == 1:
            dist.init_process_group("nccl", init_method="tcp://127.0.0.1:" + str(_free_port()), rank=0,
                                    world_size=1, device_id=torch.device("cuda", local))
        run_split(args, rank, world, local, torch.device("cuda", local))
        dist.barrier()
        dist.destroy_process_group()
        return
    if args.batch:
        if world > 1:
            dist.barrier()
        run_batch(args, rank, world)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    dev = torch.device("cuda", local)
    line = measure(args, args.workload, args.steps, args.warmup, world, rank, local, dev, baselines=True)
    if (line is not None and args.workload == "porous191" and world == 1 and not args.no_secondary):
        # the metric's second size: the 479^3 cracked image, one timed step
        sec = measure(args, "cracked479", 1, 1, world, rank, local, dev, baselines=False)
        keep = ("value", "unit", "ms_per_step", "steps", "warmup", "config", "iterations", "sweeps_per_step",
                "sweeps_per_s", "rel_res", "rebases", "C_diag", "roofline", "gpu_launches", "e2e", "clocks")
        line["secondary"] = {k: sec[k] for k in keep if k in sec}
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def measure(args, workload, steps, warmup, world, rank, local, dev, baselines):
    """Time `steps` solves of `workload` after `warmup` untimed ones; returns
    the JSON line on rank 0 (None elsewhere)."""
    import torch
    import torch.distributed as dist
    from paper_2410_20441_gb300 import ce

    w = WORKLOADS[workload]
    seed = 1 + rank
    K, G = make_image(workload, seed)
    nz, ny, nx = K.shape
    N = nx * ny * nz
    tile = args.tile if args.tile == "auto" else tuple(int(t) for t in args.tile.split(","))
    Kd = torch.tensor(K, device=dev)
    Gd = torch.tensor(G, device=dev)
    St = w.get("St", ST_POROUS)
    ctx = ce.Context(Kd, Gd, prec="fp32", St=St, tile=tile)
    tile = ctx.tile
    stream = torch.cuda.current_stream(dev)

    max_iter = w.get("max_iter", 50000)

    def step():
        ctx.solve(None, tol=w["tol"], max_iter=max_iter)
        return ctx.ceff()

    for _ in range(max(warmup, 0)):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    infos = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        C = step()
        infos.append(dict(ctx.info))
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([t_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())

    # fused-sweep kernel: device time per launch from the library's events,
    # split by phase (first phase of a refined solve: FP32 w, mode f32;
    # correction phase: mode rhs)
    sweeps = sum(i["sweeps"] for i in infos)
    case_sweeps = sum(i["case_sweeps"] for i in infos)
    sweep_ms = sum(i["sweep_ms"] for i in infos)
    peak, peak_kind = peaks()
    n_corr = sum(i["sweeps_corr"] for i in infos)
    first = "dw" if tile[3] == 2 else "f32"      # the paired-column sweep keeps the double-word state
    phase = {first: (sweeps - n_corr, case_sweeps - sum(i["case_sweeps_corr"] for i in infos),
                     sweep_ms - sum(i["sweep_ms_corr"] for i in infos)),
             "rhs": (n_corr, sum(i["case_sweeps_corr"] for i in infos), sum(i["sweep_ms_corr"] for i in infos))}

    def roof(ns, ncs, ms, mode):
        alg = BYTES_PER_VOXEL_CASE * N * ncs + BYTES_PER_VOXEL_MAT * N * ns
        vf = VFORM_BYTES_PER_VOXEL_CASE * N * ncs + BYTES_PER_VOXEL_MAT * N * ns
        t = ms / ns * 1e-3
        t6 = traffic_per_launch(workload, tile, mode)
        return {"sweeps": ns, "avg_active_cases": ncs / ns, "avg_launch_ms": ms / ns,
                "bytes_per_launch": alg / ns, "achieved": alg / ns / t / 1e9, "frac": alg / ns / t / 1e9 / peak,
                "achieved_vform": vf / ns / t / 1e9, "frac_vform": vf / ns / t / 1e9 / peak,
                "traffic_six_case_launch": t6,
                "traffic": (t6 * (ncs / ns) / 6.0 if t6 else None)}

    phases = {k: roof(*v, k) for k, v in phase.items() if v[0] > 0}
    dom = max(phases, key=lambda k: phase[k][2])
    whole = roof(sweeps, case_sweeps, sweep_ms, dom)
    launches = sum(i["launches"] for i in infos) // steps
    name = {"f32": "first phase, FP32 w", "rhs": "correction phase, FP32 correction + FP64 right-hand side",
            "dw": "double-word w"}
    if args.record_case_sweeps and rank == 0:
        d = json.load(open(CASE_SWEEPS_FILE)) if os.path.exists(CASE_SWEEPS_FILE) else {}
        d[workload] = {"case_sweeps": case_sweeps // steps, "tol": w["tol"], "St": St,
                       "iterations": infos[-1]["iters"], "when": time.strftime("%Y-%m-%d"),
                       "source": "bench.py --record-case-sweeps on one GB300"}
        with open(CASE_SWEEPS_FILE, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)

    # end to end through the public API from pinned host buffers (the timed
    # context is released first: at 703^3 two contexts do not fit in HBM)
    ctx.close()
    torch.cuda.synchronize()
    Kp = torch.from_numpy(K).pin_memory()
    Gp = torch.from_numpy(G).pin_memory()
    e2e_t = []
    for r in range(2 if N < 50_000_000 else 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ce.Context(Kp, Gp, prec="fp32", St=St, tile=tile) as c2:
            c2.solve(None, tol=w["tol"], max_iter=max_iter)
            C2 = c2.ceff()
            inf2 = dict(c2.info)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_d2h = 36 * 8 + 8 * (inf2["checks"] * 6) + 6 * 12 * 8

    if rank != 0:
        return None
    i0 = infos[-1]
    line = {
        "metric": METRIC, "value": t_ms / 1000.0 / (steps * world), "unit": "s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": t_ms / steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": config_of(workload, world),
        "precision": "FP32 fields, FP64 residual and average reductions, FP64 defect correction",
        "tile": list(tile),
        "iterations": i0["iters"], "sweeps_per_step": i0["sweeps"], "case_sweeps_per_step": i0["case_sweeps"],
        "sweeps_per_s": i0["sweeps"] * steps * world / (t_ms / 1000.0),
        "rel_res": i0["rel_res"], "rebases": i0["rebases"],
        "C_diag": [float(C[q, q]) for q in range(6)],
        "roofline": {"bound": "hbm",
                     "kernel": f"k_sweep_tma ({name.get(dom, dom)}; single-column fused TMA sweep, one load case "
                               "per block)",
                     "achieved": phases[dom]["achieved"], "peak": peak, "unit": "GB/s",
                     "frac": phases[dom]["frac"], "peak_kind": peak_kind,
                     "traffic": phases[dom]["traffic"],
                     "bytes": "the method's state: 72 B per voxel and active case + 8 B of K, G per voxel",
                     "bytes_per_launch": phases[dom]["bytes_per_launch"],
                     "avg_launch_ms": phases[dom]["avg_launch_ms"],
                     "achieved_vform": phases[dom]["achieved_vform"], "frac_vform": phases[dom]["frac_vform"],
                     "bytes_vform": "the velocity-form state the kernel keeps: 60 B per voxel and active case "
                                    "+ 8 B of K, G per voxel (first phase: 48 B)",
                     "traffic_note": "ncu DRAM bytes of a six-case launch, scaled by the average active cases",
                     "phases": phases, "all_sweeps": {k: whole[k] for k in ("achieved", "frac", "avg_launch_ms")},
                     "sweep_share_of_step": sweep_ms / t_ms},
        "gpu_launches": launches * steps,
        "e2e": {"value": min(e2e_t), "unit": "s", "h2d_bytes_per_step": 2 * N * 4,
                "d2h_bytes_per_step": e2e_d2h, "includes": "ce_create from pinned host moduli, solve, "
                                                           "ceff, destroy",
                "C_matches_device_run": bool(np.abs(C2 - C).max() <= 1e-6 * np.abs(C).max())},
        "clocks": ck,
    }
    # the FP64 CPU oracle's C of the same image, where one is stored (written
    # by tests/golden/make_golden.py from the oracle alone)
    gold = os.path.join(ROOT, "tests", "golden", f"{workload}.json")
    if seed == 1 and os.path.exists(gold):
        g = json.load(open(gold))
        Cg = np.array(g["C"])
        line["C_vs_oracle"] = {"max_rel_err": float(np.abs(C - Cg).max() / np.abs(Cg).max()),
                               "oracle": f"tests/golden/{workload}.json: the FP64 CPU oracle's C of the same "
                                         f"image converged to tol {g['tol']:g}"}
    if baselines and not args.no_fp64 and N <= FP64_SOLVE_MAX_VOXELS:
        # the plain FP64 GPU path (the paper's stress form, no fusion), the six
        # load cases solved one after another to the same tolerance, timed
        # whole; C from their averages against the FP32 run's
        t64, its, sig, eps, cs64, sw64 = 0.0, [], [], [], 0, 0.0
        with ce.Context(Kd, Gd, prec="fp64", St=St) as c3:
            for m in range(6):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c3.solve(np.eye(6)[m][None], tol=w["tol"], max_iter=max_iter)
                torch.cuda.synchronize()
                t64 += time.perf_counter() - t0
                i3 = c3.info
                its.append(i3["iters"][0])
                cs64 += i3["case_sweeps"]
                sw64 += i3["sweep_ms"]
                s3, e3 = c3.averages()
                sig.append(s3[0])
                eps.append(e3[0])
        C64 = np.array(sig).T @ np.linalg.inv(np.array(eps).T)
        per = sw64 / cs64 / 1000.0
        line["fp64_plain"] = {"value": t64, "unit": "s", "iterations": its, "case_sweeps": cs64,
                              "per_case_sweep_ms": per * 1e3, "achieved_GBps": 160 * N / per / 1e9,
                              "C_max_rel_diff_vs_fp32": float(np.abs(C64 - C).max() / np.abs(C64).max()),
                              "sample": "measured: the six load cases solved one after another to the same "
                                        "tol (wall time, synchronised)"}
    elif baselines and not args.no_fp64:
        # larger images: a bounded sample of sweeps of case xx, scaled by the
        # case-sweeps of the FP32 solve
        with ce.Context(Kd, Gd, prec="fp64", St=St, n_check=200) as c3:
            c3.solve(np.eye(6)[:1], tol=0.0, max_iter=200, check=False)
            c3.solve(np.eye(6)[:1], tol=0.0, max_iter=400, check=False)
            i3 = c3.info
        per = i3["sweep_ms"] / i3["sweeps"] / 1000.0
        line["fp64_plain"] = {"per_case_sweep_ms": per * 1e3, "value_extrapolated_s": per * case_sweeps / steps,
                              "sample": "400 plain FP64 sweeps of load case xx, scaled by the FP32 run's "
                                        "case-sweeps", "achieved_GBps": 160 * N / per / 1e9}
    if baselines and not args.no_cpu:
        s = oracle_sample(K, G, case_sweeps / steps)
        line["cpu_baseline"] = {"value": s["value"], "unit": "s", "cores": s["threads"], "kind": "oracle",
                                "sample": f"init + {s['sweeps']} FP64 sweeps of load case xx at full size "
                                          f"({s['sample_seconds']:.1f} s), scaled to the "
                                          f"{case_sweeps // steps} case-sweeps of one GPU solve"}
    return line


if __name__ == "__main__":
    main()
