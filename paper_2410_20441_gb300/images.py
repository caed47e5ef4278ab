"""Seeded synthetic voxel images (bulk modulus K and shear modulus G per voxel).

This module holds only input generation: geometry, seeds and material values.
It contains none of the solver's arithmetic, so both the CUDA path and the
CPU oracle may consume its arrays.

Conventions
-----------
* Arrays have shape ``(nz, ny, nx)`` (C order, x fastest), dtype float32, GPa.
* Voxel (i, j, k) has its centre at (i + 1/2, j + 1/2, k + 1/2) with unit
  voxel size.  A voxel belongs to a shape when its centre lies inside the
  shape; ties (distance exactly on the surface) count as inside.
* Cracks thinner than one voxel are thickened to a half-thickness of 1/2
  voxel, so that every crack is at least one voxel thick (the paper's
  discussion of accuracy states that one voxel suffices for a crack, Sec. 5.1).

Workloads (the paper's data sets are not used; these stand in for them):
* ``single_sphere``: one centred spherical inclusion (the Eshelby check, Sec. 4.2).
* ``random_spheres``: matrix with overlapping spherical pores added until a
  target porosity is first reached (a porous-rock image of the paper's
  191^3 size, Abstract and Sec. 4.3).
* ``cracked``: matrix with randomly oriented oblate-spheroid cracks added
  until a target crack density sum(a^3)/V is first reached (stands in for
  the segmented cracked-marble image of Sec. 4.3).
* ``cracked_scaled``: one crack set defined in the unit box, rasterised at any
  n (the several resolutions of one image in Sec. 4.3).
* ``laminate``: layers normal to z (Model 1, Sec. 4.1, Table 1).
"""
from __future__ import annotations

import numpy as np

CALCITE = (70.0, 30.0)          # K, G of the matrix (GPa), Table 5 background
PORE = (1e-4, 1e-4)             # near-void phase used for pores and cracks
LAYER_STIFF = (36.0, 44.0)      # Table 1, layer 1
LAYER_SOFT = (7.2, 8.8)         # Table 1, layer 2


def _shape3(n):
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = (int(v) for v in n)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid extents must be >= 1")
    return nx, ny, nz


def _fill(nx, ny, nz, phase):
    K = np.full((nz, ny, nx), phase[0], dtype=np.float32)
    G = np.full((nz, ny, nx), phase[1], dtype=np.float32)
    return K, G


def homogeneous(n, K=70.0, G=30.0):
    nx, ny, nz = _shape3(n)
    return _fill(nx, ny, nz, (K, G))


def random_moduli(n, seed, kmin=1.0, kmax=80.0, gmin=0.5, gmax=40.0):
    """Independent uniform K, G per voxel (small-grid parity inputs)."""
    nx, ny, nz = _shape3(n)
    rng = np.random.default_rng(seed)
    K = rng.uniform(kmin, kmax, size=(nz, ny, nx)).astype(np.float32)
    G = rng.uniform(gmin, gmax, size=(nz, ny, nx)).astype(np.float32)
    return K, G


def two_phase_random(n, seed, frac=0.3, matrix=CALCITE, inclusion=PORE):
    """Each voxel independently takes the inclusion phase with probability frac."""
    nx, ny, nz = _shape3(n)
    rng = np.random.default_rng(seed)
    mask = rng.random((nz, ny, nx)) < frac
    K, G = _fill(nx, ny, nz, matrix)
    K[mask] = inclusion[0]
    G[mask] = inclusion[1]
    return K, G


def _centres(nx, ny, nz):
    z = (np.arange(nz, dtype=np.float64) + 0.5)[:, None, None]
    y = (np.arange(ny, dtype=np.float64) + 0.5)[None, :, None]
    x = (np.arange(nx, dtype=np.float64) + 0.5)[None, None, :]
    return x, y, z


def sphere_mask(n, centre, radius):
    nx, ny, nz = _shape3(n)
    x, y, z = _centres(nx, ny, nz)
    d2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return d2 <= radius * radius


def single_sphere(n, radius_frac=0.25, matrix=CALCITE, inclusion=(2.25, 1e-3)):
    """Centred sphere of radius radius_frac * L (L = nx) in a uniform matrix."""
    nx, ny, nz = _shape3(n)
    K, G = _fill(nx, ny, nz, matrix)
    m = sphere_mask((nx, ny, nz), (nx / 2, ny / 2, nz / 2), radius_frac * nx)
    K[m] = inclusion[0]
    G[m] = inclusion[1]
    return K, G


def spheroid(n, centre, a, alpha, matrix=(36.0, 44.0), inclusion=(1e-3, 2e-3)):
    """Spheroid with semi-axes (a, a, alpha a), symmetry axis z, centred at
    `centre` (x, y, z; may lie on the box's faces or corners) in a uniform
    matrix; returns K, G and the voxel volume fraction of the inclusion."""
    nx, ny, nz = _shape3(n)
    x, y, z = _centres(nx, ny, nz)
    c = alpha * a
    m = ((x - centre[0]) ** 2 + (y - centre[1]) ** 2) / (a * a) + (z - centre[2]) ** 2 / (c * c) <= 1.0
    K, G = _fill(nx, ny, nz, matrix)
    K[m] = inclusion[0]
    G[m] = inclusion[1]
    return K, G, float(m.mean())


def single_spheroid(n, a, alpha, matrix=(36.0, 44.0), inclusion=(1e-3, 2e-3)):
    """Centred spheroid with semi-axes (a, a, alpha a), symmetry axis z, in a
    uniform matrix (defaults: the moduli of Sec. 4.2's single-inclusion model);
    returns K, G and the voxel volume fraction of the inclusion."""
    nx, ny, nz = _shape3(n)
    return spheroid((nx, ny, nz), (nx / 2, ny / 2, nz / 2), a, alpha, matrix, inclusion)


def random_spheres(n, porosity, seed, rmin=3.0, rmax=10.0, matrix=CALCITE,
                   pore=PORE):
    """Overlapping spheres, centres uniform in the box, radii uniform in
    [rmin, rmax]; spheres are added until the pore fraction first reaches
    ``porosity``."""
    nx, ny, nz = _shape3(n)
    rng = np.random.default_rng(seed)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    total = nx * ny * nz
    count = 0
    while count < porosity * total:
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz], dtype=np.float64)
        r = rng.uniform(rmin, rmax)
        lo = [max(0, int(np.floor(c[a] - r - 1))) for a in range(3)]
        hi = [min(s, int(np.ceil(c[a] + r + 1))) for a, s in enumerate((nx, ny, nz))]
        x = (np.arange(lo[0], hi[0], dtype=np.float64) + 0.5)[None, None, :]
        y = (np.arange(lo[1], hi[1], dtype=np.float64) + 0.5)[None, :, None]
        z = (np.arange(lo[2], hi[2], dtype=np.float64) + 0.5)[:, None, None]
        inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
        sub = mask[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        count += int(np.count_nonzero(inside & ~sub))
        sub |= inside
    K, G = _fill(nx, ny, nz, matrix)
    K[mask] = pore[0]
    G[mask] = pore[1]
    return K, G


def cracked(n, seed, density=0.1, amin=8.0, amax=25.0, alpha=(0.02, 0.05),
            matrix=CALCITE, crack=PORE):
    """Randomly oriented oblate-spheroid cracks (semi-axes a, a, c = alpha*a,
    normal uniform on the unit sphere, centre uniform in the box), added
    until sum(a^3)/V first reaches ``density``."""
    nx, ny, nz = _shape3(n)
    rng = np.random.default_rng(seed)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    vol = float(nx * ny * nz)
    acc = 0.0
    while acc < density * vol:
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz], dtype=np.float64)
        a = rng.uniform(amin, amax)
        asp = rng.uniform(alpha[0], alpha[1])
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        ceff = max(asp * a, 0.5)
        lo = [max(0, int(np.floor(c[q] - a - 1))) for q in range(3)]
        hi = [min(s, int(np.ceil(c[q] + a + 1))) for q, s in enumerate((nx, ny, nz))]
        acc += a ** 3
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        x = (np.arange(lo[0], hi[0], dtype=np.float64) + 0.5 - c[0])[None, None, :]
        y = (np.arange(lo[1], hi[1], dtype=np.float64) + 0.5 - c[1])[None, :, None]
        z = (np.arange(lo[2], hi[2], dtype=np.float64) + 0.5 - c[2])[:, None, None]
        along = x * nrm[0] + y * nrm[1] + z * nrm[2]
        r2 = x * x + y * y + z * z - along * along
        inside = r2 / (a * a) + (along * along) / (ceff * ceff) <= 1.0
        mask[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= inside
    K, G = _fill(nx, ny, nz, matrix)
    K[mask] = crack[0]
    G[mask] = crack[1]
    return K, G


def cracked_scaled(n, seed, density=0.1, a_frac=(8.0 / 479, 25.0 / 479), alpha=(0.02, 0.05), matrix=CALCITE,
                   crack=PORE):
    """One set of randomly oriented oblate-spheroid cracks defined in the unit
    box (centres, normals, radii a_frac of the box edge, aspect ratios) and
    rasterised on an n^3 grid, so that several n give the same geometry at
    several resolutions.  Cracks are drawn until sum(a^3) (box units) first
    reaches ``density``; a crack thinner than a voxel is thickened to a
    half-thickness of 1/2 voxel at every n (the paper's one-voxel rule)."""
    nx, ny, nz = _shape3(n)
    rng = np.random.default_rng(seed)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    ext = np.array([nx, ny, nz], dtype=np.float64)
    h = float(max(nx, ny, nz))
    acc = 0.0
    while acc < density:
        c = rng.uniform(0.0, 1.0, 3) * ext
        a1 = rng.uniform(a_frac[0], a_frac[1])
        asp = rng.uniform(alpha[0], alpha[1])
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        acc += a1 ** 3
        a = a1 * h
        ceff = max(asp * a, 0.5)
        lo = [max(0, int(np.floor(c[q] - a - 1))) for q in range(3)]
        hi = [min(s, int(np.ceil(c[q] + a + 1))) for q, s in enumerate((nx, ny, nz))]
        if any(hh <= ll for ll, hh in zip(lo, hi)):
            continue
        x = (np.arange(lo[0], hi[0], dtype=np.float64) + 0.5 - c[0])[None, None, :]
        y = (np.arange(lo[1], hi[1], dtype=np.float64) + 0.5 - c[1])[None, :, None]
        z = (np.arange(lo[2], hi[2], dtype=np.float64) + 0.5 - c[2])[:, None, None]
        along = x * nrm[0] + y * nrm[1] + z * nrm[2]
        r2 = x * x + y * y + z * z - along * along
        inside = r2 / (a * a) + (along * along) / (ceff * ceff) <= 1.0
        mask[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= inside
    K, G = _fill(nx, ny, nz, matrix)
    K[mask] = crack[0]
    G[mask] = crack[1]
    return K, G


def laminate(n, layer=15, stiff=LAYER_STIFF, soft=LAYER_SOFT):
    """Layers of ``layer`` voxels normal to z; odd layers (counted from z=0)
    are the stiff phase.  At nz = 191 with 15-voxel layers this gives the
    stiff fraction 90/191 = 0.4712 of Model 1 (Sec. 4.1)."""
    nx, ny, nz = _shape3(n)
    K, G = _fill(nx, ny, nz, soft)
    k = np.arange(nz)
    st = (k // layer) % 2 == 1
    K[st] = stiff[0]
    G[st] = stiff[1]
    return K, G


# ---------------------------------------------------------------- workloads
def porous_191(seed=1, n=191):
    """191^3 matrix (70/30 GPa) with overlapping spherical pores (radius
    3-10 voxels) to 10 % porosity, pores 1e-4 GPa."""
    return random_spheres(n, 0.10, seed)


def batch_samples(seeds=range(100, 116), nmin=64, nmax=160):
    """Sixteen cubes of uneven size n ~ U{nmin..nmax}, porosity ~ U[0.05, 0.20],
    random spheres as in ``porous_191``; one seed per sample."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(s)
        n = int(rng.integers(nmin, nmax + 1))
        phi = float(rng.uniform(0.05, 0.20))
        K, G = random_spheres(n, phi, seed=10_000 + s)
        out.append((n, phi, K, G))
    return out


def adjoint_weights(seed=7):
    """Weights w_mn ~ N(0, 1) of the scalar J = sum_mn w_mn C_mn."""
    return np.random.default_rng(seed).normal(size=(6, 6))


def unit_loads():
    """Six unit macroscopic strains in Voigt order xx, yy, zz, yz, xz, xy with
    engineering shear (so load 5 has eps_xz = eps_zx = 1/2)."""
    return np.eye(6, dtype=np.float64)
