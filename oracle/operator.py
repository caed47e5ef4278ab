"""ORACLE -- test infrastructure only (never imported by the product path).

Route R2 of the oracle: the discrete problem written out as a minimum of
stored energy and solved directly.  The APT iteration (route R1, the C code)
must converge to exactly this solution.

The continuous statement is equilibrium (Eq. eq:1a), Hooke's law (Eq. eq:2a)
and the strain-velocity relation (Eq. eq:3a), with the effective stiffness
defined through volume averages (Eqs. BC:1 - BC:3).  On the staggered grid of
Sec. 3.3 the velocity fluctuation w (boundary values zero) maps linearly to
the strain components

    cells:   e_xx, e_yy, e_zz                (one each per voxel)
    edges:   e_xy, e_xz, e_yz (tensor shear)  (on the edge lattices)

s(w) = B w + sbar, where sbar is the strain of v = ebar . x.  With the
elastic energy

    E(w) = 1/2 sum_cells [lambda (tr e)^2 + 2 G e_ii e_ii]
         + 1/2 sum_edges omega_e 4 G_e e_e^2,

(omega_e = trapezoid weight of the edge, G_e = mean G of the adjacent cells)
the discrete equilibrium is A w = b with A = B^T D B, b = -B^T D sbar, and the
energy form of the stiffness is C_mn = s^m . D s^n / V.  Everything here is
plain numpy / scipy; nothing is shared with the C oracle or the CUDA code.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class Operator:
    def __init__(self, K, G, bc=0):
        K = np.asarray(K, dtype=np.float64)
        G = np.asarray(G, dtype=np.float64)
        self.K, self.G, self.bc = K, G, bc
        nz, ny, nx = K.shape
        self.n = (nx, ny, nz)
        # face arrays (all faces, boundary included)
        self.shp_wx = (nz, ny, nx + 1)
        self.shp_wy = (nz, ny + 1, nx)
        self.shp_wz = (nz + 1, ny, nx)
        self.off_wy = int(np.prod(self.shp_wx))
        self.off_wz = self.off_wy + int(np.prod(self.shp_wy))
        self.nfaces = self.off_wz + int(np.prod(self.shp_wz))
        # edge lattices
        self.shp_xy = (nz, ny + 1, nx + 1)
        self.shp_xz = (nz + 1, ny, nx + 1)
        self.shp_yz = (nz + 1, ny + 1, nx)
        N = nx * ny * nz
        self.N = N
        self.row_exx, self.row_eyy, self.row_ezz = 0, N, 2 * N
        self.row_xy = 3 * N
        self.row_xz = self.row_xy + int(np.prod(self.shp_xy))
        self.row_yz = self.row_xz + int(np.prod(self.shp_xz))
        self.nrows = self.row_yz + int(np.prod(self.shp_yz))
        self._build_B()
        self._build_D()
        free = np.ones(self.nfaces, dtype=bool)
        wx = free[:self.off_wy].reshape(self.shp_wx)
        wx[:, :, 0] = False
        wx[:, :, nx] = False
        wy = free[self.off_wy:self.off_wz].reshape(self.shp_wy)
        wy[:, 0, :] = False
        wy[:, ny, :] = False
        wz = free[self.off_wz:].reshape(self.shp_wz)
        wz[0, :, :] = False
        wz[nz, :, :] = False
        self.free = free
        self.Bf = self.B[:, free]
        self.A = (self.Bf.T @ self.D @ self.Bf).tocsc()

    # ------------------------------------------------------------ strains
    def _fid(self, comp, k, j, i):
        if comp == 0:
            return np.ravel_multi_index((k, j, i), self.shp_wx)
        if comp == 1:
            return self.off_wy + np.ravel_multi_index((k, j, i), self.shp_wy)
        return self.off_wz + np.ravel_multi_index((k, j, i), self.shp_wz)

    def _build_B(self):
        nx, ny, nz = self.n
        rows, cols, vals = [], [], []

        def add(r, c, v):
            rows.append(np.asarray(r).ravel())
            cols.append(np.asarray(c).ravel())
            vals.append(np.broadcast_to(np.asarray(v, dtype=np.float64), np.asarray(r).shape).ravel())

        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        cell = np.ravel_multi_index((k, j, i), (nz, ny, nx))
        # e_xx = wx(i+1) - wx(i), etc.
        add(self.row_exx + cell, self._fid(0, k, j, i + 1), 1.0)
        add(self.row_exx + cell, self._fid(0, k, j, i), -1.0)
        add(self.row_eyy + cell, self._fid(1, k, j + 1, i), 1.0)
        add(self.row_eyy + cell, self._fid(1, k, j, i), -1.0)
        add(self.row_ezz + cell, self._fid(2, k + 1, j, i), 1.0)
        add(self.row_ezz + cell, self._fid(2, k, j, i), -1.0)

        # tensor shear strain on an edge: 1/2 (d_a w_b + d_b w_a); a derivative
        # of a component tangential to the boundary at an edge position q of
        # 0..n is (w(q+1/2) - w(q-1/2)) inside and the half-spacing difference
        # to the boundary value 0 at q = 0 and q = n (see _tang_terms).
        # xy edges (k, j, i), j in 0..ny, i in 0..nx
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        r = self.row_xy + np.ravel_multi_index((k, j, i), self.shp_xy)
        self._tang_xy(add, r, k, j, i)
        # xz edges (k, j, i), k in 0..nz, i in 0..nx
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx + 1), indexing="ij")
        r = self.row_xz + np.ravel_multi_index((k, j, i), self.shp_xz)
        self._tang_xz(add, r, k, j, i)
        # yz edges (k, j, i), k in 0..nz, j in 0..ny
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx), indexing="ij")
        r = self.row_yz + np.ravel_multi_index((k, j, i), self.shp_yz)
        self._tang_yz(add, r, k, j, i)

        self.B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.nrows, self.nfaces))

    @staticmethod
    def _tang_terms(q, n):
        """(mask, node offset, coefficient) triples of a tangential derivative
        times 1/2, evaluated at integer position q in 0..n."""
        inner = (q > 0) & (q < n)
        return [(inner, 0, 0.5), (inner, -1, -0.5), (q == 0, 0, 1.0), (q == n, -1, -1.0)]

    def _tang_xy(self, add, r, k, j, i):
        nx, ny, nz = self.n
        # d wx / dy: wx nodes at (i, j' + 1/2), j' in 0..ny-1
        for m, off, c in self._tang_terms(j, ny):
            add(r[m], self._fid(0, k[m], j[m] + off, i[m]), c)
        # d wy / dx: wy nodes at (i' + 1/2, j)
        for m, off, c in self._tang_terms(i, nx):
            add(r[m], self._fid(1, k[m], j[m], i[m] + off), c)

    def _tang_xz(self, add, r, k, j, i):
        nx, ny, nz = self.n
        for m, off, c in self._tang_terms(k, nz):     # d wx / dz
            add(r[m], self._fid(0, k[m] + off, j[m], i[m]), c)
        for m, off, c in self._tang_terms(i, nx):     # d wz / dx
            add(r[m], self._fid(2, k[m], j[m], i[m] + off), c)

    def _tang_yz(self, add, r, k, j, i):
        nx, ny, nz = self.n
        for m, off, c in self._tang_terms(k, nz):     # d wy / dz
            add(r[m], self._fid(1, k[m] + off, j[m], i[m]), c)
        for m, off, c in self._tang_terms(j, ny):     # d wz / dy
            add(r[m], self._fid(2, k[m], j[m] + off, i[m]), c)

    # ------------------------------------------------------------ moduli
    def _edge_G(self, shp, axes):
        """mean G of the existing cells adjacent to each edge; axes are the two
        grid directions (0 = z, 1 = y, 2 = x) transverse to the edge."""
        G = self.G
        pad = [(0, 0)] * 3
        for a in axes:
            pad[a] = (1, 1)
        Gp = np.pad(G, pad)
        Ep = np.pad(np.ones_like(G), pad)
        s = np.zeros(shp)
        c = np.zeros(shp)
        a0, a1 = axes
        for d0 in (0, 1):
            for d1 in (0, 1):
                sl = [slice(None)] * 3
                sl[a0] = slice(d0, d0 + shp[a0])
                sl[a1] = slice(d1, d1 + shp[a1])
                s += Gp[tuple(sl)]
                c += Ep[tuple(sl)]
        return s / c

    def _edge_weight(self, shp, axes):
        w = np.ones(shp)
        for a in axes:
            n = shp[a] - 1
            sl = [slice(None)] * 3
            sl[a] = 0
            w[tuple(sl)] *= 0.5
            sl[a] = n
            w[tuple(sl)] *= 0.5
        return w

    def _boundary_mask(self, shp, axes):
        m = np.zeros(shp, dtype=bool)
        for a in axes:
            sl = [slice(None)] * 3
            sl[a] = 0
            m[tuple(sl)] = True
            sl[a] = shp[a] - 1
            m[tuple(sl)] = True
        return m

    def _free_mask(self, name, shp, axes):
        """Edges of family `name` whose shear stress vanishes: none under
        uniform kinematic conditions (bc 0); every boundary edge under rollers
        (bc 1); under the simple shear tests of Appendix A.2 (bc 2, 3, 4: the
        yz, xz, xy components) the sheared family keeps its edges on the
        driven face pair (z, z, y faces) and is free only on the lateral faces
        of the other axis (y, x, x), every other family is free on the whole
        boundary.  Array axes: 0 = z, 1 = y, 2 = x."""
        if self.bc == 0:
            return np.zeros(shp, dtype=bool)
        lateral = {2: ("yz", 1), 3: ("xz", 2), 4: ("xy", 2)}.get(self.bc)
        if lateral is not None and lateral[0] == name:
            return self._boundary_mask(shp, (lateral[1],))
        return self._boundary_mask(shp, axes)

    def _build_D(self):
        K, G = self.K.ravel(), self.G.ravel()
        lam = K - 2.0 / 3.0 * G
        N = self.N
        blocks = []
        # cell block per voxel: lambda 1 1^T + 2 G I on (e_xx, e_yy, e_zz)
        r, c, v = [], [], []
        for a in range(3):
            for b in range(3):
                r.append(a * N + np.arange(N))
                c.append(b * N + np.arange(N))
                v.append(lam + (2.0 * G if a == b else 0.0))
        Dc = sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=(3 * N, 3 * N))
        self.Ge = {}
        self.omega = {}
        dd = []
        for name, shp, axes in (("xy", self.shp_xy, (1, 2)), ("xz", self.shp_xz, (0, 2)),
                                ("yz", self.shp_yz, (0, 1))):
            Ge = self._edge_G(shp, axes)
            om = self._edge_weight(shp, axes)
            Ge = np.where(self._free_mask(name, shp, axes), 0.0, Ge)   # traction-free edges
            self.Ge[name], self.omega[name] = Ge, om
            dd.append((4.0 * Ge * om).ravel())
        blocks = [Dc, sp.diags(np.concatenate(dd))]
        self.D = sp.block_diag(blocks, format="csr")

    # ------------------------------------------------------------ loads
    def sbar(self, e6):
        """strain vector of the affine field v = ebar . x (exact on the grid)."""
        e6 = np.asarray(e6, dtype=np.float64)
        s = np.zeros(self.nrows)
        N = self.N
        s[0:N] = e6[0]
        s[N:2 * N] = e6[1]
        s[2 * N:3 * N] = e6[2]
        s[self.row_xy:self.row_xz] = 0.5 * e6[5]
        s[self.row_xz:self.row_yz] = 0.5 * e6[4]
        s[self.row_yz:] = 0.5 * e6[3]
        return s

    def rhs(self, e6):
        return -(self.Bf.T @ (self.D @ self.sbar(e6)))

    def full_w(self, wf):
        w = np.zeros(self.nfaces)
        w[self.free] = wf
        return w

    def strains(self, w_full, e6):
        return self.B @ w_full + self.sbar(e6)

    def solve(self, e6, method="direct", tol=1e-13):
        b = self.rhs(e6)
        if not np.any(b):
            return np.zeros(self.A.shape[0])
        if method == "direct":
            # one sparse LU of A serves every load case
            if getattr(self, "_lu", None) is None:
                self._lu = spla.splu(sp.csc_matrix(self.A))
            return self._lu.solve(b)
        x, info = spla.cg(self.A, b, rtol=tol, maxiter=20000)
        if info != 0:
            raise RuntimeError(f"cg did not converge ({info})")
        return x

    # ------------------------------------------------------------ outputs
    def stresses(self, s):
        """(cells sigma_xx, sigma_yy, sigma_zz, edges tau_xy, tau_xz, tau_yz)"""
        N = self.N
        exx, eyy, ezz = s[:N], s[N:2 * N], s[2 * N:3 * N]
        K, G = self.K.ravel(), self.G.ravel()
        lam = K - 2.0 / 3.0 * G
        tr = exx + eyy + ezz
        out = {
            "sxx": lam * tr + 2 * G * exx,
            "syy": lam * tr + 2 * G * eyy,
            "szz": lam * tr + 2 * G * ezz,
            "xy": 2 * self.Ge["xy"].ravel() * s[self.row_xy:self.row_xz],
            "xz": 2 * self.Ge["xz"].ravel() * s[self.row_xz:self.row_yz],
            "yz": 2 * self.Ge["yz"].ravel() * s[self.row_yz:],
        }
        return out

    def averages(self, s):
        """<sigma>, <eps> in Voigt order (engineering shear strain)."""
        st = self.stresses(s)
        V = float(self.N)
        N = self.N
        om = {k: v.ravel() for k, v in self.omega.items()}
        sig = np.array([st["sxx"].sum(), st["syy"].sum(), st["szz"].sum(),
                        (om["yz"] * st["yz"]).sum(), (om["xz"] * st["xz"]).sum(),
                        (om["xy"] * st["xy"]).sum()]) / V
        eps = np.array([s[:N].sum(), s[N:2 * N].sum(), s[2 * N:3 * N].sum(),
                        2 * (om["yz"] * s[self.row_yz:]).sum(),
                        2 * (om["xz"] * s[self.row_xz:self.row_yz]).sum(),
                        2 * (om["xy"] * s[self.row_xy:self.row_xz]).sum()]) / V
        return sig, eps

    def energy_form(self, strains_list):
        V = float(self.N)
        n = len(strains_list)
        C = np.zeros((n, n))
        Ds = [self.D @ s for s in strains_list]
        for a in range(n):
            for b in range(n):
                C[a, b] = strains_list[a] @ Ds[b] / V
        return C

    def residual(self, w_full, e6):
        """B_f^T D s(w): the negative stress divergence at the free nodes."""
        return self.Bf.T @ (self.D @ self.strains(w_full, e6))

    # ------------------------------------------------------------ gradient
    def grad_C(self, strains_list, Wt):
        """dJ/dK_c and dJ/dG_c for J = sum_mn W_mn C_mn (energy form, at the
        equilibrium fields; the adjoint fields are the forward fields because
        A is symmetric).  Returns arrays shaped like K."""
        N = self.N
        nz, ny, nx = self.K.shape
        V = float(N)
        Ws = 0.5 * (np.asarray(Wt) + np.asarray(Wt).T)
        n = len(strains_list)
        dK = np.zeros(N)
        dG = np.zeros(N)
        ex = [s[:N] for s in strains_list]
        ey = [s[N:2 * N] for s in strains_list]
        ez = [s[2 * N:3 * N] for s in strains_list]
        tr = [ex[m] + ey[m] + ez[m] for m in range(n)]
        dev = [(ex[m] - tr[m] / 3, ey[m] - tr[m] / 3, ez[m] - tr[m] / 3) for m in range(n)]
        for a in range(n):
            for b in range(n):
                w = Ws[a, b]
                if w == 0.0:
                    continue
                dK += w * tr[a] * tr[b]
                dG += w * 2.0 * (dev[a][0] * dev[b][0] + dev[a][1] * dev[b][1] + dev[a][2] * dev[b][2])
        # edges: d/dG_c of sum_e omega_e 4 G_e e^a e^b with G_e = mean over the
        # n_e existing adjacent cells -> omega_e * 4 / n_e per adjacent cell
        for name, shp, axes, r0, r1 in (("xy", self.shp_xy, (1, 2), self.row_xy, self.row_xz),
                                        ("xz", self.shp_xz, (0, 2), self.row_xz, self.row_yz),
                                        ("yz", self.shp_yz, (0, 1), self.row_yz, self.nrows)):
            q = np.zeros(shp)
            for a in range(n):
                for b in range(n):
                    w = Ws[a, b]
                    if w == 0.0:
                        continue
                    q += w * (strains_list[a][r0:r1] * strains_list[b][r0:r1]).reshape(shp)
            cnt = np.zeros(shp)
            a0, a1 = axes
            ones = np.ones((nz, ny, nx))
            pad = [(0, 0)] * 3
            pad[a0] = (1, 1)
            pad[a1] = (1, 1)
            Ep = np.pad(ones, pad)
            for d0 in (0, 1):
                for d1 in (0, 1):
                    sl = [slice(None)] * 3
                    sl[a0] = slice(d0, d0 + shp[a0])
                    sl[a1] = slice(d1, d1 + shp[a1])
                    cnt += Ep[tuple(sl)]
            fac = 4.0 * self.omega[name] / cnt
            fac = np.where(self._free_mask(name, shp, axes), 0.0, fac)
            contrib = q * fac
            # scatter each edge's share to its existing adjacent cells
            cp = np.zeros([s + 2 if ax in axes else s for ax, s in enumerate((nz, ny, nx))])
            for d0 in (0, 1):
                for d1 in (0, 1):
                    sl = [slice(None)] * 3
                    sl[a0] = slice(d0, d0 + shp[a0])
                    sl[a1] = slice(d1, d1 + shp[a1])
                    cp[tuple(sl)] += contrib
            inner = [slice(1, -1) if ax in axes else slice(None) for ax in range(3)]
            dG += cp[tuple(inner)].ravel()
        return (dK / V).reshape(self.K.shape), (dG / V).reshape(self.K.shape)


def solve_all(K, G, loads=None, bc=0, method="direct"):
    """C (average form and energy form), strains and w for every load case."""
    op = Operator(K, G, bc=bc)
    loads = np.eye(6) if loads is None else np.asarray(loads, dtype=np.float64)
    strains, sigs, epss, ws = [], [], [], []
    for e6 in loads:
        wf = op.solve(e6, method=method)
        wfull = op.full_w(wf)
        s = op.strains(wfull, e6)
        sig, eps = op.averages(s)
        strains.append(s)
        sigs.append(sig)
        epss.append(eps)
        ws.append(wfull)
    S = np.stack(sigs, axis=1)
    E = np.stack(epss, axis=1)
    out = {"op": op, "S": S, "E": E, "strains": strains, "w": ws}
    if loads.shape[0] == 6:
        out["C"] = S @ np.linalg.inv(E)
        out["C_energy"] = op.energy_form(strains)
    return out
