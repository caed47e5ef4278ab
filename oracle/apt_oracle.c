/*
 * ORACLE -- test infrastructure only.  Plain, slow, FP64 CPU implementation of
 * the accelerated pseudo-transient (APT) solve of quasi-static elasticity on a
 * staggered voxel grid.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * What it computes (paper: Alkhimenkov, "Digital rock physics: calculation of
 * effective elastic properties of heterogeneous materials using GPUs"):
 *
 *   stress split            sigma_ij = -p delta_ij + tau_ij          (Eq. A2ssP, first)
 *   momentum (pseudo-time)  rho~ dv_i/dt~ = d_j(-p delta_ij + tau_ij) (Eq. 11111)
 *   pressure relaxation     (1/K~) dp/dt~ + p/(K dt) = -div v         (Eq. A2ssP, second)
 *   deviator relaxation     (1/2G~) dtau/dt~ + tau/(2G dt)
 *                             = (1/2)(d_i v_j + d_j v_i) - (1/3) delta_ij div v
 *                                                                     (Eq. A23ssP2; mu_s dropped)
 *   each pseudo-time step updates the stresses, then the velocities (Sec. 3.2).
 *
 * Numerical parameters (Sec. 3.1, Eqs. PT1_1t2 - PT1_1t31333AB) with the
 * numerical moduli equal to the material ones, K~ = K and G~ = G, taken at
 * every stress point (cell or edge) from its own modulus:
 *   dt~ = C~ dx St dt / Lx                     (from dt~ = C~ dx / Vp~, St = Lx/(Vp~ dt))
 *   K~ dt~ = K dt~,  G~ dt~ = G dt~            (stress points)
 *   dt~/rho~ = C~ dx Lx / (St H~ dt)           (velocity nodes, Eq. PT1_1t31222)
 * where H~ at a velocity node is the P-wave modulus that bounds the node's
 * stencil: one twelfth of the sum, over the stress points the node reads, of
 * the absolute row sums of their numerical stress-rate stencils
 * (2 H + 4 |lambda| for a cell, 4 G_e for an edge).  For a homogeneous body
 * this is exactly H~ = K~ + 4/3 G~ (when lambda >= 0), so the formulas reduce
 * to the paper's scalar ones; for a heterogeneous body the explicit update
 * stays within the 3-D stability limit C~ <= 1/sqrt(3) everywhere.
 *
 * Discretisation (Sec. 3.3, staggered grid of Virieux type), unit voxel, grid
 * of nx*ny*nz cells; every field is stored on the (nx+1)*(ny+1)*(nz+1) index
 * grid, x fastest:
 *   cell (i,j,k)         : p, tau_xx, tau_yy   (tau_zz = -tau_xx - tau_yy)
 *   x-face (i,j,k), i<=nx: w_x  at (i, j+1/2, k+1/2)
 *   y-face (i,j,k), j<=ny: w_y  at (i+1/2, j, k+1/2)
 *   z-face (i,j,k), k<=nz: w_z  at (i+1/2, j+1/2, k)
 *   xy-edge i<=nx, j<=ny : tau_xy at (i, j, k+1/2)
 *   xz-edge i<=nx, k<=nz : tau_xz at (i, j+1/2, k)
 *   yz-edge j<=ny, k<=nz : tau_yz at (i+1/2, j, k)
 * The velocity is v = ebar.x + w; only the fluctuation w is stored and the
 * macroscopic part enters every strain rate exactly.  Boundary normal
 * velocities are Dirichlet (w = 0).  With bc = 0 (kinematic uniform boundary
 * conditions, v = ebar.x on the whole boundary) a tangential derivative at a
 * boundary edge is the half-spacing difference to the boundary value w = 0.
 * With bc = 1 (rollers: normal velocity prescribed, tangential traction
 * free, Appendix A.1) all boundary-edge shear stresses are zero.  With
 * bc = 2, 3, 4 (the simple shear tests of Appendix A.2 for the yz, xz and xy
 * components) the sheared component is prescribed on its driven face pair
 * (v_y on the z faces, v_x on the z faces, v_x on the y faces): those edges
 * keep the kinematic treatment, every other boundary edge is free.
 * The edge shear modulus is the arithmetic mean of the existing adjacent
 * cells.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    int bc;          /* 0: uniform kinematic, 1: rollers, 2-4: simple shear yz, xz, xy */
    double dtt;      /* pseudo-time step dt~ */
    double cdr;      /* C~ dx Lx / (St dt): dt~/rho~ = cdr / H~ at a velocity node */
    double dt;       /* physical step dt of the relaxation terms */
} apt_par;

#define NF 9
enum { F_P = 0, F_TXX, F_TYY, F_TXY, F_TXZ, F_TYZ, F_WX, F_WY, F_WZ };

static inline size_t ix(const apt_par* g, int i, int j, int k)
{
    return ((size_t)k * (size_t)(g->ny + 1) + (size_t)j) * (size_t)(g->nx + 1) + (size_t)i;
}
static inline size_t ic(const apt_par* g, int i, int j, int k)
{
    return ((size_t)k * (size_t)g->ny + (size_t)j) * (size_t)g->nx + (size_t)i;
}
static inline size_t nidx(const apt_par* g)
{
    return (size_t)(g->nx + 1) * (size_t)(g->ny + 1) * (size_t)(g->nz + 1);
}

/* macroscopic strain tensor from Voigt (xx, yy, zz, yz, xz, xy), engineering shear */
typedef struct { double xx, yy, zz, yz, xz, xy; } tens;
static tens from_voigt(const double e[6])
{
    tens t = { e[0], e[1], e[2], 0.5 * e[3], 0.5 * e[4], 0.5 * e[5] };
    return t;
}

/* ------------------------------------------------------------- strain rates */
static void cell_rates(const apt_par* g, double* const* f, tens eb, int i, int j, int k,
                       double* exx, double* eyy, double* ezz)
{
    const double* wx = f[F_WX]; const double* wy = f[F_WY]; const double* wz = f[F_WZ];
    *exx = wx[ix(g, i + 1, j, k)] - wx[ix(g, i, j, k)] + eb.xx;
    *eyy = wy[ix(g, i, j + 1, k)] - wy[ix(g, i, j, k)] + eb.yy;
    *ezz = wz[ix(g, i, j, k + 1)] - wz[ix(g, i, j, k)] + eb.zz;
}

/* derivative along a direction of a velocity component that is tangential at
 * the boundaries of that direction: nodes sit at half-integer positions
 * 0..n-1 (stored at index m), the derivative is wanted at the integer
 * position q in 0..n.  lo = value at node q-1, hi = value at node q. */
static double tangential_diff(int q, int n, double lo, double hi)
{
    if (q == 0) return 2.0 * hi;          /* (w(1/2) - 0) / (1/2) */
    if (q == n) return -2.0 * lo;         /* (0 - w(n-1/2)) / (1/2) */
    return hi - lo;
}

static double rate_xy(const apt_par* g, double* const* f, tens eb, int i, int j, int k)
{
    const double* wx = f[F_WX]; const double* wy = f[F_WY];
    double lo = j > 0 ? wx[ix(g, i, j - 1, k)] : 0.0;
    double hi = j < g->ny ? wx[ix(g, i, j, k)] : 0.0;
    double dwx_dy = tangential_diff(j, g->ny, lo, hi);
    lo = i > 0 ? wy[ix(g, i - 1, j, k)] : 0.0;
    hi = i < g->nx ? wy[ix(g, i, j, k)] : 0.0;
    double dwy_dx = tangential_diff(i, g->nx, lo, hi);
    return 0.5 * (dwx_dy + dwy_dx) + eb.xy;
}

static double rate_xz(const apt_par* g, double* const* f, tens eb, int i, int j, int k)
{
    const double* wx = f[F_WX]; const double* wz = f[F_WZ];
    double lo = k > 0 ? wx[ix(g, i, j, k - 1)] : 0.0;
    double hi = k < g->nz ? wx[ix(g, i, j, k)] : 0.0;
    double dwx_dz = tangential_diff(k, g->nz, lo, hi);
    lo = i > 0 ? wz[ix(g, i - 1, j, k)] : 0.0;
    hi = i < g->nx ? wz[ix(g, i, j, k)] : 0.0;
    double dwz_dx = tangential_diff(i, g->nx, lo, hi);
    return 0.5 * (dwx_dz + dwz_dx) + eb.xz;
}

static double rate_yz(const apt_par* g, double* const* f, tens eb, int i, int j, int k)
{
    const double* wy = f[F_WY]; const double* wz = f[F_WZ];
    double lo = k > 0 ? wy[ix(g, i, j, k - 1)] : 0.0;
    double hi = k < g->nz ? wy[ix(g, i, j, k)] : 0.0;
    double dwy_dz = tangential_diff(k, g->nz, lo, hi);
    lo = j > 0 ? wz[ix(g, i, j - 1, k)] : 0.0;
    hi = j < g->ny ? wz[ix(g, i, j, k)] : 0.0;
    double dwz_dy = tangential_diff(j, g->ny, lo, hi);
    return 0.5 * (dwy_dz + dwz_dy) + eb.yz;
}

/* arithmetic mean of G over the existing cells among the 2x2 cells that share
 * an edge: cells (a0|a1, b0|b1) in the two directions across the edge */
static double edge_modulus(const apt_par* g, const double* G, int dir, int i, int j, int k)
{
    double s = 0.0; int n = 0;
    for (int da = -1; da <= 0; ++da)
        for (int db = -1; db <= 0; ++db) {
            int ci = i, cj = j, ck = k;
            if (dir == 0) { ci = i + da; cj = j + db; }        /* xy edge: x,y neighbours */
            else if (dir == 1) { ci = i + da; ck = k + db; }   /* xz edge */
            else { cj = j + da; ck = k + db; }                 /* yz edge */
            if (ci < 0 || cj < 0 || ck < 0 || ci >= g->nx || cj >= g->ny || ck >= g->nz) continue;
            s += G[ic(g, ci, cj, ck)];
            ++n;
        }
    return s / (double)n;
}

/* Is the shear stress of this boundary edge held at zero?  Rollers free
 * every boundary edge; a simple shear test frees all but the edges of its
 * sheared component on its driven face pair (Appendix A.2), where that pair
 * does not meet a lateral face. */
static int stress_free_xy(const apt_par* g, int i, int j)
{
    int on_x = i == 0 || i == g->nx, on_y = j == 0 || j == g->ny;
    if (g->bc == 0) return 0;
    if (g->bc == 4) return on_x;      /* xy shear, v_x driven on the y faces */
    return on_x || on_y;
}
static int stress_free_xz(const apt_par* g, int i, int k)
{
    int on_x = i == 0 || i == g->nx, on_z = k == 0 || k == g->nz;
    if (g->bc == 0) return 0;
    if (g->bc == 3) return on_x;      /* xz shear, v_x driven on the z faces */
    return on_x || on_z;
}
static int stress_free_yz(const apt_par* g, int j, int k)
{
    int on_y = j == 0 || j == g->ny, on_z = k == 0 || k == g->nz;
    if (g->bc == 0) return 0;
    if (g->bc == 2) return on_y;      /* yz shear, v_y driven on the z faces */
    return on_y || on_z;
}

/* --------------------------------------------------------------- init (w=0) */
/* Stresses of the elastic state at w = 0: sigma = C(x):ebar.  A homogeneous
 * body is then a fixed point of the iteration from the first step. */
void apt_init(const apt_par* g, const double* K, const double* G, const double e6[6], double* state)
{
    size_t n = nidx(g);
    double* f[NF];
    for (int q = 0; q < NF; ++q) f[q] = state + (size_t)q * n;
    memset(state, 0, sizeof(double) * n * NF);
    tens eb = from_voigt(e6);
    double tr = eb.xx + eb.yy + eb.zz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= g->nz; ++k)
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i) {
                size_t q = ix(g, i, j, k);
                if (i < g->nx && j < g->ny && k < g->nz) {
                    double Kc = K[ic(g, i, j, k)], Gc = G[ic(g, i, j, k)];
                    f[F_P][q] = -Kc * tr;
                    f[F_TXX][q] = 2.0 * Gc * (eb.xx - tr / 3.0);
                    f[F_TYY][q] = 2.0 * Gc * (eb.yy - tr / 3.0);
                }
                if (k < g->nz)
                    f[F_TXY][q] = stress_free_xy(g, i, j) ? 0.0
                                 : 2.0 * edge_modulus(g, G, 0, i, j, k) * eb.xy;
                if (j < g->ny)
                    f[F_TXZ][q] = stress_free_xz(g, i, k) ? 0.0
                                 : 2.0 * edge_modulus(g, G, 1, i, j, k) * eb.xz;
                if (i < g->nx)
                    f[F_TYZ][q] = stress_free_yz(g, j, k) ? 0.0
                                 : 2.0 * edge_modulus(g, G, 2, i, j, k) * eb.yz;
            }
}

/* ------------------------------------------------------------ stress update */
/* Backward-Euler in pseudo time of the relaxation equations, solved for the
 * new stress: (x_new - x_old)/(M~ dt~) + x_new/(M dt) = rate. */
static double relax(double old, double Mdt_tilde, double Mloc_dt, double rate)
{
    return (old / Mdt_tilde + rate) / (1.0 / Mdt_tilde + 1.0 / Mloc_dt);
}

/* the stress update of the index planes k0 <= k < k1 (all planes: 0, nz+1) */
static void stress_update_planes(const apt_par* g, const double* K, const double* G, const double e6[6],
                                 double* state, int k0, int k1)
{
    size_t n = nidx(g);
    double* f[NF];
    for (int q = 0; q < NF; ++q) f[q] = state + (size_t)q * n;
    tens eb = from_voigt(e6);
    const double dt = g->dt;
    /* every stress at step n+1 depends on velocities at step n only, so the
     * update can be done in place */
#pragma omp parallel for schedule(static)
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i) {
                size_t q = ix(g, i, j, k);
                if (i < g->nx && j < g->ny && k < g->nz) {
                    double exx, eyy, ezz;
                    cell_rates(g, f, eb, i, j, k, &exx, &eyy, &ezz);
                    double div = exx + eyy + ezz;
                    double Kc = K[ic(g, i, j, k)], Gc = G[ic(g, i, j, k)];
                    /* (1/K~) dp/dt~ + p/(K dt) = -div v, with K~ = K */
                    f[F_P][q] = relax(f[F_P][q], Kc * g->dtt, Kc * dt, -div);
                    /* (1/2G~) dtau/dt~ + tau/(2G dt) = e_ii - div/3, with G~ = G */
                    f[F_TXX][q] = relax(f[F_TXX][q], 2.0 * Gc * g->dtt, 2.0 * Gc * dt, exx - div / 3.0);
                    f[F_TYY][q] = relax(f[F_TYY][q], 2.0 * Gc * g->dtt, 2.0 * Gc * dt, eyy - div / 3.0);
                }
                if (k < g->nz) {
                    if (stress_free_xy(g, i, j)) f[F_TXY][q] = 0.0;
                    else {
                        double Ge = edge_modulus(g, G, 0, i, j, k);
                        f[F_TXY][q] = relax(f[F_TXY][q], 2.0 * Ge * g->dtt, 2.0 * Ge * dt,
                                             rate_xy(g, f, eb, i, j, k));
                    }
                }
                if (j < g->ny) {
                    if (stress_free_xz(g, i, k)) f[F_TXZ][q] = 0.0;
                    else {
                        double Ge = edge_modulus(g, G, 1, i, j, k);
                        f[F_TXZ][q] = relax(f[F_TXZ][q], 2.0 * Ge * g->dtt, 2.0 * Ge * dt,
                                             rate_xz(g, f, eb, i, j, k));
                    }
                }
                if (i < g->nx) {
                    if (stress_free_yz(g, j, k)) f[F_TYZ][q] = 0.0;
                    else {
                        double Ge = edge_modulus(g, G, 2, i, j, k);
                        f[F_TYZ][q] = relax(f[F_TYZ][q], 2.0 * Ge * g->dtt, 2.0 * Ge * dt,
                                             rate_yz(g, f, eb, i, j, k));
                    }
                }
            }
}

void apt_stress_update(const apt_par* g, const double* K, const double* G, const double e6[6], double* state)
{
    stress_update_planes(g, K, G, e6, state, 0, g->nz + 1);
}

/* ------------------------------------------------------- stress divergence */
/* Divergence of sigma = -p I + tau at the three velocity nodes of index
 * (i,j,k); s = {p, tau_xx, tau_yy, tau_xy, tau_xz, tau_yz}. */
static double sxx(const apt_par* g, double* const* s, int i, int j, int k)
{ size_t q = ix(g, i, j, k); return -s[0][q] + s[1][q]; }
static double syy(const apt_par* g, double* const* s, int i, int j, int k)
{ size_t q = ix(g, i, j, k); return -s[0][q] + s[2][q]; }
static double szz(const apt_par* g, double* const* s, int i, int j, int k)
{ size_t q = ix(g, i, j, k); return -s[0][q] - s[1][q] - s[2][q]; }

static double div_x(const apt_par* g, double* const* s, int i, int j, int k)
{
    return (sxx(g, s, i, j, k) - sxx(g, s, i - 1, j, k))
         + (s[3][ix(g, i, j + 1, k)] - s[3][ix(g, i, j, k)])
         + (s[4][ix(g, i, j, k + 1)] - s[4][ix(g, i, j, k)]);
}
static double div_y(const apt_par* g, double* const* s, int i, int j, int k)
{
    return (s[3][ix(g, i + 1, j, k)] - s[3][ix(g, i, j, k)])
         + (syy(g, s, i, j, k) - syy(g, s, i, j - 1, k))
         + (s[5][ix(g, i, j, k + 1)] - s[5][ix(g, i, j, k)]);
}
static double div_z(const apt_par* g, double* const* s, int i, int j, int k)
{
    return (s[4][ix(g, i + 1, j, k)] - s[4][ix(g, i, j, k)])
         + (s[5][ix(g, i, j + 1, k)] - s[5][ix(g, i, j, k)])
         + (szz(g, s, i, j, k) - szz(g, s, i, j, k - 1));
}

/* ------------------------------------------------- pseudo P-wave modulus */
/* row-sum bound of the stress-rate stencil of a cell: 2 H + 4 |lambda| */
static double cell_rowsum(const apt_par* g, const double* K, const double* G, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) return 0.0;
    double Kc = K[ic(g, i, j, k)], Gc = G[ic(g, i, j, k)];
    return 2.0 * (Kc + 4.0 / 3.0 * Gc) + 4.0 * fabs(Kc - 2.0 / 3.0 * Gc);
}

/* H~ at the velocity node of component c (0 = x, 1 = y, 2 = z) and index
 * (i,j,k): one twelfth of the summed row bounds of the two cells and four
 * edges whose stresses enter the node's update (an edge: 4 G_e). */
static double node_modulus(const apt_par* g, const double* K, const double* G, int c, int i, int j, int k)
{
    double r;
    if (c == 0)
        r = cell_rowsum(g, K, G, i - 1, j, k) + cell_rowsum(g, K, G, i, j, k)
          + 4.0 * (edge_modulus(g, G, 0, i, j, k) + edge_modulus(g, G, 0, i, j + 1, k)
                   + edge_modulus(g, G, 1, i, j, k) + edge_modulus(g, G, 1, i, j, k + 1));
    else if (c == 1)
        r = cell_rowsum(g, K, G, i, j - 1, k) + cell_rowsum(g, K, G, i, j, k)
          + 4.0 * (edge_modulus(g, G, 0, i, j, k) + edge_modulus(g, G, 0, i + 1, j, k)
                   + edge_modulus(g, G, 2, i, j, k) + edge_modulus(g, G, 2, i, j, k + 1));
    else
        r = cell_rowsum(g, K, G, i, j, k - 1) + cell_rowsum(g, K, G, i, j, k)
          + 4.0 * (edge_modulus(g, G, 1, i, j, k) + edge_modulus(g, G, 1, i + 1, j, k)
                   + edge_modulus(g, G, 2, i, j, k) + edge_modulus(g, G, 2, i, j + 1, k));
    return r / 12.0;
}

/* ---------------------------------------------------------- velocity update */
/* H~ of every velocity node on the index grid (3 arrays; zero at Dirichlet
 * nodes).  It depends only on the moduli, so it is formed once per call. */
static double* node_moduli_alloc(const apt_par* g, const double* K, const double* G)
{
    size_t n = nidx(g);
    double* h = (double*)calloc(n * 3, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                if (i > 0) h[ix(g, i, j, k)] = node_modulus(g, K, G, 0, i, j, k);
                if (j > 0) h[n + ix(g, i, j, k)] = node_modulus(g, K, G, 1, i, j, k);
                if (k > 0) h[2 * n + ix(g, i, j, k)] = node_modulus(g, K, G, 2, i, j, k);
            }
    return h;
}

/* rho~ dv/dt~ = div sigma at every interior velocity node (boundary normal
 * velocities are Dirichlet and stay put); dt~/rho~ = cdr / H~ per node. */
/* the velocity update of the index planes k0 <= k < k1 (faces of planes
 * nz and above are Dirichlet or absent) */
static void velocity_update_planes(const apt_par* g, const double* Hn, double* state, int k0, int k1)
{
    size_t n = nidx(g);
    double* f[NF];
    for (int q = 0; q < NF; ++q) f[q] = state + (size_t)q * n;
    double* s[6] = { f[F_P], f[F_TXX], f[F_TYY], f[F_TXY], f[F_TXZ], f[F_TYZ] };
    if (k1 > g->nz) k1 = g->nz;
    /* the new velocity at a node depends only on stresses, so in place is fine */
#pragma omp parallel for schedule(static)
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t q = ix(g, i, j, k);
                if (i > 0) f[F_WX][q] += g->cdr / Hn[q] * div_x(g, s, i, j, k);
                if (j > 0) f[F_WY][q] += g->cdr / Hn[n + q] * div_y(g, s, i, j, k);
                if (k > 0) f[F_WZ][q] += g->cdr / Hn[2 * n + q] * div_z(g, s, i, j, k);
            }
}

void apt_velocity_update(const apt_par* g, const double* Hn, double* state)
{
    velocity_update_planes(g, Hn, state, 0, g->nz);
}

void apt_sweeps(const apt_par* g, const double* K, const double* G, const double e6[6],
                double* state, int nsweeps)
{
    double* Hn = node_moduli_alloc(g, K, G);
    for (int it = 0; it < nsweeps; ++it) {
        apt_stress_update(g, K, G, e6, state);
        apt_velocity_update(g, Hn, state);
    }
    free(Hn);
}

/* ----------------------------------------------------- elastic stress state */
/* sigma = C(x) : eps(ebar.x + w) with no memory terms: the explicit operator
 * whose equilibrium the iteration converges to.  s must hold 6 arrays. */
void apt_elastic_stress(const apt_par* g, const double* K, const double* G, const double e6[6],
                        const double* state, double* sout)
{
    size_t n = nidx(g);
    double* f[NF];
    for (int q = 0; q < NF; ++q) f[q] = (double*)state + (size_t)q * n;
    double* s[6];
    for (int q = 0; q < 6; ++q) s[q] = sout + (size_t)q * n;
    memset(sout, 0, sizeof(double) * n * 6);
    tens eb = from_voigt(e6);
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= g->nz; ++k)
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i) {
                size_t q = ix(g, i, j, k);
                if (i < g->nx && j < g->ny && k < g->nz) {
                    double exx, eyy, ezz;
                    cell_rates(g, f, eb, i, j, k, &exx, &eyy, &ezz);
                    double div = exx + eyy + ezz;
                    double Kc = K[ic(g, i, j, k)], Gc = G[ic(g, i, j, k)];
                    s[0][q] = -Kc * div;
                    s[1][q] = 2.0 * Gc * (exx - div / 3.0);
                    s[2][q] = 2.0 * Gc * (eyy - div / 3.0);
                }
                if (k < g->nz && !stress_free_xy(g, i, j))
                    s[3][q] = 2.0 * edge_modulus(g, G, 0, i, j, k) * rate_xy(g, f, eb, i, j, k);
                if (j < g->ny && !stress_free_xz(g, i, k))
                    s[4][q] = 2.0 * edge_modulus(g, G, 1, i, j, k) * rate_xz(g, f, eb, i, j, k);
                if (i < g->nx && !stress_free_yz(g, j, k))
                    s[5][q] = 2.0 * edge_modulus(g, G, 2, i, j, k) * rate_yz(g, f, eb, i, j, k);
            }
}

/* ---------------------------------------------------------------- residual */
/* Squared 2-norm of the divergence of the elastic stress over all interior
 * velocity nodes.  Summed per z-plane, then over planes in order, so the
 * result does not depend on the thread count. */
double apt_residual2(const apt_par* g, const double* K, const double* G, const double e6[6],
                     const double* state, double* scratch6)
{
    size_t n = nidx(g);
    apt_elastic_stress(g, K, G, e6, state, scratch6);
    double* s[6];
    for (int q = 0; q < 6; ++q) s[q] = scratch6 + (size_t)q * n;
    double* part = (double*)calloc((size_t)g->nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        double acc = 0.0;
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                if (i > 0) { double r = div_x(g, s, i, j, k); acc += r * r; }
                if (j > 0) { double r = div_y(g, s, i, j, k); acc += r * r; }
                if (k > 0) { double r = div_z(g, s, i, j, k); acc += r * r; }
            }
        part[k] = acc;
    }
    double tot = 0.0;
    for (int k = 0; k < g->nz; ++k) tot += part[k];
    free(part);
    return tot;
}

/* ----------------------------------------------------------- volume average */
/* <sigma> and <eps> (Eqs. BC:2, BC:1) in Voigt order with engineering shear
 * strain.  Cells carry weight 1; an edge carries the product over its two
 * transverse directions of 1/2 when it lies on the boundary in that
 * direction, else 1 (trapezoid rule on the edge lattice), so the weights of
 * every field sum to V = nx*ny*nz. */
void apt_average(const apt_par* g, const double e6[6], const double* state,
                 double sig[6], double eps[6])
{
    size_t n = nidx(g);
    double* f[NF];
    for (int q = 0; q < NF; ++q) f[q] = (double*)state + (size_t)q * n;
    tens eb = from_voigt(e6);
    double* part = (double*)calloc((size_t)(g->nz + 1) * 12, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= g->nz; ++k) {
        double a[12] = { 0 };
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i) {
                size_t q = ix(g, i, j, k);
                if (i < g->nx && j < g->ny && k < g->nz) {
                    double p = f[F_P][q], txx = f[F_TXX][q], tyy = f[F_TYY][q];
                    a[0] += -p + txx;
                    a[1] += -p + tyy;
                    a[2] += -p - txx - tyy;
                    double exx, eyy, ezz;
                    cell_rates(g, f, eb, i, j, k, &exx, &eyy, &ezz);
                    a[6] += exx; a[7] += eyy; a[8] += ezz;
                }
                double wi = (i == 0 || i == g->nx) ? 0.5 : 1.0;
                double wj = (j == 0 || j == g->ny) ? 0.5 : 1.0;
                double wk = (k == 0 || k == g->nz) ? 0.5 : 1.0;
                if (i < g->nx) { /* yz edge */
                    a[3] += wj * wk * f[F_TYZ][q];
                    a[9] += wj * wk * 2.0 * rate_yz(g, f, eb, i, j, k);
                }
                if (j < g->ny) { /* xz edge */
                    a[4] += wi * wk * f[F_TXZ][q];
                    a[10] += wi * wk * 2.0 * rate_xz(g, f, eb, i, j, k);
                }
                if (k < g->nz) { /* xy edge */
                    a[5] += wi * wj * f[F_TXY][q];
                    a[11] += wi * wj * 2.0 * rate_xy(g, f, eb, i, j, k);
                }
            }
        for (int c = 0; c < 12; ++c) part[(size_t)k * 12 + c] = a[c];
    }
    double V = (double)g->nx * (double)g->ny * (double)g->nz;
    for (int c = 0; c < 12; ++c) {
        double t = 0.0;
        for (int k = 0; k <= g->nz; ++k) t += part[(size_t)k * 12 + c];
        if (c < 6) sig[c] = t / V; else eps[c - 6] = t / V;
    }
    free(part);
}

/* -------------------------------------------------------------------- solve */
/* Pseudo-time loop (Sec. 3.2): check the relative residual
 * ||div sigma(w)|| / ||div sigma(0)|| every n_check sweeps and stop at
 * rel <= tol, at max_iter sweeps, or when the residual is not finite or has
 * grown beyond 1e10.  Returns 0 converged, 4 not converged, 5 diverged. */
int apt_solve(const apt_par* g, const double* K, const double* G, const double e6[6],
              double tol, int max_iter, int n_check, int init, double* state,
              double* hist, int hist_cap, int* n_hist, int* iters, double* rel_out,
              double* r0_out)
{
    size_t n = nidx(g);
    double* scratch = (double*)malloc(sizeof(double) * n * 6);
    if (init) apt_init(g, K, G, e6, state);
    double* zero = (double*)calloc(n * NF, sizeof(double));
    double r0 = sqrt(apt_residual2(g, K, G, e6, zero, scratch));
    free(zero);
    int it = 0, nh = 0, status;
    double rel = r0 > 0.0 ? sqrt(apt_residual2(g, K, G, e6, state, scratch)) / r0 : 0.0;
    if (nh < hist_cap) hist[nh++] = rel;
    while (rel > tol && it < max_iter && isfinite(rel) && rel <= 1e10) {
        int m = max_iter - it < n_check ? max_iter - it : n_check;
        apt_sweeps(g, K, G, e6, state, m);
        it += m;
        rel = sqrt(apt_residual2(g, K, G, e6, state, scratch)) / r0;
        if (nh < hist_cap) hist[nh++] = rel;
    }
    free(scratch);
    if (!isfinite(rel) || rel > 1e10) status = 5;
    else status = rel <= tol ? 0 : 4;
    *n_hist = nh;
    *iters = it;
    *rel_out = rel;
    *r0_out = r0;
    return status;
}

/* flat-argument wrappers for foreign-function callers */
static apt_par mkpar(int nx, int ny, int nz, int bc, double dtt, double cdr, double dt)
{
    apt_par g = { nx, ny, nz, bc, dtt, cdr, dt };
    return g;
}

int oracle_solve(int nx, int ny, int nz, int bc, double dtt, double cdr, double dt,
                 const double* K, const double* G, const double* e6, double tol, int max_iter,
                 int n_check, int init, double* state, double* hist, int hist_cap, int* n_hist,
                 int* iters, double* rel, double* r0)
{
    apt_par g = mkpar(nx, ny, nz, bc, dtt, cdr, dt);
    return apt_solve(&g, K, G, e6, tol, max_iter, n_check, init, state, hist, hist_cap, n_hist,
                     iters, rel, r0);
}

void oracle_init(int nx, int ny, int nz, int bc, const double* K, const double* G,
                 const double* e6, double* state)
{
    apt_par g = mkpar(nx, ny, nz, bc, 1.0, 1.0, 1.0);
    apt_init(&g, K, G, e6, state);
}

void oracle_sweeps(int nx, int ny, int nz, int bc, double dtt, double cdr, double dt,
                   const double* K, const double* G, const double* e6, double* state, int nsweeps)
{
    apt_par g = mkpar(nx, ny, nz, bc, dtt, cdr, dt);
    apt_sweeps(&g, K, G, e6, state, nsweeps);
}

double oracle_residual2(int nx, int ny, int nz, int bc, const double* K, const double* G,
                        const double* e6, const double* state)
{
    apt_par g = mkpar(nx, ny, nz, bc, 1.0, 1.0, 1.0);
    double* scratch = (double*)malloc(sizeof(double) * nidx(&g) * 6);
    double r = apt_residual2(&g, K, G, e6, state, scratch);
    free(scratch);
    return r;
}

void oracle_elastic_stress(int nx, int ny, int nz, int bc, const double* K, const double* G,
                           const double* e6, const double* state, double* sout)
{
    apt_par g = mkpar(nx, ny, nz, bc, 1.0, 1.0, 1.0);
    apt_elastic_stress(&g, K, G, e6, state, sout);
}

void oracle_average(int nx, int ny, int nz, const double* e6, const double* state,
                    double* sig, double* eps)
{
    apt_par g = mkpar(nx, ny, nz, 0, 1.0, 1.0, 1.0);
    apt_average(&g, e6, state, sig, eps);
}

/* One half of a sweep restricted to the index planes k0 <= k < k1: the
 * building blocks of a z-slab decomposition, where each rank updates only its
 * own planes and receives the neighbouring planes it reads between halves.
 * Every point is computed by the same code as in oracle_sweeps. */
void oracle_stress_planes(int nx, int ny, int nz, int bc, double dtt, double dt, const double* K,
                          const double* G, const double* e6, double* state, int k0, int k1)
{
    apt_par g = mkpar(nx, ny, nz, bc, dtt, 1.0, dt);
    stress_update_planes(&g, K, G, e6, state, k0, k1);
}

void oracle_velocity_planes(int nx, int ny, int nz, double cdr, const double* Hn, double* state, int k0,
                            int k1)
{
    apt_par g = mkpar(nx, ny, nz, 0, 1.0, cdr, 1.0);
    velocity_update_planes(&g, Hn, state, k0, k1);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* H~ of every interior velocity node, written on the index grid (3 arrays of
 * (nx+1)(ny+1)(nz+1), zero at Dirichlet nodes); test access only. */
void oracle_node_moduli(int nx, int ny, int nz, const double* K, const double* G, double* out)
{
    apt_par g = mkpar(nx, ny, nz, 0, 1.0, 1.0, 1.0);
    size_t n = nidx(&g);
    memset(out, 0, sizeof(double) * n * 3);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (i > 0) out[ix(&g, i, j, k)] = node_modulus(&g, K, G, 0, i, j, k);
                if (j > 0) out[n + ix(&g, i, j, k)] = node_modulus(&g, K, G, 1, i, j, k);
                if (k > 0) out[2 * n + ix(&g, i, j, k)] = node_modulus(&g, K, G, 2, i, j, k);
            }
}
