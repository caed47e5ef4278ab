/*
 * ce.h -- C interface of libce: effective elastic stiffness of a voxel image
 * by the accelerated pseudo-transient (APT) method on a staggered grid.
 *
 * Method (Alkhimenkov, "Digital rock physics: calculation of effective
 * elastic properties of heterogeneous materials using GPUs"):
 *   - quasi-static elasticity, Eqs. eq:1a-eq:3a, solved as the attractor of a
 *     damped pseudo-transient system: momentum Eq. 11111, pressure and
 *     deviator relaxation Eqs. A2ssP and A23ssP2, numerical parameters of
 *     Sec. 3.1 (Eqs. PT1_1t2-PT24q);
 *   - staggered grid of Sec. 3.3: pressure and normal deviators in cells,
 *     shear stresses on edges, velocities on faces;
 *   - an imposed macroscopic strain per load case (velocity boundary
 *     conditions, Sec. 3.4 and Appendix A) and the stiffness from volume
 *     averages <sigma> = C <eps>, Eqs. BC:1-BC:3 and eq:4.
 *
 * Conventions for every call
 *   - Grids: nx*ny*nz voxels of unit size, x fastest.  Moduli arrays hold
 *     nx*ny*nz float32 values in GPa in that order (index (k*ny + j)*nx + i).
 *   - Load cases: Voigt order (xx, yy, zz, yz, xz, xy), engineering shear
 *     strain (a case with entry 5 equal to 1 has eps_xz = eps_zx = 1/2).
 *   - C is 6x6, row-major, Voigt, GPa.
 *   - Every function returns a ce_status and never lets a C++ exception or a
 *     CUDA error escape; after an error ce_last_error() gives a message.
 *   - All device work is issued on the stream given at creation.  Calls on
 *     one context must not run concurrently from several host threads.
 *   - A "device pointer" is a CUDA global-memory address of the current
 *     device; a "host pointer" is ordinary host memory.
 */
#ifndef CE_H
#define CE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CE_MAX_CASES 6

typedef struct ce_ctx ce_ctx; /* opaque; owned by the library */

typedef enum {
    CE_OK = 0,
    CE_EINVAL = 1,     /* invalid argument (sizes, non-finite or non-positive moduli, NULL) */
    CE_ENOMEM = 2,     /* device allocation failed */
    CE_ECUDA = 3,      /* a CUDA call failed; see ce_last_error */
    CE_ENOTCONV = 4,   /* max_iter reached before tol; results are those of the last sweep */
    CE_EDIVERGED = 5,  /* residual became non-finite or grew beyond 1e10 */
    CE_ESTATE = 6,     /* call out of order (e.g. ce_ceff before ce_solve) */
    CE_ENOTIMPL = 7    /* option combination not supported */
} ce_status;

typedef enum {
    CE_PREC_FP32 = 0,  /* FP32 fields, all cases in one sweep, FP64 reductions */
    CE_PREC_FP64 = 1   /* FP64 fields, one load case at a time */
} ce_precision;

typedef enum {
    CE_BC_KUBC = 0,      /* v = ebar.x on the whole boundary (uniform kinematic) */
    CE_BC_ROLLER = 1,    /* normal velocity prescribed, boundary shear traction zero
                            (Appendix A.1); meaningful for normal load cases */
    CE_BC_SHEAR_YZ = 2,  /* simple shear tests of Appendix A.2: normal velocities prescribed, */
    CE_BC_SHEAR_XZ = 3,  /* the sheared component prescribed on the driven face pair (v_y on */
    CE_BC_SHEAR_XY = 4   /* the z faces for YZ, v_x on the z faces for XZ, v_x on the y faces
                            for XY), every other tangential traction zero (the lateral faces
                            free-slip); the load is the matching unit shear (Voigt 4, 5, 6) */
} ce_bc;

typedef enum {
    CE_KERNEL_AUTO = 0,      /* FP32: fused multi-case sweep with TMA loads; FP64: plain */
    CE_KERNEL_PLAIN = 1,     /* two kernels per sweep (stress, then velocity), stress form */
    CE_KERNEL_FUSED = 2,     /* one kernel per sweep for all cases, TMA loads (FP32 only) */
    CE_KERNEL_FUSED_LSU = 3  /* the same sweep with ordinary loads (FP32 only; for comparison) */
} ce_kernel;

typedef struct {
    int nx, ny, nz;       /* voxels per axis, each >= 2 */
} ce_grid;

/* Optional device allocator.  alloc returns a device pointer of at least
 * `bytes` bytes aligned to 256 bytes (NULL on failure); free releases it.
 * `stream` is the context's stream.  Both are called from the creating host
 * thread (alloc during ce_create, free during ce_destroy). */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} ce_allocator;

typedef struct {
    ce_precision prec;
    ce_bc bc;
    ce_kernel kernel;
    double St;         /* Strouhal number St (Eq. PT1_1t311); <= 0: 2 pi sqrt 3 (Eq. PT24q) */
    double Ct;         /* Courant number C~ (Eq. PT1_1t2); <= 0: 0.95 / sqrt 3 */
    int n_check;       /* sweeps between residual checks; <= 0: max(16, nx/4) */
    int tile[4];       /* fused-kernel launch shape, 0 = default: tile[0] copy stages of
                          the TMA sweep (2, 3 or, paired, 4; default 3), tile[1] rows
                          per block (8, 16 or, single-column, 24; default 16 single,
                          8 paired; the ordinary-load kernel takes 24 as 16), tile[2]
                          z-planes per block (TMA default 32), tile[3] columns per
                          thread (1 = single-column sweep, default; 2 = paired f32x2) */
    double St_first;   /* Strouhal number of the first phase of a refined solve (FP32 w
                          alone, until the first rebase); <= 0: St.  The phase ends at
                          a residual of 1e-3, where the St of the correction phases
                          takes over; the converged C does not depend on either. */
} ce_opts;

typedef struct {
    int n_cases;
    int iters[CE_MAX_CASES];        /* sweeps done for each case */
    double rel_res[CE_MAX_CASES];   /* final ||div sigma(w)|| / ||div sigma(0)|| */
    double res0[CE_MAX_CASES];      /* ||div sigma(0)||: norm of the load */
    int status[CE_MAX_CASES];       /* ce_status per case */
    int sweeps;                     /* sweep launches issued (all cases share one in FP32) */
    int checks;                     /* residual evaluations */
    long long case_sweeps;          /* sum over sweeps of the cases each one advanced */
    int launches;                   /* kernel launches issued by the call */
    double sweep_ms;                /* device time of the sweep launches (CUDA events on the stream) */
    double check_ms;                /* device time of the residual evaluations */
    double seconds;                 /* wall time of the call */
    double teff_gbs;                /* effective throughput of the sweeps, GB/s: the bytes each sweep
                                       must move (FP32 fused: 60 B per voxel and active case, 48 B in
                                       the first phase of a refined solve, + 8 B of K, G per voxel;
                                       plain stress form: 160 B per voxel and case in FP64, 80 B in
                                       FP32) over sweep_ms */
    int rebases;                    /* case rebases of the defect correction (refined solves) */
    int sweeps_corr;                /* of `sweeps`: those in the correction phase (refined solves) */
    long long case_sweeps_corr;     /* of `case_sweeps`: those in the correction phase */
    double sweep_ms_corr;           /* of `sweep_ms`: the correction phase's */
} ce_solve_info;

/* Fill *o with the defaults (FP32, KUBC, AUTO kernel, paper's St and C~). */
void ce_default_opts(ce_opts* o);

/* Create a context for one image.
 *   g                grid (copied).
 *   K, G             nx*ny*nz float32 moduli (GPa), all finite and > 0.
 *                    moduli_on_device = 0: host pointers; 1: device pointers.
 *                    The library copies them; the caller keeps ownership.
 *   opts             NULL for defaults (copied).
 *   a                NULL to use cudaMallocAsync/cudaFreeAsync on `stream`.
 *   stream           cudaStream_t (NULL = legacy default stream).
 *   out              receives the context.
 * Numerical parameters: dt~ = C~ St / L with L = max(nx, ny, nz) (Sec. 3.1);
 * numerical moduli K~ = K, G~ = G at each stress point; dt~/rho~ per velocity
 * node from the P-wave modulus H~ that bounds the node's stencil.
 * Errors: CE_EINVAL (grid < 2, NULL, non-finite or <= 0 modulus),
 * CE_ENOMEM, CE_ECUDA.  Allocates all device memory the solve needs. */
ce_status ce_create(const ce_grid* g, const float* K, const float* G, int moduli_on_device,
                    const ce_opts* opts, const ce_allocator* a, void* stream, ce_ctx** out);

#define CE_WARM_START 1u          /* continue from the current fields instead of re-initialising */
#define CE_NO_REFINE 2u           /* FP32: no defect correction (FP32-measured convergence only) */
#define CE_REFINE_EACH_CHECK 4u   /* FP32: rebase every case at every check (for verification) */

/* Solve n_cases (1..6) load cases to the relative residual tol.
 *   loads            n_cases*6 doubles (Voigt strain per case, host memory);
 *                    NULL = the six unit cases (n_cases must then be 6).
 *   tol              stop a case when ||div sigma(w)|| <= tol ||div sigma(0)||
 *                    (elastic operator, FP64 reduction), checked every
 *                    n_check sweeps; a case whose load is already in
 *                    equilibrium converges at sweep 0.
 *   max_iter         upper bound of sweeps per case (>= 0).
 *   flags            0 or an OR of CE_WARM_START, CE_NO_REFINE,
 *                    CE_REFINE_EACH_CHECK.
 * Refined solves (FP32 with the single-column TMA sweep on a whole image,
 * unless CE_NO_REFINE): defect correction.  When a case's residual has
 * fallen by 1e-3 since its last rebase, or reached tol, the solve rebases it:
 * w is moved into an FP64 base w_base, the right-hand side
 * r = div sigma(ebar.x + w_base) is formed in FP64 (its norm is the exact
 * residual, which alone decides convergence), and the sweeps continue on the
 * FP32 correction w - w_base with the force r + div C : eps(w - w_base).
 * The iteration is the same in exact arithmetic; FP32 rounding then scales
 * with the residual, so any tol is reachable (plain FP32 fields stall near a
 * relative residual of 1e-6 to 3e-5 on porous or cracked images).  The first
 * rebase takes every active case into the correction phase.  After the call
 * the fields are in the ordinary layout (w = w_base as FP32 + BF16).
 *   info             NULL or receives per-case iterations and residuals.
 * Fields start at w = 0 with sigma = C(x):ebar (Sec. 3.2 attractor) unless
 * CE_WARM_START.  Afterwards the volume averages of every case are stored in
 * the context and the converged fields are kept for ce_grad.
 * Returns CE_OK, CE_ENOTCONV or CE_EDIVERGED (worst case over the cases),
 * CE_EINVAL, CE_ECUDA.  Synchronises the stream before returning. */
ce_status ce_solve(ce_ctx* c, const double* loads, int n_cases, double tol, int max_iter,
                   unsigned flags, ce_solve_info* info);

/* Effective stiffness C = S E^-1 (Eq. BC:3) with S and E the 6x6 matrices
 * whose columns are <sigma> and <eps> (Voigt, engineering shear) of the six
 * cases of the last ce_solve (FP64 on the host).  C: 36 doubles, host.
 * Errors: CE_ESTATE if the last solve did not have 6 cases, CE_EINVAL if E
 * is singular. */
ce_status ce_ceff(const ce_ctx* c, double C[36]);

/* Volume averages of the last solve: sig and eps receive n_cases*6 doubles
 * each (host), Voigt order, engineering shear for eps. */
ce_status ce_averages(const ce_ctx* c, double* sig, double* eps);

/* The paper's direct tests (Sec. 3.4, Appendix A), from the last solve of
 * the four loads e1, e2, e3 and e1 + e2 + e3 (Voigt normal strains, any
 * nonzero scale; the paper runs them with CE_BC_ROLLER: each normal velocity
 * prescribed on one face pair, tangential tractions free):
 *   out[0..2] = C11, C22, C33 = <sigma_ii> / <eps_ii> of the single-axis
 *               tests (Eq. eq:4, Appendix A.1);
 *   out[3..5] = C12, C13, C23 from the combined test by Eqs. D1-D5
 *               (Appendix A.3): sbar_i = <sigma_ii> - C_ii <eps_ii>,
 *               ebar_i = <eps_ii>, then the closed forms D3, D4, D5.
 * 6 doubles, host.  Exact for an orthorhombic medium whose axes are the grid
 * axes.  Errors: CE_ESTATE if the last solve was not those four loads,
 * CE_EINVAL for a zero average strain. */
ce_status ce_direct_tests(const ce_ctx* c, double out[6]);

/* Gradient of J = sum_mn w_mn C_mn with respect to every voxel's K and G,
 * from the fields of the last ce_solve of the six unit load cases (the
 * operator is symmetric, so the adjoint fields are the forward ones, and
 * dC_mn/dp = (1/V) a_p(u^m, u^n) at equilibrium; future item 5 of Sec. 5.3).
 *   w                36 doubles, row-major (host).
 *   dJdK, dJdG       nx*ny*nz float32 each; out_on_device = 0: host pointers,
 *                    1: device pointers.  Caller-owned.
 * Errors: CE_ESTATE if the last solve was not the six unit cases. */
ce_status ce_grad(ce_ctx* c, const double w[36], float* dJdK, float* dJdG, int out_on_device);

/* Copy one state field of one case to host memory as doubles, on the dense
 * (nz+1)*(ny+1)*(nx+1) index grid (x fastest).  field: 0 p, 1 tau_xx,
 * 2 tau_yy, 3 tau_xy, 4 tau_xz, 5 tau_yz, 6 w_x, 7 w_y, 8 w_z (w is the
 * velocity fluctuation v - ebar.x).  Entries outside a field's own lattice
 * are zero.  The fused FP32 path keeps the state in velocity form (w and the
 * last increment u = w_{n+1} - w_n); there fields 0-5 are the elastic stress
 * C : eps(ebar.x + w) of the current w and fields 9, 10, 11 give u_x, u_y,
 * u_z.  For tests and inspection. */
ce_status ce_get_field(const ce_ctx* c, int case_index, int field, double* host_out);

/* Release the context and all device memory it holds (NULL is a no-op). */
void ce_destroy(ce_ctx* c);

const char* ce_status_str(ce_status s);
const char* ce_last_error(const ce_ctx* c); /* never NULL; per context; with c == NULL the last
                                              error of a context-free call in this thread */

/* ---------------------------------------------------- allocation-free check
 * The paper has no counterpart to this call: it exists for callers that
 * cannot allocate device memory -- code inside a host framework that owns all
 * GPU memory through its own pool, code that must not allocate while a CUDA
 * graph is captured or replayed, real-time loops that forbid allocation --
 * and still want to verify a state.  It evaluates the elastic residual of a
 * given fluctuation field without any allocation: its only scratch is a
 * file-scope device array of 2 x 32768 doubles (512 KiB) that every GPU
 * which loads the library holds until the process exits.
 *   g          grid; rejected with CE_EINVAL when ceil(nx/32) * ceil(ny/8)
 *              exceeds 32768 (the array's block capacity), e.g. beyond
 *              4096 x 2048 voxels per plane; any nz.
 *   K, G       device pointers, nx*ny*nz float32 moduli (as in ce_create).
 *   w          device pointer, three float32 arrays w_x, w_y, w_z one after
 *              the other, each on the dense (nz+1)*(ny+1)*(nx+1) index grid
 *              (the layout of ce_get_field).
 *   e6         the load case (6 doubles, host, Voigt, engineering shear).
 *   bc         a ce_bc boundary mode.
 *   out        device pointer to 2 doubles: out[0] = ||div sigma(ebar.x + w)||,
 *              out[1] = ||div sigma(ebar.x)|| (2-norms over the interior
 *              velocity nodes; FP32 stresses, FP64 sums).
 *   stream     cudaStream_t; the call is asynchronous on it.
 * The first call on a device looks up the array's device address (with that
 * device current), and so does the first call after the device's CUDA
 * context changed (a device reset, or a host framework that re-created the
 * primary context); make such a call before any stream capture.  Calls
 * share the array and keep the previous call's contents there; every slot a
 * call reads is written by the same call first, so nothing needs clearing,
 * but calls that overlap on the GPU (on different streams) race.  Errors:
 * CE_EINVAL (NULL, grid, bc, non-finite load) and CE_ECUDA; the message is
 * available from ce_last_error(NULL) in the calling thread. */
ce_status ce_residual_noalloc(const ce_grid* g, const float* K, const float* G, const float* w,
                              const double e6[6], int bc, double* out, void* stream);

/* Replace the moduli of a context (same grid and layout as ce_create) and
 * recompute dt~/rho~; the fields of the last solve stay, so the next
 * ce_solve may warm start from them (an inverse problem or a finite
 * difference moves the moduli a little).  CE_EINVAL for moduli that are not
 * positive and finite: the context then refuses to solve (CE_ESTATE) until
 * valid moduli are set.  No counterpart in the paper, which solves each
 * image once. */
ce_status ce_set_moduli(ce_ctx* c, const float* K, const float* G, int moduli_on_device);

/* -------------------------------------------------------------- autotuning
 * Launch-shape search for the FP32 TMA sweep of one image (no counterpart in
 * the paper, whose kernel has a fixed launch shape).  Times `sweeps` sweeps
 * (1..1000) of the six unit load cases for every candidate: (columns per
 * thread, copy stages) in {(1,3), (1,2), (2,3), (2,4), (2,2)} x rows per
 * block {8, 16, and 24 for one column per thread} x z-planes per block
 * {16, 24, 32, 48, 64, 96, 128, 192, 256}, on the context's
 * stream, and keeps the fastest as the context's tile.  A context that runs
 * refined solves (FP32, one whole image) is timed in their two sweep modes
 * (half the sweeps each) on the single-column shapes, the ones they run on.
 * tile_out (NULL or 4 ints) receives it, ms_out (NULL or 1 double) its time
 * per sweep.  The fields are overwritten: a warm start after it returns
 * CE_ESTATE.  CE_ENOTIMPL for FP64, plain or ordinary-load kernels and
 * batches. */
ce_status ce_autotune(ce_ctx* c, int sweeps, int* tile_out, double* ms_out);

/* The same search for the solves the tile will serve: CE_TUNE_AUTO as
 * ce_autotune; CE_TUNE_PLAIN times the double-word sweep of unrefined solves,
 * batches and slabs (every shape); CE_TUNE_REFINED the two modes of refined
 * solves (single-column shapes; CE_ENOTIMPL on a context that runs none).
 * CE_EINVAL for another value. */
enum { CE_TUNE_AUTO = 0, CE_TUNE_PLAIN = 1, CE_TUNE_REFINED = 2 };
ce_status ce_autotune_for(ce_ctx* c, int sweeps, int solves, int* tile_out, double* ms_out);

/* z-planes per block that the FP32 TMA sweep of a whole image of grid g
 * (tile as ce_opts.tile) uses for a launch over n_cases (1..6) of the six
 * load cases on a device with n_sm SMs, into *planes.  The tile's chunk is
 * sized for six cases; a launch over fewer shortens it (down to 16 planes)
 * when that fills the grid's last wave of blocks better (no counterpart in the
 * paper).  n_sm <= 0 or the paired-column sweep: the tile's chunk.  Host
 * only, no GPU needed.  CE_EINVAL for a bad grid, case count or NULL. */
ce_status ce_sweep_chunk(const ce_grid* g, const int tile[4], int n_cases, int n_sm, int* planes);

/* Set the tile of a single-image context (meaning as ce_opts.tile), e.g. one
 * found earlier by ce_autotune and cached by the caller.  CE_EINVAL for a
 * shape outside those listed there. */
ce_status ce_set_tile(ce_ctx* c, const int tile[4]);

/* ---------------------------------------------------------------- batches
 * Many independent images of uneven size solved together: every sweep is one
 * launch over all active samples' tiles, the whole pseudo-time loop is one
 * CUDA graph with a device-side WHILE condition (bounded by max_iter), and
 * converged samples drop out.  FP32 only.
 *   n                number of samples (1..1024).
 *   g, K, G          arrays of n grids and n moduli pointers (host pointers
 *                    to the arrays; the moduli themselves host or device
 *                    memory per moduli_on_device).
 */
ce_status ce_create_batch(int n, const ce_grid* g, const float* const* K, const float* const* G,
                          int moduli_on_device, const ce_opts* opts, const ce_allocator* a,
                          void* stream, ce_ctx** out);

/* Solve the six unit load cases of every sample; sample s stops when all
 * its cases are at tol.  With the single-column sweep the graph first keeps
 * w in FP32 alone while any active sample's residual is above 1e-3, then
 * sweeps the double-word state (whose precision sets the reachable tol, about
 * 1e-5 at 191^3).  iters (NULL or n ints) receives the sweeps each sample
 * needed.  Returns the worst status over the samples; CE_ECUDA when a
 * sample's sweep raised the device error flag. */
ce_status ce_solve_batch(ce_ctx* c, double tol, int max_iter, int* iters);

/* C of every sample: n*36 doubles (host). */
ce_status ce_ceff_batch(const ce_ctx* c, double* C);

/* ----------------------------------------------------------------- z-slabs
 * One grid split along z into slabs, each its own context (on its own
 * stream or GPU): the domain decomposition the paper plans for several GPUs
 * (Sec. 5.3, item 1).  A slab owns the index planes z0 <= k < z1 of the
 * grid's planes 0..nz (the slabs of one grid partition 0..nz; each owns at
 * least one plane) and updates only those; it also holds one ghost plane on
 * each side that has a neighbour.  The caller drives the pseudo-time loop:
 *   ce_slab_start                        (every slab)
 *   repeat: ce_slab_sweep(.., 1, check)  (every slab)
 *           ce_slab_pack(side 0 and 1) -> move each message to the neighbour
 *           on that side -> ce_slab_unpack on the receiving side
 *           when check: ce_slab_residual, summed over the slabs; the case is
 *           converged at sqrt(sum r2) <= tol * sqrt(sum b2)
 *   ce_slab_sums (every slab), summed, / (nx ny nz) -> <sigma>, <eps>.
 * Every point is computed by the whole-grid sweep's arithmetic, so the
 * slabs' fields equal those of one whole-grid context after as many sweeps;
 * only the sums (residuals, averages) add in another order.  FP32 TMA sweep
 * only (single-column tiles): other precisions and kernels give CE_ENOTIMPL,
 * and so do ce_solve, ce_grad and ce_autotune on a slab context; ce_ceff and
 * ce_averages give CE_ESTATE.  ce_get_field works and returns the slab's
 * local planes (global plane = local plane + c0 of ce_slab_cells). */

/* Cells [*c0, *c1) along z (of the grid g) that the slab owning planes
 * [z0, z1) reads: its own cells plus one ghost cell layer on each side that
 * has a neighbour.  CE_EINVAL when 0 <= z0 < z1 <= nz + 1 fails or the
 * window would hold fewer than 2 cell layers. */
ce_status ce_slab_cells(const ce_grid* g, int z0, int z1, int* c0, int* c1);

/* A slab context.  g is the whole grid; K and G hold the slab's cells
 * [c0, c1) only (nx*ny*(c1-c0) floats each, x fastest, host or device per
 * moduli_on_device).  The numerical scalars (Sec. 3.1) use the whole grid's
 * extent.  Other arguments as ce_create. */
ce_status ce_create_slab(const ce_grid* g, int z0, int z1, const float* K, const float* G,
                         int moduli_on_device, const ce_opts* opts, const ce_allocator* a,
                         void* stream, ce_ctx** out);

/* Initial state of n_cases load cases (loads as ce_solve; NULL = the six
 * unit cases) and b2[n_cases] (host): this slab's share of ||div sigma(0)||^2
 * over its own velocity nodes.  Synchronous.  The ghost planes need no
 * exchange before the first sweep (w = 0 everywhere). */
ce_status ce_slab_start(ce_ctx* c, const double* loads, int n_cases, double* b2);

/* n_sweeps sweeps of the cases in `cases` (n entries; NULL = all cases of
 * the start), asynchronous on the slab's stream.  With check != 0 the last
 * sweep also measures the residual of the state it started from; read it
 * with ce_slab_residual.  Between two sweeps the ghost planes must be
 * refreshed (pack, move, unpack): n_sweeps > 1 is only right for a slab
 * without neighbours. */
ce_status ce_slab_sweep(ce_ctx* c, const int* cases, int n, int n_sweeps, int check);

/* One sweep of the cases in `cases` (as ce_slab_sweep, one sweep, no
 * residual) split in two, so that the halo exchange can run while the
 * interior is swept: part 1 updates the own planes next to a neighbour
 * (z0 with a neighbour below, z1 - 1 with one above), after which
 * ce_slab_pack packs those new planes; part 2 updates the other own planes
 * and completes the sweep (ce_slab_unpack then fills the new state's ghost
 * planes).  The fields equal those of ce_slab_sweep.  Asynchronous on the
 * slab's stream.  CE_ESTATE when part 2 does not follow a part 1 of the same
 * cases (ce_slab_sweep is refused in between). */
ce_status ce_slab_sweep_part(ce_ctx* c, const int* cases, int n, int part);

/* r2[n] (host): this slab's share of ||div sigma(w)||^2 for the n cases of
 * the last checked ce_slab_sweep.  Synchronous; CE_ECUDA when a copy wait of
 * the sweep timed out; CE_ESTATE without a checked sweep. */
ce_status ce_slab_residual(ce_ctx* c, double* r2);

/* Size in bytes of one halo message: 18 * (ny + 1) * pitch * n_cases, with
 * pitch = nx + 1 rounded up to a multiple of 32 (per case the three FP32
 * high parts and the three BF16 low parts of w on one index plane). */
ce_status ce_slab_halo_bytes(const ce_ctx* c, size_t* bytes);

/* Copy the own plane next to `side` (0: plane z0, 1: plane z1 - 1) of every
 * case's current state into msg (device, 16-byte aligned, caller-owned,
 * ce_slab_halo_bytes long).  Asynchronous on the slab's stream. */
ce_status ce_slab_pack(ce_ctx* c, int side, void* msg);

/* Copy msg (a message packed by the neighbour on `side`) into the ghost
 * plane on that side (0: plane z0 - 1, 1: plane z1).  CE_EINVAL when that
 * side has no neighbour.  Asynchronous on the slab's stream. */
ce_status ce_slab_unpack(ce_ctx* c, int side, const void* msg);

/* Per case 12 sums (host, n_cases x 12): sigma xx, yy, zz, yz, xz, xy and
 * the engineering strains in the same order, over this slab's own cells and
 * edges with the whole grid's trapezoid weights (Eqs. BC:1-BC:3); divide the
 * slabs' total by nx*ny*nz for the averages.  Synchronous. */
ce_status ce_slab_sums(ce_ctx* c, double* sums);

/* C = S E^-1 (Eq. BC:3) from the sums of the six unit (or any six
 * independent) load cases added over all slabs of one grid: `sums` is
 * 6 x 12 doubles (host) in the layout of ce_slab_sums, g the whole grid
 * (the averages are the sums over nx ny nz).  C: 36 doubles, host.
 * Context-free: errors (CE_EINVAL: NULL, n_cases != 6, singular strains)
 * leave their message for ce_last_error(NULL). */
ce_status ce_ceff_from_sums(const double* sums, int n_cases, const ce_grid* g, double C[36]);

#ifdef __cplusplus
}
#endif
#endif /* CE_H */
