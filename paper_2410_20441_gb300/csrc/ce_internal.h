// Internal declarations of libce: device layout, stencil helpers and kernel
// launchers.  Staggered grid of Sec. 3.3: every field lives on the
// (nx+1)(ny+1)(nz+1) index grid, x fastest, rows padded to `pitch` elements.
//   cell (i,j,k)      p, tau_xx, tau_yy (tau_zz = -tau_xx - tau_yy), K, G
//   x-face i<=nx      w_x at (i, j+1/2, k+1/2)       (Dirichlet at i = 0, nx)
//   y-face j<=ny      w_y at (i+1/2, j, k+1/2)       (Dirichlet at j = 0, ny)
//   z-face k<=nz      w_z at (i+1/2, j+1/2, k)       (Dirichlet at k = 0, nz)
//   xy-edge           tau_xy at (i, j, k+1/2), i<=nx, j<=ny
//   xz-edge           tau_xz at (i, j+1/2, k), i<=nx, k<=nz
//   yz-edge           tau_yz at (i+1/2, j, k), j<=ny, k<=nz
// w is the velocity fluctuation v - ebar.x; the macroscopic strain rate ebar
// enters every strain rate exactly.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ce.h"

namespace ce {

enum { F_P = 0, F_TXX, F_TYY, F_TXY, F_TXZ, F_TYZ, F_WX, F_WY, F_WZ, NFIELD = 9 };
// velocity-form state (fused FP32 path): per load case and buffer
//   slots 0, 1, 2   u = w_{n+1} - w_n (FP32)
//   slots 6, 7, 8   w, high part (FP32)
//   slot 3          low parts of w_x and w_y (two BF16 arrays of fsize)
//   slot 4          low part of w_z (BF16, first half of the slot)
// w = hi + lo is a double-word value: |lo| <= ulp(hi)/2, kept exact to about
// 2^-33 relative by an error-free sum in every update.
// Correction phase of a refined solve (defect correction): slots 6-8 hold the
// FP32 correction dw accumulated since the last rebase (no low part), slots
// 3, 4, 5 the FP32 right-hand side r = div sigma(ebar.x + w_base) computed in
// FP64, in both buffers; w_base itself is an FP64 array outside the buffers.
enum { F_UX = 0, F_UY = 1, F_UZ = 2, F_WLO_XY = 3, F_WLO_Z = 4, F_RX = 3, F_RY = 4, F_RZ = 5 };

struct Layout {
    int nx, ny, nz;
    int pitch;        // elements per padded row (multiple of 32)
    long long plane;  // pitch * (ny + 1)
    long long fsize;  // plane * (nz + 1): elements per field
    // z-slab window (a context holding planes of a larger grid): the sweeps
    // update, and the reductions sum over, the local index planes
    // kz0 <= k < kz1 only; local plane k is plane k + zoff of a grid of nzg
    // cells in z.  A whole grid has kz0 = 0, kz1 = nz + 1, zoff = 0, nzg = nz.
    int kz0, kz1, zoff, nzg;
    __host__ __device__ __forceinline__ long long at(int i, int j, int k) const
    {
        return (long long)k * plane + (long long)j * pitch + i;
    }
};

// macroscopic strain (tensor components; Voigt engineering shear halved)
template <class T>
struct Ebar {
    T xx, yy, zz, yz, xz, xy;
};

template <class T>
__host__ inline Ebar<T> ebar_from_voigt(const double e[6])
{
    Ebar<T> b;
    b.xx = (T)e[0]; b.yy = (T)e[1]; b.zz = (T)e[2];
    b.yz = (T)(0.5 * e[3]); b.xz = (T)(0.5 * e[4]); b.xy = (T)(0.5 * e[5]);
    return b;
}

template <class T>
struct CaseArgs {
    T* f[NFIELD];     // field base pointers of one case
    Ebar<T> eb;
    const __nv_bfloat16* lo[3] = { nullptr, nullptr, nullptr };   // low parts of w (velocity form)
};

// per-sweep numerical parameters (Sec. 3.1 with K~ = K, G~ = G).  The
// relaxation (x - x_old)/(M dt~) + x/(M dt) = rate is solved for the new
// value in increment form, x_new = x_old + a (M rate - x_old) with
// a = theta/(1+theta), theta = dt~/dt: the same value as
// (x_old + theta M rate)/(1 + theta), but FP32 rounding of x_old is no longer
// amplified by 1/theta at the fixed point.
template <class T>
struct Relax {
    T a;       // theta / (1 + theta)
};

// derivative of a boundary-tangential component at integer position q in
// 0..n: interior central difference, half-spacing difference to the
// Dirichlet value 0 at q = 0 and q = n.  lo = node q-1, hi = node q.
template <class T>
__device__ __forceinline__ T tdiff(int q, int n, T lo, T hi)
{
    return q == 0 ? (T)2 * hi : (q == n ? (T)(-2) * lo : hi - lo);
}

// Boundary edges whose shear stress is held at zero (a traction-free
// tangential component) under boundary mode bc; on_x etc. say whether the
// edge lies on an x, y or z face of the box.  KUBC: none.  ROLLER: every
// boundary edge.  SHEAR_* (Appendix A.2): every boundary edge except those of
// the sheared component on its driven face pair, and the edges where that
// pair meets a lateral face.
__host__ __device__ __forceinline__ bool free_xy(int bc, bool on_x, bool on_y)
{
    return bc == CE_BC_KUBC ? false : bc == CE_BC_SHEAR_XY ? on_x : (on_x || on_y);
}
__host__ __device__ __forceinline__ bool free_xz(int bc, bool on_x, bool on_z)
{
    return bc == CE_BC_KUBC ? false : bc == CE_BC_SHEAR_XZ ? on_x : (on_x || on_z);
}
__host__ __device__ __forceinline__ bool free_yz(int bc, bool on_y, bool on_z)
{
    return bc == CE_BC_KUBC ? false : bc == CE_BC_SHEAR_YZ ? on_y : (on_y || on_z);
}
__host__ __device__ __forceinline__ bool valid_bc(int bc) { return bc >= CE_BC_KUBC && bc <= CE_BC_SHEAR_XY; }

// arithmetic mean of G over the existing cells adjacent to an edge; dir 0:
// xy edge (cells i-1..i, j-1..j at k), 1: xz edge (i-1..i, k-1..k at j),
// 2: yz edge (j-1..j, k-1..k at i)
template <class T>
__device__ __forceinline__ T edge_G(const Layout& L, const float* __restrict__ G, int dir, int i, int j,
                                    int k)
{
    T s = 0;
    int n = 0;
#pragma unroll
    for (int da = -1; da <= 0; ++da)
#pragma unroll
        for (int db = -1; db <= 0; ++db) {
            int ci = i, cj = j, ck = k;
            if (dir == 0) { ci += da; cj += db; }
            else if (dir == 1) { ci += da; ck += db; }
            else { cj += da; ck += db; }
            if (ci >= 0 && cj >= 0 && ck >= 0 && ci < L.nx && cj < L.ny && ck < L.nz) {
                s += (T)G[L.at(ci, cj, ck)];
                ++n;
            }
        }
    // n is 4 inside, 2 on a face, 1 on an outer edge line: multiplying by
    // its reciprocal is exact and gives the quotient's bits without an FP64
    // division (a long instruction sequence on this part)
    return n == 4 ? s * (T)0.25 : n == 2 ? s * (T)0.5 : n == 1 ? s : s / (T)n;
}

// ------------------------------------------------------------ launchers
// all launchers enqueue on `st` and report launch errors via cudaGetLastError
template <class T>
void launch_node_coef(const Layout& L, const float* K, const float* G, T* rx, T* ry, T* rz, double cdr,
                      cudaStream_t st);
void launch_validate(const Layout& L, const float* K, const float* G, int* bad, cudaStream_t st);
void launch_scatter_moduli(const Layout& L, const float* Kd, const float* Gd, float* K, float* G,
                           cudaStream_t st);
template <class T>
void launch_init(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases, int ncases,
                 int bc, cudaStream_t st);
template <class T>
void launch_plain_sweep(const Layout& L, const float* K, const float* G, const T* rx, const T* ry,
                        const T* rz, const CaseArgs<T>* cases, int ncases, Relax<T> rp, int bc,
                        cudaStream_t st);
template <class T>
void launch_residual(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases,
                     const CaseArgs<T>* scratch, int ncases, int bc, int zero_w, double* partials,
                     int nblk_cap, double* out, cudaStream_t st);
template <class T>
void launch_elastic_stress(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases,
                           const CaseArgs<T>* dst, int ncases, int bc, cudaStream_t st);
// u = r div sigma(src stresses) at interior velocity nodes, 0 elsewhere
template <class T>
void launch_uinit(const Layout& L, const T* rx, const T* ry, const T* rz, const CaseArgs<T>* src,
                  const CaseArgs<T>* dst, int ncases, cudaStream_t st);
// elastic = 0: average the stored stresses; 1: the elastic stress of w
template <class T>
void launch_average(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases, int ncases,
                    int elastic, int bc, double* partials, int nblk_cap, double* out, cudaStream_t st);
template <class T>
void launch_gather_field(const Layout& L, const T* f, double* dense, cudaStream_t st);
// velocity form: field 0-5 elastic stress of w, 6-8 w = hi + lo, 9-11 u
void launch_gather_vform(const Layout& L, const float* K, const float* G, const CaseArgs<float>& c, int field,
                         int bc, double* dense, cudaStream_t st);
void launch_grad(const Layout& L, const float* K, const float* G, const CaseArgs<float>* cases32,
                 const CaseArgs<double>* cases64, const double* wsym, float* dK, float* dG, int bc,
                 cudaStream_t st);
int reduce_blocks(const Layout& L);
// message of the last failed context-free call in the calling thread
// (ce_last_error(NULL)); set by every failure that has no context to hold it
const char* free_last_error();
void set_free_error(const char* fmt, ...);
// fixed-order sum of nblk partials per case (one double each) into out[case]
void launch_reduce(const double* partials, int nblk, int ncases, double* out, cudaStream_t st);

// fused multi-case FP32 sweep in velocity form: reads `in`, writes `out`
// (ping-pong); with `partials` != nullptr it also writes, per case and
// block, the sum of squares of div T(w_in) over the interior velocity nodes
struct FusedArgs {
    Layout L;
    const float* K;
    const float* G;
    const float* rx;
    const float* ry;
    const float* rz;
    int ncase;
    int bc;
    float a;          // theta / (1 + theta), see Relax
    const float* in[CE_MAX_CASES][NFIELD];
    float* out[CE_MAX_CASES][NFIELD];
    Ebar<float> eb[CE_MAX_CASES];
    double* partials;   // [case][block] or nullptr
};
// returns the number of blocks of the launch (the partials stride)
int launch_fused_sweep(const FusedArgs& a, const int tile[3], cudaStream_t st);
int fused_blocks(const Layout& L, const int tile[3]);

// representation of the state a TMA sweep reads and writes:
//   MODE_DW   w = FP32 high + BF16 low part, load T(0) = C : ebar (default);
//   MODE_F32  w in FP32 alone, load T(0) (first phase of a refined solve);
//   MODE_RHS  FP32 correction dw of an FP64 base, load r in slots 3-5
//             (correction phase of a refined solve)
enum { MODE_DW = 0, MODE_F32 = 1, MODE_RHS = 2 };

// TMA variant of the fused sweep: the state is read through tensor maps of
// the two ping-pong buffers (FP32 and BF16 views, 4-D: x, y, z, field slot)
// and of the material block (K, G, rx, ry, rz as slots 0-4)
struct TmaArgs {
    CUtensorMap st32[2];
    CUtensorMap st16[2];
    CUtensorMap mat;
    Layout L;
    int ncase;
    int bc;
    float a;
    int buf[CE_MAX_CASES];       // buffer holding the state of active entry q
    int case_id[CE_MAX_CASES];   // load case of entry q (field slots case_id * 9 + f)
    float* base[2];              // the two ping-pong buffers (entry q writes base[1 - buf[q]])
    Ebar<float> eb[CE_MAX_CASES];
    double* partials;            // [entry][block] sums of squares, or nullptr
    int* err;                    // set to 1 when an mbarrier wait timed out
    const float* matp;           // the moduli block: K, G, rx, ry, rz slots
    int cols;                    // columns per thread the maps were encoded for (1 or 2)
    int mode;                    // representation of w of every entry: MODE_DW, MODE_F32 or MODE_RHS
};
// encode the five maps; box height ty rows, box rows sized for the sweep
// with `cols` columns per thread (1 or 2); returns false on failure
bool encode_tma_maps(TmaArgs& a, const Layout& L, void* state0, void* state1, void* mat, int ty, int cols);
// rows per block of the TMA sweep for a tile (default 8 paired-column,
// 16 single-column)
int sweep_rows(const int tile[4]);
// one TMA sweep (the single- or paired-column kernel the maps were encoded for)
int launch_fused_tma(const TmaArgs& a, const int tile[4], cudaStream_t st);
int fused_tma_blocks(const Layout& L, const int tile[4]);
int fused_tma_chunk(const Layout& L, const int tile[4], int n, int nsm);
// the paired-column sweep (k_pair.cu)
void pair_geometry(const Layout& L, const int tile[4], int* ty, int* nst, int* nbx, int* nby, int* nch, int* zc);
int launch_pair_tma(const TmaArgs& a, const int tile[4], cudaStream_t st);
const void* pair_batch_kernel(int ty, int nst, bool check, int* smem);

// one sample of a batched solve (device array; 64-byte aligned for the maps)
struct BatchEntry {
    TmaArgs a;
    int nbx, nby, nch, zc;
    int off;   // first block of this sample in the batched grid
};
static_assert(alignof(BatchEntry) % 64 == 0 && sizeof(BatchEntry) % 64 == 0, "tensor maps need 64-byte alignment");
void batch_geometry(const Layout& L, const int tile[4], int* nbx, int* nby, int* nch, int* zc);
// the batched sweep kernel k_sweep_tma_batch<ty, nst, check, mode> (mode
// MODE_DW or MODE_F32; arguments: ents, nsamp, active, parity, k, part,
// pstride; block (32, ty)) and its dynamic shared memory in *smem; nullptr
// when the attribute cannot be set
const void* batch_kernel(int ty, int nst, bool check, int mode, int* smem);

// defect correction of refined solves (k_refine.cu); flat kernels over all
// fsize elements of the fields
struct RefineW {                  // w_base (+)= hi + lo, hi = 0
    double* wb[3];
    float* hi[3];
    const __nv_bfloat16* lo[3];   // nullptr in the correction phase (no low part)
};
struct RefineR {                  // r = div s at interior velocity nodes, FP32 into r0 and r1
    const double* s[6];           // p, tau_xx, tau_yy, tau_xy, tau_xz, tau_yz (FP64)
    float* r0[3];
    float* r1[3];
};
struct RefineF {                  // hi = fl32(w_base), lo = bf16(w_base - hi); pad halves zeroed
    const double* wb[3];
    float* hi[3];
    __nv_bfloat16* lo[3];
    __nv_bfloat16* lo_pad;        // the unused second half of slot 4 (BF16 view)
    float* slot5;
};
void launch_rebase_w(const Layout& L, const RefineW& a, int first, cudaStream_t st);
// blocks (= residual partials) of launch_rhs
int rhs_blocks(const Layout& L);
void launch_rhs(const Layout& L, const RefineR& a, double* partials, cudaStream_t st);
void launch_finalize(const Layout& L, const RefineF& a, cudaStream_t st);

// halo planes of a z-slab (k_slab.cu): per case, the base of the case's
// field slots in the buffer that holds its current state
struct HaloArgs {
    float* base[CE_MAX_CASES];
};
// bytes of one plane's message for ncases load cases
size_t halo_bytes(const Layout& L, int ncases);
// copy w (high and low parts) of local plane `plane` into msg (unpack = 0)
// or from msg into the plane (unpack = 1)
void launch_halo(const Layout& L, const HaloArgs& h, int ncases, int plane, void* msg, int unpack,
                 cudaStream_t st);

}  // namespace ce
