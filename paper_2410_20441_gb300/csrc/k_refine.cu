// Defect correction of the FP32 velocity-form solve (refined solves).
//
// The pseudo-time iteration of Sec. 3.2 converges to the solution of the
// linear system div sigma(ebar.x + w) = 0 at the interior velocity nodes
// (Eqs. eq:1a-eq:3a discretised on the staggered grid of Sec. 3.3).  With
// FP32 fields the computed force stops shrinking near a relative residual of
// a few 1e-6 (the rounding of the elastic stresses around near-void pores).
// A refined solve therefore splits w = w_base + dw at a "rebase":
//   * w_base (FP64) absorbs the current w (or dw), and dw restarts at 0;
//   * the right-hand side r = div sigma(ebar.x + w_base) is formed in FP64
//     (elastic stresses by k_stress<double>, divergence here), its FP64 norm
//     is the exact residual of w_base, and r is stored as FP32;
//   * the sweeps then iterate on dw alone with the force r + div C : eps(dw)
//     (the RHS variant of the TMA sweep).  By linearity this is, in exact
//     arithmetic, the same iteration (u is kept), but the FP32 arithmetic now
//     acts on the small correction, so its rounding scales with the residual
//     instead of with C : ebar.
// Finalising writes w_base back as the double-word w (FP32 high part and
// BF16 low part) of the ordinary layout, so averages, gradients, field
// export and warm starts see the usual state.
//
// Every kernel covers every element of the fields (padding included) with a
// flat index, so the slots they rewrite hold defined values everywhere.
#include "ce_internal.h"

namespace ce {

namespace {

constexpr int NT = 256;

struct Pt {
    int i, j, k;
};

__device__ __forceinline__ Pt point(const Layout& L, long long q)
{
    Pt p;
    if (L.fsize <= 0xffffffffLL) {
        // (every grid of a few GB: 32-bit divisions, far shorter than 64-bit ones)
        const unsigned pl = (unsigned)L.plane, pi = (unsigned)L.pitch, u = (unsigned)q;
        const unsigned k = u / pl, r = u - k * pl, j = r / pi;
        p.k = (int)k;
        p.j = (int)j;
        p.i = (int)(r - j * pi);
        return p;
    }
    p.k = (int)(q / L.plane);
    long long r = q - (long long)p.k * L.plane;
    p.j = (int)(r / L.pitch);
    p.i = (int)(r - (long long)p.j * L.pitch);
    return p;
}

// w_base = (first ? 0 : w_base) + hi + lo, hi = 0, per component f
__global__ void k_rebase_w(long long n, RefineW a, int first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double w = first ? 0.0 : a.wb[f][q];
            w += (double)a.hi[f][q];
            if (a.lo[f]) w += (double)__bfloat162float(a.lo[f][q]);
            a.wb[f][q] = w;
            a.hi[f][q] = 0.f;
        }
    }
}

// r = div sigma at the interior velocity nodes from the FP64 stresses s
// (p, tau_xx, tau_yy, tau_xy, tau_xz, tau_yz; tau_zz = -tau_xx - tau_yy),
// FP32 copies into r0 and r1, zero at every other element; per block the sum
// of r^2 in FP64 (fixed element-to-thread map: deterministic)
__global__ void k_rhs(Layout L, RefineR a, double* partials)
{
    const long long n = L.fsize;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double* const* s = a.s;
    auto v = [&](int f, int i, int j, int k) { return s[f][L.at(i, j, k)]; };
    auto sxx = [&](int i, int j, int k) { return -v(F_P, i, j, k) + v(F_TXX, i, j, k); };
    auto syy = [&](int i, int j, int k) { return -v(F_P, i, j, k) + v(F_TYY, i, j, k); };
    auto szz = [&](int i, int j, int k) { return -v(F_P, i, j, k) - v(F_TXX, i, j, k) - v(F_TYY, i, j, k); };
    double acc = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        const Pt p = point(L, q);
        const int i = p.i, j = p.j, k = p.k;
        double rx = 0.0, ry = 0.0, rz = 0.0;
        if (i < L.nx && j < L.ny && k < L.nz) {
            if (i > 0)
                rx = (sxx(i, j, k) - sxx(i - 1, j, k)) + (v(F_TXY, i, j + 1, k) - v(F_TXY, i, j, k))
                   + (v(F_TXZ, i, j, k + 1) - v(F_TXZ, i, j, k));
            if (j > 0)
                ry = (v(F_TXY, i + 1, j, k) - v(F_TXY, i, j, k)) + (syy(i, j, k) - syy(i, j - 1, k))
                   + (v(F_TYZ, i, j, k + 1) - v(F_TYZ, i, j, k));
            if (k > 0)
                rz = (v(F_TXZ, i + 1, j, k) - v(F_TXZ, i, j, k)) + (v(F_TYZ, i, j + 1, k) - v(F_TYZ, i, j, k))
                   + (szz(i, j, k) - szz(i, j, k - 1));
        }
        acc += rx * rx + ry * ry + rz * rz;
        const float fr[3] = { (float)rx, (float)ry, (float)rz };
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            a.r0[f][q] = fr[f];
            a.r1[f][q] = fr[f];
        }
    }
    __shared__ double sh[NT / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = t;
    }
}

// double-word w from w_base: hi = fl32(w), lo = bf16(w - hi); the low-part
// slots are rewritten whole (the unused half of slot 4 and all of slot 5 get
// zeros), as the correction phase had stored r there
__global__ void k_finalize(long long n, RefineF a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const double w = a.wb[f][q];
            const float h = (float)w;
            a.hi[f][q] = h;
            a.lo[f][q] = __float2bfloat16_rn((float)(w - (double)h));
        }
        a.lo_pad[q] = __float2bfloat16_rn(0.f);
        a.slot5[q] = 0.f;
    }
}

int flat_blocks(long long n)
{
    long long b = (n + NT - 1) / NT;
    return b > 4096 ? 4096 : (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_rebase_w(const Layout& L, const RefineW& a, int first, cudaStream_t st)
{
    k_rebase_w<<<flat_blocks(L.fsize), NT, 0, st>>>(L.fsize, a, first);
}

int rhs_blocks(const Layout& L) { return flat_blocks(L.fsize); }

void launch_rhs(const Layout& L, const RefineR& a, double* partials, cudaStream_t st)
{
    k_rhs<<<flat_blocks(L.fsize), NT, 0, st>>>(L, a, partials);
}

void launch_finalize(const Layout& L, const RefineF& a, cudaStream_t st)
{
    k_finalize<<<flat_blocks(L.fsize), NT, 0, st>>>(L.fsize, a);
}

}  // namespace ce
