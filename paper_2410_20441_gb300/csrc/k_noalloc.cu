// Allocation-free residual norm (ce_residual_noalloc in include/ce.h).
//
// Some callers cannot allocate device memory at all: code that runs inside a
// host framework which owns every byte of the GPU's memory through its own
// pool, code that must not allocate while a CUDA graph is being captured or
// replayed, and real-time loops that forbid allocation for its latency.  For
// them this entry point evaluates the elastic residual of a given state with
// no allocation: its only scratch is the file-scope array below, which every
// GPU that loads the library holds until the process exits.
//
// The caller passes the moduli and the fluctuation field in device memory
// and receives ||div sigma(ebar.x + w)||_2 and ||div sigma(ebar.x)||_2 in a
// device buffer of two doubles.  Stresses are formed on the fly from w at
// every interior velocity node (no stress scratch), summed in FP64 per block
// into the static array, then summed in a fixed order.
#include <cudaTypedefs.h>
#include <math.h>
#include <mutex>
#include <stdio.h>

#include "ce_internal.h"

namespace ce {

namespace {

// block partials: two sums (w and w = 0) per block
constexpr int NOALLOC_MAX_BLOCKS = 32768;
static __device__ __align__(256) double g_noalloc_partials[2 * NOALLOC_MAX_BLOCKS];

constexpr int NBX = 32, NBY = 8;

struct Dense {
    int nx, ny, nz;
    __device__ __forceinline__ long long idx(int i, int j, int k) const
    {
        return ((long long)k * (ny + 1) + j) * (nx + 1) + i;
    }
    __device__ __forceinline__ long long cell(int i, int j, int k) const
    {
        return ((long long)k * ny + j) * nx + i;
    }
    __device__ __forceinline__ bool in_cells(int i, int j, int k) const
    {
        return i >= 0 && j >= 0 && k >= 0 && i < nx && j < ny && k < nz;
    }
};

struct Field {
    const Dense& d;
    const float* __restrict__ w;   // w_x, w_y, w_z, each (nz+1)(ny+1)(nx+1)
    const float* __restrict__ K;
    const float* __restrict__ G;
    Ebar<float> eb;
    bool zero;
    int bc;
    long long n;
    __device__ __forceinline__ float wv(int c, int i, int j, int k) const { return zero ? 0.f : w[c * n + d.idx(i, j, k)]; }
    __device__ __forceinline__ float tang(int q, int nq, int c, int ia, int ja, int ka, int ib, int jb, int kb) const
    {
        if (q == 0) return 2.f * wv(c, ib, jb, kb);
        if (q == nq) return -2.f * wv(c, ia, ja, ka);
        return wv(c, ib, jb, kb) - wv(c, ia, ja, ka);
    }
    // arithmetic mean of G over the existing cells around an edge
    __device__ float edge_g(int dir, int i, int j, int k) const
    {
        float s = 0.f;
        int n = 0;
        for (int a = -1; a <= 0; ++a)
            for (int b = -1; b <= 0; ++b) {
                int ci = i, cj = j, ck = k;
                if (dir == 0) { ci += a; cj += b; }
                else if (dir == 1) { ci += a; ck += b; }
                else { cj += a; ck += b; }
                if (d.in_cells(ci, cj, ck)) { s += G[d.cell(ci, cj, ck)]; ++n; }
            }
        return s / (float)n;
    }
    // cell normal stress component c (0 xx, 1 yy, 2 zz) of C : eps(ebar.x + w)
    __device__ float cell_s(int c, int i, int j, int k) const
    {
        float exx = wv(0, i + 1, j, k) - wv(0, i, j, k) + eb.xx;
        float eyy = wv(1, i, j + 1, k) - wv(1, i, j, k) + eb.yy;
        float ezz = wv(2, i, j, k + 1) - wv(2, i, j, k) + eb.zz;
        float Kc = K[d.cell(i, j, k)], Gc = G[d.cell(i, j, k)];
        float lam = (Kc - (2.f / 3.f) * Gc) * (exx + eyy + ezz);
        return lam + 2.f * Gc * (c == 0 ? exx : (c == 1 ? eyy : ezz));
    }
    __device__ float txy(int i, int j, int k) const
    {
        if (free_xy(bc, i == 0 || i == d.nx, j == 0 || j == d.ny)) return 0.f;
        float e = 0.5f * (tang(j, d.ny, 0, i, j - 1, k, i, j, k) + tang(i, d.nx, 1, i - 1, j, k, i, j, k)) + eb.xy;
        return 2.f * edge_g(0, i, j, k) * e;
    }
    __device__ float txz(int i, int j, int k) const
    {
        if (free_xz(bc, i == 0 || i == d.nx, k == 0 || k == d.nz)) return 0.f;
        float e = 0.5f * (tang(k, d.nz, 0, i, j, k - 1, i, j, k) + tang(i, d.nx, 2, i - 1, j, k, i, j, k)) + eb.xz;
        return 2.f * edge_g(1, i, j, k) * e;
    }
    __device__ float tyz(int i, int j, int k) const
    {
        if (free_yz(bc, j == 0 || j == d.ny, k == 0 || k == d.nz)) return 0.f;
        float e = 0.5f * (tang(k, d.nz, 1, i, j, k - 1, i, j, k) + tang(j, d.ny, 2, i, j - 1, k, i, j, k)) + eb.yz;
        return 2.f * edge_g(2, i, j, k) * e;
    }
    // sum of squares of div sigma over the velocity nodes of index (i,j,k)
    __device__ double node_sq(int i, int j, int k) const
    {
        double s = 0.0;
        if (i > 0) {
            float r = (cell_s(0, i, j, k) - cell_s(0, i - 1, j, k)) + (txy(i, j + 1, k) - txy(i, j, k))
                    + (txz(i, j, k + 1) - txz(i, j, k));
            s += (double)r * r;
        }
        if (j > 0) {
            float r = (txy(i + 1, j, k) - txy(i, j, k)) + (cell_s(1, i, j, k) - cell_s(1, i, j - 1, k))
                    + (tyz(i, j, k + 1) - tyz(i, j, k));
            s += (double)r * r;
        }
        if (k > 0) {
            float r = (txz(i + 1, j, k) - txz(i, j, k)) + (tyz(i, j + 1, k) - tyz(i, j, k))
                    + (cell_s(2, i, j, k) - cell_s(2, i, j, k - 1));
            s += (double)r * r;
        }
        return s;
    }
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// one thread per (i, j) column, striding over k; 2 sums per block written to
// the static partials (every slot used is written, so nothing needs clearing)
__global__ void k_residual_noalloc(Dense d, const float* K, const float* G, const float* w, Ebar<float> eb,
                                   int bc, int nzr, double* part)
{
    __shared__ double sh[2][NBX * NBY / 32];
    const int i = blockIdx.x * NBX + threadIdx.x, j = blockIdx.y * NBY + threadIdx.y;
    const long long n = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    Field fw{d, w, K, G, eb, false, bc, n}, f0{d, w, K, G, eb, true, bc, n};
    double a = 0.0, b = 0.0;
    if (i < d.nx && j < d.ny)
        for (int k = blockIdx.z; k < d.nz; k += nzr) {
            a += fw.node_sq(i, j, k);
            b += f0.node_sq(i, j, k);
        }
    const int t = threadIdx.y * NBX + threadIdx.x, lane = t & 31, warp = t >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
    __syncthreads();
    if (t == 0) {
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < NBX * NBY / 32; ++q) { sa += sh[0][q]; sb += sh[1][q]; }
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[2 * bid] = sa;
        part[2 * bid + 1] = sb;
    }
}

__global__ void k_finish_noalloc(const double* __restrict__ part, int nblk, double* out)
{
    __shared__ double sh[2][32];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < (int)(blockDim.x / 32); ++q) { sa += sh[0][q]; sb += sh[1][q]; }
        out[0] = sqrt(sa);
        out[1] = sqrt(sb);
    }
}

// device address of the static partials, looked up once per device and
// CUDA context: a device reset, or a host framework that releases and
// re-creates the primary context, gives the array a new address, so the
// cached one is only used while the current context is the one it came from
constexpr int MAX_DEVICES = 64;
double* g_addr[MAX_DEVICES] = { nullptr };
CUcontext g_ctx[MAX_DEVICES] = { nullptr };
std::mutex g_addr_mu;

PFN_cuCtxGetCurrent_v4000 ctx_getter()
{
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult qr;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &qr) == cudaSuccess
            && qr == cudaDriverEntryPointSuccess)
            fn = (PFN_cuCtxGetCurrent_v4000)p;
    }
    return fn;
}

}  // namespace

}  // namespace ce

using namespace ce;

extern "C" ce_status ce_residual_noalloc(const ce_grid* g, const float* K, const float* G, const float* w,
                                         const double e6[6], int bc, double* out, void* stream)
{
    if (!g || !K || !G || !w || !e6 || !out) {
        set_free_error("ce_residual_noalloc: NULL argument");
        return CE_EINVAL;
    }
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || !valid_bc(bc)) {
        set_free_error("ce_residual_noalloc: grid below 2 voxels per axis or bad bc");
        return CE_EINVAL;
    }
    const long long gx = (g->nx + NBX - 1) / NBX, gy = (g->ny + NBY - 1) / NBY;
    if (gx * gy > NOALLOC_MAX_BLOCKS) {
        set_free_error("ce_residual_noalloc: grid too large for the static scratch: ceil(nx/%d)*ceil(ny/%d) = %lld "
                       "exceeds %d", NBX, NBY, gx * gy, NOALLOC_MAX_BLOCKS);
        return CE_EINVAL;
    }
    for (int t = 0; t < 6; ++t)
        if (!isfinite(e6[t])) {
            set_free_error("ce_residual_noalloc: non-finite load");
            return CE_EINVAL;
        }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        set_free_error("ce_residual_noalloc: no usable current device");
        return CE_ECUDA;
    }
    double* part = nullptr;
    {
        // the host-side symbol is a stand-in: the kernel must get the device
        // address of this device's copy of the array (in the current context)
        auto getctx = ctx_getter();
        CUcontext cx = nullptr;
        if (!getctx || getctx(&cx) != CUDA_SUCCESS) cx = nullptr;
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev] || !cx || g_ctx[dev] != cx) {
            g_addr[dev] = nullptr;
            e = cudaGetSymbolAddress((void**)&g_addr[dev], g_noalloc_partials);
            if (e == cudaSuccess && !cx && getctx && getctx(&cx) != CUDA_SUCCESS) cx = nullptr;
            g_ctx[dev] = cx;
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                set_free_error("ce_residual_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return CE_ECUDA;
            }
        }
        part = g_addr[dev];
    }
    int nzr = (int)(NOALLOC_MAX_BLOCKS / (gx * gy));
    if (nzr > g->nz) nzr = g->nz;
    if (nzr > 64) nzr = 64;
    if (nzr < 1) nzr = 1;
    Dense d{ g->nx, g->ny, g->nz };
    cudaStream_t st = (cudaStream_t)stream;
    k_residual_noalloc<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)nzr), dim3(NBX, NBY), 0, st>>>(
        d, K, G, w, ebar_from_voigt<float>(e6), bc, nzr, part);
    k_finish_noalloc<<<1, 1024, 0, st>>>(part, (int)(gx * gy * nzr), out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_free_error("ce_residual_noalloc: launch failed: %s", cudaGetErrorString(e));
        return CE_ECUDA;
    }
    return CE_OK;
}
