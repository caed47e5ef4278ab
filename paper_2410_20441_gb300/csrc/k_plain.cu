// Plain (unfused) kernels of libce, templated on the field type T (float or
// double): material set-up, initial state, one pseudo-time sweep as two
// kernels (stress update, then velocity update; Sec. 3.2), the elastic
// residual ||div sigma(w)|| and the volume averages (Eqs. BC:1, BC:2).
// One thread per index-grid point (i, j, k); case index from blockIdx.z.
#include <math.h>

#include "ce_internal.h"

namespace ce {

namespace {

constexpr int BX = 32, BY = 8;
constexpr int ZR = 8;   // z-planes strided by one reduction block column

template <class T>
struct Cases {
    CaseArgs<T> c[CE_MAX_CASES];
    int n;
};

template <class T>
Cases<T> pack(const CaseArgs<T>* cases, int n)
{
    Cases<T> p;
    for (int m = 0; m < n; ++m) p.c[m] = cases[m];
    p.n = n;
    return p;
}

dim3 grid_for(const Layout& L, int ncases)
{
    return dim3((L.nx + 1 + BX - 1) / BX, (L.ny + 1 + BY - 1) / BY, (L.nz + 1) * ncases);
}

int zr(const Layout& L) { return L.nz + 1 < ZR ? L.nz + 1 : ZR; }

// reductions: gridDim.z = zr * ncases, each block strides over k
dim3 grid_red(const Layout& L, int ncases)
{
    return dim3((L.nx + 1 + BX - 1) / BX, (L.ny + 1 + BY - 1) / BY, zr(L) * ncases);
}

struct Pos {
    int i, j, k, m;
    bool ok;
};

__device__ __forceinline__ Pos pos(const Layout& L)
{
    Pos p;
    p.i = blockIdx.x * BX + threadIdx.x;
    p.j = blockIdx.y * BY + threadIdx.y;
    p.k = blockIdx.z % (L.nz + 1);
    p.m = blockIdx.z / (L.nz + 1);
    p.ok = p.i <= L.nx && p.j <= L.ny;
    return p;
}

__device__ __forceinline__ bool is_cell(const Layout& L, int i, int j, int k)
{
    return i < L.nx && j < L.ny && k < L.nz;
}

// row-sum bound 2 H + 4 |lambda| of a cell's stress-rate stencil; 0 outside
__device__ double cell_rowsum(const Layout& L, const float* __restrict__ K, const float* __restrict__ G,
                              int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= L.nx || j >= L.ny || k >= L.nz) return 0.0;
    double Kc = K[L.at(i, j, k)], Gc = G[L.at(i, j, k)];
    return 2.0 * (Kc + 4.0 / 3.0 * Gc) + 4.0 * fabs(Kc - 2.0 / 3.0 * Gc);
}

template <class T>
__global__ void k_node_coef(Layout L, const float* __restrict__ K, const float* __restrict__ G, T* rx, T* ry,
                            T* rz, double cdr)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    long long q = L.at(i, j, k);
    T vx = 0, vy = 0, vz = 0;
    if (is_cell(L, i, j, k)) {
        if (i > 0) {
            double r = cell_rowsum(L, K, G, i - 1, j, k) + cell_rowsum(L, K, G, i, j, k)
                     + 4.0 * (edge_G<double>(L, G, 0, i, j, k) + edge_G<double>(L, G, 0, i, j + 1, k)
                              + edge_G<double>(L, G, 1, i, j, k) + edge_G<double>(L, G, 1, i, j, k + 1));
            vx = (T)(cdr / (r / 12.0));
        }
        if (j > 0) {
            double r = cell_rowsum(L, K, G, i, j - 1, k) + cell_rowsum(L, K, G, i, j, k)
                     + 4.0 * (edge_G<double>(L, G, 0, i, j, k) + edge_G<double>(L, G, 0, i + 1, j, k)
                              + edge_G<double>(L, G, 2, i, j, k) + edge_G<double>(L, G, 2, i, j, k + 1));
            vy = (T)(cdr / (r / 12.0));
        }
        if (k > 0) {
            double r = cell_rowsum(L, K, G, i, j, k - 1) + cell_rowsum(L, K, G, i, j, k)
                     + 4.0 * (edge_G<double>(L, G, 1, i, j, k) + edge_G<double>(L, G, 1, i + 1, j, k)
                              + edge_G<double>(L, G, 2, i, j, k) + edge_G<double>(L, G, 2, i, j + 1, k));
            vz = (T)(cdr / (r / 12.0));
        }
    }
    rx[q] = vx;
    ry[q] = vy;
    rz[q] = vz;
}

__global__ void k_validate(Layout L, const float* __restrict__ K, const float* __restrict__ G, int* bad)
{
    Pos p = pos(L);
    if (!p.ok || !is_cell(L, p.i, p.j, p.k)) return;
    long long q = L.at(p.i, p.j, p.k);
    float a = K[q], b = G[q];
    if (!(isfinite(a) && isfinite(b) && a > 0.f && b > 0.f)) atomicAdd(bad, 1);
}

__global__ void k_scatter(Layout L, const float* __restrict__ Kd, const float* __restrict__ Gd, float* K,
                          float* G)
{
    Pos p = pos(L);
    if (!p.ok || !is_cell(L, p.i, p.j, p.k)) return;
    long long d = ((long long)p.k * L.ny + p.j) * L.nx + p.i;
    long long q = L.at(p.i, p.j, p.k);
    K[q] = Kd[d];
    G[q] = Gd[d];
}

// boundary edges held at zero shear stress under boundary mode bc
__device__ __forceinline__ bool fxy(const Layout& L, int bc, int i, int j)
{
    return free_xy(bc, i == 0 || i == L.nx, j == 0 || j == L.ny);
}
__device__ __forceinline__ bool fxz(const Layout& L, int bc, int i, int k)
{
    return free_xz(bc, i == 0 || i == L.nx, k == 0 || k == L.nz);
}
__device__ __forceinline__ bool fyz(const Layout& L, int bc, int j, int k)
{
    return free_yz(bc, j == 0 || j == L.ny, k == 0 || k == L.nz);
}

// strain rates of the fluctuation field plus ebar; w may be a double-word
// value hi + lo (velocity form), whose differences are taken part by part
template <class T>
struct Rates {
    const Layout& L;
    const CaseArgs<T>& c;
    bool zero;
    __device__ __forceinline__ T hi(int f, int i, int j, int k) const { return zero ? (T)0 : c.f[f][L.at(i, j, k)]; }
    __device__ __forceinline__ T lo(int f, int i, int j, int k) const
    {
        const __nv_bfloat16* l = c.lo[f - F_WX];
        return (zero || !l) ? (T)0 : (T)__bfloat162float(l[L.at(i, j, k)]);
    }
    // w(f) at (i1,j1,k1) minus w(f) at (i0,j0,k0); FP64 fields have no low
    // part, so their difference is the plain one (no additions of zeros in
    // the FP64 path, whose arithmetic rate is low on this part)
    __device__ __forceinline__ T dif(int f, int i1, int j1, int k1, int i0, int j0, int k0) const
    {
        if constexpr (sizeof(T) == 8) return hi(f, i1, j1, k1) - hi(f, i0, j0, k0);
        else return (hi(f, i1, j1, k1) - hi(f, i0, j0, k0)) + (lo(f, i1, j1, k1) - lo(f, i0, j0, k0));
    }
    __device__ __forceinline__ T val(int f, int i, int j, int k) const
    {
        if constexpr (sizeof(T) == 8) return hi(f, i, j, k);
        else return hi(f, i, j, k) + lo(f, i, j, k);
    }
    // tangential derivative at integer position q of 0..n between nodes a (q-1) and b (q)
    __device__ __forceinline__ T tang(int q, int n, int f, int ia, int ja, int ka, int ib, int jb, int kb) const
    {
        if (q == 0) return (T)2 * val(f, ib, jb, kb);
        if (q == n) return (T)(-2) * val(f, ia, ja, ka);
        return dif(f, ib, jb, kb, ia, ja, ka);
    }
    __device__ __forceinline__ void cell(int i, int j, int k, T& exx, T& eyy, T& ezz) const
    {
        exx = dif(F_WX, i + 1, j, k, i, j, k) + c.eb.xx;
        eyy = dif(F_WY, i, j + 1, k, i, j, k) + c.eb.yy;
        ezz = dif(F_WZ, i, j, k + 1, i, j, k) + c.eb.zz;
    }
    __device__ __forceinline__ T xy(int i, int j, int k) const
    {
        T a = tang(j, L.ny, F_WX, i, j - 1, k, i, j, k);
        T b = tang(i, L.nx, F_WY, i - 1, j, k, i, j, k);
        return (T)0.5 * (a + b) + c.eb.xy;
    }
    __device__ __forceinline__ T xz(int i, int j, int k) const
    {
        T a = tang(k, L.nz, F_WX, i, j, k - 1, i, j, k);
        T b = tang(i, L.nx, F_WZ, i - 1, j, k, i, j, k);
        return (T)0.5 * (a + b) + c.eb.xz;
    }
    __device__ __forceinline__ T yz(int i, int j, int k) const
    {
        T a = tang(k, L.nz, F_WY, i, j, k - 1, i, j, k);
        T b = tang(j, L.ny, F_WZ, i, j - 1, k, i, j, k);
        return (T)0.5 * (a + b) + c.eb.yz;
    }
};

// ------------------------------------------------------------------ init
// sigma = C(x) : ebar, w = 0 (a homogeneous body is a fixed point)
template <class T>
__global__ void k_init(Layout L, const float* __restrict__ K, const float* __restrict__ G, Cases<T> cs, int bc)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    const CaseArgs<T>& c = cs.c[p.m];
    long long q = L.at(i, j, k);
    T tr = c.eb.xx + c.eb.yy + c.eb.zz;
    T pv = 0, txx = 0, tyy = 0, txy = 0, txz = 0, tyz = 0;
    if (is_cell(L, i, j, k)) {
        T Kc = K[q], Gc = G[q];
        pv = -Kc * tr;
        txx = (T)2 * Gc * (c.eb.xx - tr / (T)3);
        tyy = (T)2 * Gc * (c.eb.yy - tr / (T)3);
    }
    if (k < L.nz && !(fxy(L, bc, i, j))) txy = (T)2 * edge_G<T>(L, G, 0, i, j, k) * c.eb.xy;
    if (j < L.ny && !(fxz(L, bc, i, k))) txz = (T)2 * edge_G<T>(L, G, 1, i, j, k) * c.eb.xz;
    if (i < L.nx && !(fyz(L, bc, j, k))) tyz = (T)2 * edge_G<T>(L, G, 2, i, j, k) * c.eb.yz;
    c.f[F_P][q] = pv;
    c.f[F_TXX][q] = txx;
    c.f[F_TYY][q] = tyy;
    c.f[F_TXY][q] = txy;
    c.f[F_TXZ][q] = txz;
    c.f[F_TYZ][q] = tyz;
    c.f[F_WX][q] = 0;
    c.f[F_WY][q] = 0;
    c.f[F_WZ][q] = 0;
}

// ---------------------------------------------------- stress (in place)
// ELASTIC = false: APT relaxation (Eqs. A2ssP, A23ssP2 with K~ = K, G~ = G):
//   x_new = x_old + a (M rate - x_old), a = theta / (1 + theta)
// ELASTIC = true: sigma = C : eps(ebar.x + w) written to `dst` (residual)
template <class T, bool ELASTIC>
__global__ void k_stress(Layout L, const float* __restrict__ K, const float* __restrict__ G, Cases<T> cs,
                         Cases<T> dst, Relax<T> rp, int bc, int zero_w)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    const CaseArgs<T>& c = cs.c[p.m];
    T* const* o = ELASTIC ? dst.c[p.m].f : c.f;
    Rates<T> r{L, c, ELASTIC && zero_w != 0};
    long long q = L.at(i, j, k);
    if (is_cell(L, i, j, k)) {
        T exx, eyy, ezz;
        r.cell(i, j, k, exx, eyy, ezz);
        T div = exx + eyy + ezz;
        T Kc = K[q], Gc = G[q];
        if (ELASTIC) {
            o[F_P][q] = -Kc * div;
            o[F_TXX][q] = (T)2 * Gc * (exx - div / (T)3);
            o[F_TYY][q] = (T)2 * Gc * (eyy - div / (T)3);
        } else {
            T po = c.f[F_P][q], xo = c.f[F_TXX][q], yo = c.f[F_TYY][q];
            o[F_P][q] = po + rp.a * (-Kc * div - po);
            o[F_TXX][q] = xo + rp.a * ((T)2 * Gc * (exx - div / (T)3) - xo);
            o[F_TYY][q] = yo + rp.a * ((T)2 * Gc * (eyy - div / (T)3) - yo);
        }
    }
    if (k < L.nz) {
        if (fxy(L, bc, i, j)) {
            if (ELASTIC) o[F_TXY][q] = 0;
        } else {
            T Ge = edge_G<T>(L, G, 0, i, j, k), e = r.xy(i, j, k);
            o[F_TXY][q] = ELASTIC ? (T)2 * Ge * e : c.f[F_TXY][q] + rp.a * ((T)2 * Ge * e - c.f[F_TXY][q]);
        }
    }
    if (j < L.ny) {
        if (fxz(L, bc, i, k)) {
            if (ELASTIC) o[F_TXZ][q] = 0;
        } else {
            T Ge = edge_G<T>(L, G, 1, i, j, k), e = r.xz(i, j, k);
            o[F_TXZ][q] = ELASTIC ? (T)2 * Ge * e : c.f[F_TXZ][q] + rp.a * ((T)2 * Ge * e - c.f[F_TXZ][q]);
        }
    }
    if (i < L.nx) {
        if (fyz(L, bc, j, k)) {
            if (ELASTIC) o[F_TYZ][q] = 0;
        } else {
            T Ge = edge_G<T>(L, G, 2, i, j, k), e = r.yz(i, j, k);
            o[F_TYZ][q] = ELASTIC ? (T)2 * Ge * e : c.f[F_TYZ][q] + rp.a * ((T)2 * Ge * e - c.f[F_TYZ][q]);
        }
    }
}

// divergence of sigma = -p I + tau at the three velocity nodes of (i,j,k)
template <class T>
struct Div {
    const Layout& L;
    T* const* s;   // p, txx, tyy, txy, txz, tyz
    __device__ __forceinline__ T v(int f, int i, int j, int k) const { return s[f][L.at(i, j, k)]; }
    __device__ __forceinline__ T sxx(int i, int j, int k) const { return -v(F_P, i, j, k) + v(F_TXX, i, j, k); }
    __device__ __forceinline__ T syy(int i, int j, int k) const { return -v(F_P, i, j, k) + v(F_TYY, i, j, k); }
    __device__ __forceinline__ T szz(int i, int j, int k) const
    {
        return -v(F_P, i, j, k) - v(F_TXX, i, j, k) - v(F_TYY, i, j, k);
    }
    __device__ __forceinline__ T x(int i, int j, int k) const
    {
        return (sxx(i, j, k) - sxx(i - 1, j, k)) + (v(F_TXY, i, j + 1, k) - v(F_TXY, i, j, k))
             + (v(F_TXZ, i, j, k + 1) - v(F_TXZ, i, j, k));
    }
    __device__ __forceinline__ T y(int i, int j, int k) const
    {
        return (v(F_TXY, i + 1, j, k) - v(F_TXY, i, j, k)) + (syy(i, j, k) - syy(i, j - 1, k))
             + (v(F_TYZ, i, j, k + 1) - v(F_TYZ, i, j, k));
    }
    __device__ __forceinline__ T z(int i, int j, int k) const
    {
        return (v(F_TXZ, i + 1, j, k) - v(F_TXZ, i, j, k)) + (v(F_TYZ, i, j + 1, k) - v(F_TYZ, i, j, k))
             + (szz(i, j, k) - szz(i, j, k - 1));
    }
};

// rho~ dw/dt~ = div sigma at interior velocity nodes (in place)
template <class T>
__global__ void k_velocity(Layout L, const T* __restrict__ rx, const T* __restrict__ ry,
                           const T* __restrict__ rz, Cases<T> cs)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    if (!is_cell(L, i, j, k)) return;
    const CaseArgs<T>& c = cs.c[p.m];
    Div<T> d{L, c.f};
    long long q = L.at(i, j, k);
    if (i > 0) c.f[F_WX][q] += rx[q] * d.x(i, j, k);
    if (j > 0) c.f[F_WY][q] += ry[q] * d.y(i, j, k);
    if (k > 0) c.f[F_WZ][q] += rz[q] * d.z(i, j, k);
}

// velocity form: u_{-1} = r div T(w_0) from the stresses in `src`, written to
// the u slots of `dst` (zero at Dirichlet and padding nodes)
template <class T>
__global__ void k_uinit(Layout L, const T* __restrict__ rx, const T* __restrict__ ry, const T* __restrict__ rz,
                        Cases<T> src, Cases<T> dst)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    long long q = L.at(i, j, k);
    T ux = 0, uy = 0, uz = 0;
    if (is_cell(L, i, j, k)) {
        Div<T> d{L, src.c[p.m].f};
        if (i > 0) ux = rx[q] * d.x(i, j, k);
        if (j > 0) uy = ry[q] * d.y(i, j, k);
        if (k > 0) uz = rz[q] * d.z(i, j, k);
    }
    dst.c[p.m].f[F_UX][q] = ux;
    dst.c[p.m].f[F_UY][q] = uy;
    dst.c[p.m].f[F_UZ][q] = uz;
}

// ------------------------------------------------------- block reduction
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* out)
{
    __shared__ double sh[32][NV];
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int a = 0; a < NV; ++a)
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < NV; ++a) sh[warp][a] = v[a];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            double t = lane < nwarp ? sh[lane][a] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) out[a] = t;
        }
    }
}

template <class T>
__global__ void k_divnorm(Layout L, Cases<T> s, double* partials, int nblk, int nzr)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int m = blockIdx.z / nzr, kz = blockIdx.z % nzr;
    double acc[1] = { 0.0 };
    if (i <= L.nx && j <= L.ny) {
        Div<T> d{L, s.c[m].f};
        for (int k = L.kz0 + kz; k < L.kz1 && k < L.nz; k += nzr) {
            if (!is_cell(L, i, j, k)) continue;
            if (i > 0) { double r = (double)d.x(i, j, k); acc[0] += r * r; }
            if (j > 0) { double r = (double)d.y(i, j, k); acc[0] += r * r; }
            if (k > 0) { double r = (double)d.z(i, j, k); acc[0] += r * r; }
        }
    }
    const int b = (kz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_sum<1>(acc, partials + (size_t)m * nblk + b);
}

// fixed-order second pass: one block per case sums `nblk` partials of NV values
template <int NV>
__global__ void k_reduce_partials(const double* __restrict__ partials, int nblk, double* out)
{
    const double* src = partials + (size_t)blockIdx.x * nblk * NV;
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] += src[(size_t)b * NV + a];
    block_sum<NV>(v, out + (size_t)blockIdx.x * NV);
}

// --------------------------------------------------------- volume averages
// 12 sums per case: sigma (xx, yy, zz, yz, xz, xy) and engineering strain,
// cells weight 1, edges the trapezoid weight (1/2 per boundary direction)
template <class T, bool ELASTIC>
__global__ void k_average(Layout L, const float* __restrict__ K, const float* __restrict__ G, Cases<T> cs, int bc,
                          double* partials, int nblk, int nzr)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int m = blockIdx.z / nzr, kz = blockIdx.z % nzr;
    double a[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) a[t] = 0.0;
    if (i <= L.nx && j <= L.ny) {
        const CaseArgs<T>& c = cs.c[m];
        Rates<T> r{L, c, false};
        const double wi = (i == 0 || i == L.nx) ? 0.5 : 1.0;
        const double wj = (j == 0 || j == L.ny) ? 0.5 : 1.0;
        for (int k = L.kz0 + kz; k < L.kz1 && k <= L.nz; k += nzr) {
            long long q = L.at(i, j, k);
            if (is_cell(L, i, j, k)) {
                T exx, eyy, ezz;
                r.cell(i, j, k, exx, eyy, ezz);
                if (ELASTIC) {
                    double dv = (double)exx + (double)eyy + (double)ezz;
                    double lam = ((double)K[q] - 2.0 / 3.0 * (double)G[q]) * dv, g2 = 2.0 * (double)G[q];
                    a[0] += lam + g2 * exx;
                    a[1] += lam + g2 * eyy;
                    a[2] += lam + g2 * ezz;
                } else {
                    double pv = c.f[F_P][q], txx = c.f[F_TXX][q], tyy = c.f[F_TYY][q];
                    a[0] += -pv + txx;
                    a[1] += -pv + tyy;
                    a[2] += -pv - txx - tyy;
                }
                a[6] += exx;
                a[7] += eyy;
                a[8] += ezz;
            }
            const double wk = (k + L.zoff == 0 || k + L.zoff == L.nzg) ? 0.5 : 1.0;
            if (i < L.nx) {
                double e = r.yz(i, j, k);
                double s = ELASTIC ? ((fyz(L, bc, j, k)) ? 0.0 : 2.0 * edge_G<double>(L, G, 2, i, j, k) * e)
                                   : (double)c.f[F_TYZ][q];
                a[3] += wj * wk * s;
                a[9] += wj * wk * 2.0 * e;
            }
            if (j < L.ny) {
                double e = r.xz(i, j, k);
                double s = ELASTIC ? ((fxz(L, bc, i, k)) ? 0.0 : 2.0 * edge_G<double>(L, G, 1, i, j, k) * e)
                                   : (double)c.f[F_TXZ][q];
                a[4] += wi * wk * s;
                a[10] += wi * wk * 2.0 * e;
            }
            if (k < L.nz) {
                double e = r.xy(i, j, k);
                double s = ELASTIC ? ((fxy(L, bc, i, j)) ? 0.0 : 2.0 * edge_G<double>(L, G, 0, i, j, k) * e)
                                   : (double)c.f[F_TXY][q];
                a[5] += wi * wj * s;
                a[11] += wi * wj * 2.0 * e;
            }
        }
    }
    const int b = (kz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_sum<12>(a, partials + ((size_t)m * nblk + b) * 12);
}


// ---------------------------------------------------------- adjoint gradient
// J = sum_ab W_ab C_ab with C_ab = a(u^a, u^b)/V at equilibrium; the operator
// is symmetric, so dJ/dp = (1/V) sum_ab W_ab a_p(u^a, u^b) with the forward
// fields (no second solve).  Per cell:
//   dJ/dK = (1/V) sum_ab W_ab div^a div^b
//   dJ/dG = (1/V) sum_ab W_ab [2 sum_ii dev^a_ii dev^b_ii
//                               + sum_{12 edges e of the cell} f_e e^a_e e^b_e]
// where f_e = 4 omega_e / n_e = 1 (edge weight over adjacent-cell count), and
// 0 for boundary edges under rollers.  W is symmetrised on the host.
template <class T>
__device__ __forceinline__ T quad6(const double* __restrict__ W, const T (&x)[6])
{
    T s = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        T t = 0;
#pragma unroll
        for (int b = 0; b < 6; ++b) t += (T)W[a * 6 + b] * x[b];
        s += x[a] * t;
    }
    return s;
}

template <class T>
__global__ void k_grad(Layout L, Cases<T> cs, const double* __restrict__ W, float* dK, float* dG, int bc)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    if (!is_cell(L, i, j, k)) return;
    T dv[6], d0[6], d1[6], d2[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        Rates<T> r{L, cs.c[m], false};
        T exx, eyy, ezz;
        r.cell(i, j, k, exx, eyy, ezz);
        T dvm = exx + eyy + ezz;
        dv[m] = dvm;
        d0[m] = exx - dvm / (T)3;
        d1[m] = eyy - dvm / (T)3;
        d2[m] = ezz - dvm / (T)3;
    }
    T gK = quad6<T>(W, dv);
    T gG = (T)2 * (quad6<T>(W, d0) + quad6<T>(W, d1) + quad6<T>(W, d2));
    T e[6];
    // xy edges (i..i+1, j..j+1, k)
    for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b) {
            if (fxy(L, bc, i + a, j + b)) continue;
#pragma unroll
            for (int m = 0; m < 6; ++m) e[m] = Rates<T>{L, cs.c[m], false}.xy(i + a, j + b, k);
            gG += quad6<T>(W, e);
        }
    // xz edges (i..i+1, j, k..k+1)
    for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b) {
            if (fxz(L, bc, i + a, k + b)) continue;
#pragma unroll
            for (int m = 0; m < 6; ++m) e[m] = Rates<T>{L, cs.c[m], false}.xz(i + a, j, k + b);
            gG += quad6<T>(W, e);
        }
    // yz edges (i, j..j+1, k..k+1)
    for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b) {
            if (fyz(L, bc, j + a, k + b)) continue;
#pragma unroll
            for (int m = 0; m < 6; ++m) e[m] = Rates<T>{L, cs.c[m], false}.yz(i, j + a, k + b);
            gG += quad6<T>(W, e);
        }
    const double V = (double)L.nx * L.ny * L.nz;
    long long d = ((long long)k * L.ny + j) * L.nx + i;
    dK[d] = (float)((double)gK / V);
    dG[d] = (float)((double)gG / V);
}

template <class T>
__global__ void k_gather(Layout L, const T* __restrict__ f, double* dense)
{
    Pos p = pos(L);
    if (!p.ok) return;
    dense[((long long)p.k * (L.ny + 1) + p.j) * (L.nx + 1) + p.i] = (double)f[L.at(p.i, p.j, p.k)];
}

// velocity form export: 0-5 elastic stress of w (p, tau_xx, tau_yy, tau_xy,
// tau_xz, tau_yz), 6-8 w = hi + lo, 9-11 u
__global__ void k_gather_vform(Layout L, const float* __restrict__ K, const float* __restrict__ G,
                               CaseArgs<float> c, int field, int bc, double* dense)
{
    Pos p = pos(L);
    if (!p.ok) return;
    const int i = p.i, j = p.j, k = p.k;
    long long q = L.at(i, j, k);
    double v = 0.0;
    Rates<float> rf{L, c, false};
    if (field >= 9) {
        v = c.f[field - 9][q];
    } else if (field >= 6) {
        v = (double)c.f[field][q] + (double)(c.lo[field - 6] ? __bfloat162float(c.lo[field - 6][q]) : 0.f);
    } else if (field <= 2) {
        if (is_cell(L, i, j, k)) {
            float exx, eyy, ezz;
            rf.cell(i, j, k, exx, eyy, ezz);
            double dv = (double)exx + eyy + ezz;
            if (field == 0) v = -(double)K[q] * dv;
            else v = 2.0 * (double)G[q] * ((field == 1 ? exx : eyy) - dv / 3.0);
        }
    } else if (field == 3) {
        if (k < L.nz && !(fxy(L, bc, i, j))) v = 2.0 * edge_G<double>(L, G, 0, i, j, k) * rf.xy(i, j, k);
    } else if (field == 4) {
        if (j < L.ny && !(fxz(L, bc, i, k))) v = 2.0 * edge_G<double>(L, G, 1, i, j, k) * rf.xz(i, j, k);
    } else {
        if (i < L.nx && !(fyz(L, bc, j, k))) v = 2.0 * edge_G<double>(L, G, 2, i, j, k) * rf.yz(i, j, k);
    }
    dense[((long long)k * (L.ny + 1) + j) * (L.nx + 1) + i] = v;
}

}  // namespace

void launch_gather_vform(const Layout& L, const float* K, const float* G, const CaseArgs<float>& c, int field,
                         int bc, double* dense, cudaStream_t st)
{
    k_gather_vform<<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, K, G, c, field, bc, dense);
}

void launch_reduce(const double* partials, int nblk, int ncases, double* out, cudaStream_t st)
{
    k_reduce_partials<1><<<ncases, 1024, 0, st>>>(partials, nblk, out);
}

int reduce_blocks(const Layout& L)
{
    dim3 g = grid_red(L, 1);
    return (int)(g.x * g.y * g.z);
}

template <class T>
void launch_node_coef(const Layout& L, const float* K, const float* G, T* rx, T* ry, T* rz, double cdr,
                      cudaStream_t st)
{
    k_node_coef<T><<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, K, G, rx, ry, rz, cdr);
}

void launch_validate(const Layout& L, const float* K, const float* G, int* bad, cudaStream_t st)
{
    k_validate<<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, K, G, bad);
}

void launch_scatter_moduli(const Layout& L, const float* Kd, const float* Gd, float* K, float* G,
                           cudaStream_t st)
{
    k_scatter<<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, Kd, Gd, K, G);
}

template <class T>
void launch_init(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases, int ncases,
                 int bc, cudaStream_t st)
{
    k_init<T><<<grid_for(L, ncases), dim3(BX, BY), 0, st>>>(L, K, G, pack(cases, ncases), bc);
}

template <class T>
void launch_plain_sweep(const Layout& L, const float* K, const float* G, const T* rx, const T* ry,
                        const T* rz, const CaseArgs<T>* cases, int ncases, Relax<T> rp, int bc,
                        cudaStream_t st)
{
    Cases<T> cs = pack(cases, ncases);
    k_stress<T, false><<<grid_for(L, ncases), dim3(BX, BY), 0, st>>>(L, K, G, cs, cs, rp, bc, 0);
    k_velocity<T><<<grid_for(L, ncases), dim3(BX, BY), 0, st>>>(L, rx, ry, rz, cs);
}

template <class T>
void launch_residual(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases,
                     const CaseArgs<T>* scratch, int ncases, int bc, int zero_w, double* partials,
                     int nblk_cap, double* out, cudaStream_t st)
{
    Cases<T> cs = pack(cases, ncases), sc = pack(scratch, ncases);
    Relax<T> rp{0};
    k_stress<T, true><<<grid_for(L, ncases), dim3(BX, BY), 0, st>>>(L, K, G, cs, sc, rp, bc, zero_w);
    int nblk = reduce_blocks(L);
    (void)nblk_cap;
    k_divnorm<T><<<grid_red(L, ncases), dim3(BX, BY), 0, st>>>(L, sc, partials, nblk, zr(L));
    k_reduce_partials<1><<<ncases, 1024, 0, st>>>(partials, nblk, out);
}

template <class T>
void launch_elastic_stress(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases,
                           const CaseArgs<T>* dst, int ncases, int bc, cudaStream_t st)
{
    Relax<T> rp{0};
    k_stress<T, true><<<grid_for(L, ncases), dim3(BX, BY), 0, st>>>(L, K, G, pack(cases, ncases),
                                                                     pack(dst, ncases), rp, bc, 0);
}

template <class T>
void launch_uinit(const Layout& L, const T* rx, const T* ry, const T* rz, const CaseArgs<T>* src,
                  const CaseArgs<T>* dst, int ncases, cudaStream_t st)
{
    k_uinit<T><<<grid_for(L, ncases), dim3(BX, BY), 0, st>>>(L, rx, ry, rz, pack(src, ncases), pack(dst, ncases));
}

template <class T>
void launch_average(const Layout& L, const float* K, const float* G, const CaseArgs<T>* cases, int ncases,
                    int elastic, int bc, double* partials, int nblk_cap, double* out, cudaStream_t st)
{
    int nblk = reduce_blocks(L);
    (void)nblk_cap;
    if (elastic)
        k_average<T, true><<<grid_red(L, ncases), dim3(BX, BY), 0, st>>>(L, K, G, pack(cases, ncases), bc, partials,
                                                                          nblk, zr(L));
    else
        k_average<T, false><<<grid_red(L, ncases), dim3(BX, BY), 0, st>>>(L, K, G, pack(cases, ncases), bc,
                                                                           partials, nblk, zr(L));
    k_reduce_partials<12><<<ncases, 1024, 0, st>>>(partials, nblk, out);
}

template <class T>
void launch_gather_field(const Layout& L, const T* f, double* dense, cudaStream_t st)
{
    k_gather<T><<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, f, dense);
}

void launch_grad(const Layout& L, const float* K, const float* G, const CaseArgs<float>* cases32,
                 const CaseArgs<double>* cases64, const double* wsym, float* dK, float* dG, int bc,
                 cudaStream_t st)
{
    (void)K;
    (void)G;
    if (cases64)
        k_grad<double><<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, pack(cases64, 6), wsym, dK, dG, bc);
    else
        k_grad<float><<<grid_for(L, 1), dim3(BX, BY), 0, st>>>(L, pack(cases32, 6), wsym, dK, dG, bc);
}

#define CE_INST(T)                                                                                         \
    template void launch_node_coef<T>(const Layout&, const float*, const float*, T*, T*, T*, double,       \
                                      cudaStream_t);                                                       \
    template void launch_init<T>(const Layout&, const float*, const float*, const CaseArgs<T>*, int, int,  \
                                 cudaStream_t);                                                            \
    template void launch_plain_sweep<T>(const Layout&, const float*, const float*, const T*, const T*,     \
                                        const T*, const CaseArgs<T>*, int, Relax<T>, int, cudaStream_t);   \
    template void launch_residual<T>(const Layout&, const float*, const float*, const CaseArgs<T>*,        \
                                     const CaseArgs<T>*, int, int, int, double*, int, double*,             \
                                     cudaStream_t);                                                        \
    template void launch_average<T>(const Layout&, const float*, const float*, const CaseArgs<T>*, int,    \
                                    int, int, double*, int, double*, cudaStream_t);                        \
    template void launch_gather_field<T>(const Layout&, const T*, double*, cudaStream_t);                 \
    template void launch_elastic_stress<T>(const Layout&, const float*, const float*, const CaseArgs<T>*,  \
                                           const CaseArgs<T>*, int, int, cudaStream_t);                     \
    template void launch_uinit<T>(const Layout&, const T*, const T*, const T*, const CaseArgs<T>*,          \
                                  const CaseArgs<T>*, int, cudaStream_t);
CE_INST(float)
CE_INST(double)

}  // namespace ce
