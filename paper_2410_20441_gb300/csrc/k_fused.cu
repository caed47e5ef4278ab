// Fused FP32 pseudo-time sweep for all load cases of one image, in velocity
// form with a double-word displacement fluctuation.
//
// The paper's step (Sec. 3.2) relaxes every stress towards its elastic value
// T(w) = C : eps(ebar.x + w) (Eqs. A2ssP, A23ssP2) and then moves the
// velocities with the divergence of the new stresses (Eq. 11111).  With the
// numerical moduli equal to the material ones (K~ = K, G~ = G, Sec. 3.1) the
// relaxation factor a = theta / (1 + theta) is the same at every stress
// point, so the relaxed stress is a linear filter of past elastic stresses and
// the step is exactly (in exact arithmetic) the second-order recurrence
//
//     u_n     = (1 - a) u_{n-1} + a r div T(w_n)        (r = dt~/rho~ per node)
//     w_{n+1} = w_n + u_n,                 u_{-1} = r div T(w_0) at the start.
//
// Precision.  A stored FP32 stress stops moving once a |sigma - T| falls below
// half an ulp of sigma, which leaves a lag of ulp/(2a) (a ~ 1e-2) and floors
// the residual near 1e-4; here T is recomputed from w every sweep instead.
// w itself is kept as hi (FP32) + lo (BF16) with |lo| <= ulp(hi)/2, updated by
// an error-free two-sum, and strains are formed as (hi difference) + (lo
// difference); an FP32 w alone would floor the residual near 1e-5 at 191^3.
// The elastic stress is split as T = T(0) + T'(w) with T(0) = C : ebar and
// T'(w) = C : eps(w), and the divergence is formed part by part: T(0) is
// bitwise equal wherever the moduli are, so its differences vanish exactly
// away from interfaces, and T' carries only the (small) fluctuation.
// Per load case and voxel the sweep moves 30 bytes in (u, w hi, w lo) and 30
// bytes out.
//
// Design (memory-bound stencil, no tensor-core work):
//  * A block of 32 x TY threads owns the interior (30 x (TY-2)) of its tile of
//    index-grid columns and recomputes the one-column halo of elastic stresses
//    itself (overlapped tiling), so one sweep is one launch.  Neighbouring
//    tiles read each other's old values, so the state is ping-ponged.
//  * The block marches in z over a chunk of planes.  Per plane it loads the
//    old state, K, G and dt~/rho~ once (coalesced rows), exchanges w and G
//    through shared memory, forms T at the cells and edges of the plane,
//    exchanges T, and updates (w_z, u_z) of the plane and (w_x, u_x),
//    (w_y, u_y) of the previous plane, whose z-flux needs T of this plane.
//    z-neighbours stay in registers, so every field is read once per sweep.
//  * Load cases are processed one after another inside the block; the
//    material rows of the chunk are re-read from L2.
//  * On check sweeps the same div T(w_n) gives the residual: each block adds
//    its squares in FP64 and writes one partial per load case (a fixed-order
//    second pass sums them), so checking costs no extra pass over memory.
#include "ce_internal.h"

namespace ce {

namespace {

constexpr int TX = 32;

// derivative of a boundary-tangential component at integer position q of
// 0..n from nodes lo-side (q-1) and hi-side (q), each a double-word (h, l)
__device__ __forceinline__ float tdw(int q, int n, float ha, float la, float hb, float lb)
{
    return q == 0 ? 2.f * (hb + lb) : (q == n ? -2.f * (ha + la) : (hb - ha) + (lb - la));
}

// (h, l) + u with an error-free two-sum, renormalised so that |l| <= ulp(h)/2
__device__ __forceinline__ void dw_add(float h, float l, float u, float& ho, __nv_bfloat16& lo)
{
    float s = h + u;
    float bp = s - h;
    float e = (h - (s - bp)) + (u - bp);
    float l2 = l + e;
    float h2 = s + l2;
    float l3 = l2 - (h2 - s);
    ho = h2;
    lo = __float2bfloat16_rn(l3);
}

template <int TY, bool CHECK>
__global__ void __launch_bounds__(TX* TY, 1024 / (TX * TY) > 2 ? 2 : 1024 / (TX * TY))
    k_fused(const __grid_constant__ FusedArgs a, int zc)
{
    __shared__ float s_wxh[TY][TX], s_wyh[TY][TX], s_wzh[TY][TX];
    __shared__ float s_wxl[TY][TX], s_wyl[TY][TX], s_wzl[TY][TX];
    __shared__ float s_G[2][TY][TX];
    __shared__ float s_sxx[TY][TX], s_syy[TY][TX], s_txy[TY][TX], s_txz[TY][TX], s_tyz[TY][TX];
    __shared__ float s_bxx[TY][TX], s_byy[TY][TX], s_bxy[TY][TX], s_bxz[TY][TX], s_byz[TY][TX];
    __shared__ double s_red[TY];

    const Layout& L = a.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = (int)blockIdx.x * (TX - 2) - 1 + tx;
    const int j = (int)blockIdx.y * (TY - 2) - 1 + ty;
    const int k0 = (int)blockIdx.z * zc;
    const int k1 = min(k0 + zc, nz + 1);
    const bool ing = i >= 0 && i <= nx && j >= 0 && j <= ny;
    const bool own = ing && tx >= 1 && tx <= TX - 2 && ty >= 1 && ty <= TY - 2;
    const bool cellc = ing && i < nx && j < ny;
    const bool upd_x = own && i > 0 && i < nx && j < ny;
    const bool upd_y = own && i < nx && j > 0 && j < ny;
    const bool upd_zc = own && i < nx && j < ny;
    const bool rol = a.bc == CE_BC_ROLLER;
    // existence of the cells around this column's edges
    const bool cxm = i - 1 >= 0 && i - 1 < nx, cx0 = i < nx;   // cells i-1, i
    const bool cym = j - 1 >= 0 && j - 1 < ny, cy0 = j < ny;   // cells j-1, j
    const long long plane = L.plane;
    const long long fsize = L.fsize;
    const long long col = ing ? (long long)j * L.pitch + i : 0;
    const float ra = a.a, rb = 1.f - a.a;
    const int s_begin = k0 > 0 ? k0 - 1 : 0;
    const int s_end = k1 <= nz ? k1 : nz;
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int nblk = gridDim.x * gridDim.y * gridDim.z;

    for (int m = 0; m < a.ncase; ++m) {
        const float* __restrict__ iUX = a.in[m][F_UX];
        const float* __restrict__ iUY = a.in[m][F_UY];
        const float* __restrict__ iUZ = a.in[m][F_UZ];
        const float* __restrict__ iWX = a.in[m][F_WX];
        const float* __restrict__ iWY = a.in[m][F_WY];
        const float* __restrict__ iWZ = a.in[m][F_WZ];
        const __nv_bfloat16* __restrict__ iLX = (const __nv_bfloat16*)a.in[m][F_WLO_XY];
        const __nv_bfloat16* __restrict__ iLY = iLX + fsize;
        const __nv_bfloat16* __restrict__ iLZ = (const __nv_bfloat16*)a.in[m][F_WLO_Z];
        float* __restrict__ oUX = a.out[m][F_UX];
        float* __restrict__ oUY = a.out[m][F_UY];
        float* __restrict__ oUZ = a.out[m][F_UZ];
        float* __restrict__ oWX = a.out[m][F_WX];
        float* __restrict__ oWY = a.out[m][F_WY];
        float* __restrict__ oWZ = a.out[m][F_WZ];
        __nv_bfloat16* __restrict__ oLX = (__nv_bfloat16*)a.out[m][F_WLO_XY];
        __nv_bfloat16* __restrict__ oLY = oLX + fsize;
        __nv_bfloat16* __restrict__ oLZ = (__nv_bfloat16*)a.out[m][F_WLO_Z];
        const Ebar<float> eb = a.eb[m];
        const float trb = eb.xx + eb.yy + eb.zz;

        float wzh_cur = 0.f, wzl_cur = 0.f;
        if (ing && s_begin <= nz) {
            wzh_cur = iWZ[s_begin * plane + col];
            wzl_cur = __bfloat162float(iLZ[s_begin * plane + col]);
        }
        float wxh_prev = 0.f, wxl_prev = 0.f, wyh_prev = 0.f, wyl_prev = 0.f, ux_prev = 0.f, uy_prev = 0.f;
        float szz_prev = 0.f, txz_prev = 0.f, tyz_prev = 0.f;
        float bzz_prev = 0.f, bxz_prev = 0.f, byz_prev = 0.f;
        float rx_prev = 0.f, ry_prev = 0.f, dxy_x = 0.f, dxy_y = 0.f, dbxy_x = 0.f, dbxy_y = 0.f;
        double acc = 0.0;

        for (int s = s_begin; s <= s_end; ++s) {
            const bool warm = s < k0;
            const bool tail = s >= k1;
            const long long q = s * plane + col;
            // ---- old state of plane s
            float wxh = 0.f, wxl = 0.f, wyh = 0.f, wyl = 0.f, wzh_n = 0.f, wzl_n = 0.f;
            float ux_o = 0.f, uy_o = 0.f, uz_o = 0.f;
            float Kc = 0.f, Gc = 0.f, rxv = 0.f, ryv = 0.f, rzv = 0.f;
            if (ing) {
                wxh = iWX[q];
                wyh = iWY[q];
                wxl = __bfloat162float(iLX[q]);
                wyl = __bfloat162float(iLY[q]);
                if (s + 1 <= nz) {
                    wzh_n = iWZ[q + plane];
                    wzl_n = __bfloat162float(iLZ[q + plane]);
                }
                ux_o = iUX[q];
                uy_o = iUY[q];
                uz_o = iUZ[q];
                Kc = a.K[q];
                Gc = a.G[q];
                rxv = a.rx[q];
                ryv = a.ry[q];
                rzv = a.rz[q];
            }
            s_wxh[ty][tx] = wxh;
            s_wxl[ty][tx] = wxl;
            s_wyh[ty][tx] = wyh;
            s_wyl[ty][tx] = wyl;
            s_wzh[ty][tx] = wzh_cur;
            s_wzl[ty][tx] = wzl_cur;
            s_G[s & 1][ty][tx] = Gc;
            __syncthreads();

            // ---- elastic stresses at plane s: T' = C : eps(w) (s*_n, t*_n) and
            //      T(0) = C : ebar (b*_n)
            float sxx_n = 0.f, syy_n = 0.f, szz_n = 0.f, txy_n = 0.f, txz_n = 0.f, tyz_n = 0.f;
            float bxx_n = 0.f, byy_n = 0.f, bzz_n = 0.f, bxy_n = 0.f, bxz_n = 0.f, byz_n = 0.f;
            if (cellc && s < nz && tx < TX - 1 && ty < TY - 1) {
                float exx = (s_wxh[ty][tx + 1] - wxh) + (s_wxl[ty][tx + 1] - wxl);
                float eyy = (s_wyh[ty + 1][tx] - wyh) + (s_wyl[ty + 1][tx] - wyl);
                float ezz = (wzh_n - wzh_cur) + (wzl_n - wzl_cur);
                float lk = Kc - (2.f / 3.f) * Gc;
                float lam = lk * (exx + eyy + ezz);
                float g2 = 2.f * Gc;
                sxx_n = lam + g2 * exx;
                syy_n = lam + g2 * eyy;
                szz_n = lam + g2 * ezz;
                float lb = lk * trb;
                bxx_n = lb + g2 * eb.xx;
                byy_n = lb + g2 * eb.yy;
                bzz_n = lb + g2 * eb.zz;
            }
            if (ing && s < nz && tx > 0 && ty > 0 && !(rol && (i == 0 || i == nx || j == 0 || j == ny))) {
                const float(&g)[TY][TX] = s_G[s & 1];
                float sg = 0.f;
                int n = 0;
                if (cxm && cym) { sg += g[ty - 1][tx - 1]; ++n; }
                if (cx0 && cym) { sg += g[ty - 1][tx]; ++n; }
                if (cxm && cy0) { sg += g[ty][tx - 1]; ++n; }
                if (cx0 && cy0) { sg += g[ty][tx]; ++n; }
                float e = 0.5f * (tdw(j, ny, s_wxh[ty - 1][tx], s_wxl[ty - 1][tx], wxh, wxl)
                                  + tdw(i, nx, s_wyh[ty][tx - 1], s_wyl[ty][tx - 1], wyh, wyl));
                float g2 = 2.f * (sg / (float)n);
                txy_n = g2 * e;
                bxy_n = g2 * eb.xy;
            }
            const bool czm = s - 1 >= 0, cz0 = s < nz;   // cells s-1, s
            if (ing && j < ny && tx > 0 && !(rol && (i == 0 || i == nx || s == 0 || s == nz))) {
                float sg = 0.f;
                int n = 0;
                if (cxm && czm) { sg += s_G[(s - 1) & 1][ty][tx - 1]; ++n; }
                if (cx0 && czm) { sg += s_G[(s - 1) & 1][ty][tx]; ++n; }
                if (cxm && cz0) { sg += s_G[s & 1][ty][tx - 1]; ++n; }
                if (cx0 && cz0) { sg += s_G[s & 1][ty][tx]; ++n; }
                float e = 0.5f * (tdw(s, nz, wxh_prev, wxl_prev, wxh, wxl)
                                  + tdw(i, nx, s_wzh[ty][tx - 1], s_wzl[ty][tx - 1], wzh_cur, wzl_cur));
                float g2 = 2.f * (sg / (float)n);
                txz_n = g2 * e;
                bxz_n = g2 * eb.xz;
            }
            if (ing && i < nx && ty > 0 && !(rol && (j == 0 || j == ny || s == 0 || s == nz))) {
                float sg = 0.f;
                int n = 0;
                if (cym && czm) { sg += s_G[(s - 1) & 1][ty - 1][tx]; ++n; }
                if (cy0 && czm) { sg += s_G[(s - 1) & 1][ty][tx]; ++n; }
                if (cym && cz0) { sg += s_G[s & 1][ty - 1][tx]; ++n; }
                if (cy0 && cz0) { sg += s_G[s & 1][ty][tx]; ++n; }
                float e = 0.5f * (tdw(s, nz, wyh_prev, wyl_prev, wyh, wyl)
                                  + tdw(j, ny, s_wzh[ty - 1][tx], s_wzl[ty - 1][tx], wzh_cur, wzl_cur));
                float g2 = 2.f * (sg / (float)n);
                tyz_n = g2 * e;
                byz_n = g2 * eb.yz;
            }
            s_sxx[ty][tx] = sxx_n;
            s_syy[ty][tx] = syy_n;
            s_txy[ty][tx] = txy_n;
            s_txz[ty][tx] = txz_n;
            s_tyz[ty][tx] = tyz_n;
            s_bxx[ty][tx] = bxx_n;
            s_byy[ty][tx] = byy_n;
            s_bxy[ty][tx] = bxy_n;
            s_bxz[ty][tx] = bxz_n;
            s_byz[ty][tx] = byz_n;
            __syncthreads();

            // ---- velocity recurrence and stores
            if (own && !warm) {
                if (!tail && upd_zc && s > 0 && s < nz) {
                    float d = ((s_txz[ty][tx + 1] - txz_n) + (s_tyz[ty + 1][tx] - tyz_n) + (szz_n - szz_prev))
                            + ((s_bxz[ty][tx + 1] - bxz_n) + (s_byz[ty + 1][tx] - byz_n) + (bzz_n - bzz_prev));
                    float un = rb * uz_o + ra * rzv * d;
                    float h;
                    __nv_bfloat16 l;
                    dw_add(wzh_cur, wzl_cur, un, h, l);
                    oUZ[q] = un;
                    oWZ[q] = h;
                    oLZ[q] = l;
                    if (CHECK) acc += (double)d * (double)d;
                }
                if (s > k0) {
                    const long long qm = q - plane;
                    if (upd_x) {
                        float d = (dxy_x + (txz_n - txz_prev)) + (dbxy_x + (bxz_n - bxz_prev));
                        float un = rb * ux_prev + ra * rx_prev * d;
                        float h;
                        __nv_bfloat16 l;
                        dw_add(wxh_prev, wxl_prev, un, h, l);
                        oUX[qm] = un;
                        oWX[qm] = h;
                        oLX[qm] = l;
                        if (CHECK) acc += (double)d * (double)d;
                    }
                    if (upd_y) {
                        float d = (dxy_y + (tyz_n - tyz_prev)) + (dbxy_y + (byz_n - byz_prev));
                        float un = rb * uy_prev + ra * ry_prev * d;
                        float h;
                        __nv_bfloat16 l;
                        dw_add(wyh_prev, wyl_prev, un, h, l);
                        oUY[qm] = un;
                        oWY[qm] = h;
                        oLY[qm] = l;
                        if (CHECK) acc += (double)d * (double)d;
                    }
                }
            }
            // in-plane flux differences of plane s for w_x(s), w_y(s)
            if (own && s < nz) {
                dxy_x = (sxx_n - s_sxx[ty][tx - 1]) + (s_txy[ty + 1][tx] - txy_n);
                dxy_y = (s_txy[ty][tx + 1] - txy_n) + (syy_n - s_syy[ty - 1][tx]);
                dbxy_x = (bxx_n - s_bxx[ty][tx - 1]) + (s_bxy[ty + 1][tx] - bxy_n);
                dbxy_y = (s_bxy[ty][tx + 1] - bxy_n) + (byy_n - s_byy[ty - 1][tx]);
            }
            wxh_prev = wxh;
            wxl_prev = wxl;
            wyh_prev = wyh;
            wyl_prev = wyl;
            ux_prev = ux_o;
            uy_prev = uy_o;
            txz_prev = txz_n;
            tyz_prev = tyz_n;
            szz_prev = szz_n;
            bxz_prev = bxz_n;
            byz_prev = byz_n;
            bzz_prev = bzz_n;
            rx_prev = rxv;
            ry_prev = ryv;
            wzh_cur = wzh_n;
            wzl_cur = wzl_n;
        }
        if (CHECK) {
            // block sum in FP64: warp shuffles, then one value per warp row
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (tx == 0) s_red[ty] = acc;
            __syncthreads();
            if (ty == 0) {
                double t = tx < TY ? s_red[tx] : 0.0;
                for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
                if (tx == 0) a.partials[(size_t)m * nblk + bid] = t;
            }
            __syncthreads();
        }
    }
}

struct Geo {
    int ty, zc, nbx, nby, nch;
};

Geo geometry(const Layout& L, const int tile[3])
{
    Geo g;
    g.ty = tile && tile[1] > 0 ? tile[1] : 16;
    if (g.ty != 8 && g.ty != 16) g.ty = 16;
    g.nbx = (L.nx + 1 + TX - 3) / (TX - 2);
    g.nby = (L.ny + 1 + g.ty - 3) / (g.ty - 2);
    g.zc = tile && tile[2] > 0 ? tile[2] : 0;
    if (g.zc <= 0) {
        // aim for about two resident blocks per SM on a 152-SM part, with
        // chunks of at least 16 planes
        long long cols = (long long)g.nbx * g.nby;
        long long want = 2 * 152;
        int nch = (int)((want + cols - 1) / cols);
        if (nch < 1) nch = 1;
        g.zc = (L.nz + 1 + nch - 1) / nch;
        if (g.zc < 16) g.zc = 16;
    }
    g.nch = (L.nz + 1 + g.zc - 1) / g.zc;
    return g;
}

template <bool CHECK>
void launch_t(const FusedArgs& a, const Geo& g, cudaStream_t st)
{
    dim3 grid(g.nbx, g.nby, g.nch);
    if (g.ty == 8) k_fused<8, CHECK><<<grid, dim3(TX, 8), 0, st>>>(a, g.zc);
    else k_fused<16, CHECK><<<grid, dim3(TX, 16), 0, st>>>(a, g.zc);
}

}  // namespace

int fused_blocks(const Layout& L, const int tile[3])
{
    Geo g = geometry(L, tile);
    return g.nbx * g.nby * g.nch;
}

int launch_fused_sweep(const FusedArgs& a, const int tile[3], cudaStream_t st)
{
    Geo g = geometry(a.L, tile);
    if (a.partials) launch_t<true>(a, g, st);
    else launch_t<false>(a, g, st);
    return g.nbx * g.nby * g.nch;
}

}  // namespace ce
