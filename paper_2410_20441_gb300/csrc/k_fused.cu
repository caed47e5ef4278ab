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
// bytes out; in the first phase of a refined solve (w in FP32 alone) 24 in
// and 24 out; in its correction phase (the FP32 correction and the stored
// FP32 right-hand side) 36 in and 24 out.
//
// Design (memory-bound stencil, no tensor-core work):
//  * A block of 32 x TY threads owns the interior (30 x (TY-2)) of its tile of
//    index-grid columns and recomputes the one-column halo of elastic stresses
//    itself (overlapped tiling), so one sweep is one launch.  Neighbouring
//    tiles read each other's old values, so the state is ping-ponged.
//  * The block marches in z over a chunk of planes; z-neighbours stay in
//    registers, so every field is read once per sweep (plus the halo).
//  * Two sweep kernels share this plan.  k_fused reads with ordinary
//    coalesced loads and updates (w_z, u_z) of plane s and (w_x, u_x),
//    (w_y, u_y) of plane s-1 at step s.  The TMA sweep (sweep_body) streams
//    the planes through a ring of shared-memory stages filled by bulk tensor
//    copies and updates all three components of plane s-1 at step s, which
//    needs one plane per stage and one block barrier per step.
//  * k_fused processes the load cases one after another inside the block;
//    the TMA sweep gives each load case of a tile its own block, and the
//    blocks of one tile run side by side, so the material planes come from
//    DRAM about once per sweep and from L2 for the other cases.
//  * On check sweeps the same div T(w_n) gives the residual: each block adds
//    its squares in FP64 and writes one partial per load case (a fixed-order
//    second pass sums them), so checking costs no extra pass over memory.
#include <cudaTypedefs.h>

#include "ce_internal.h"
#include "tma_util.cuh"

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
// w + u for a double-word w = h + l (|l| <= ulp(h)/2).  The rounding error e
// of s = h + u is taken by the fast two-sum e = u - (s - h), exact when
// |h| >= |u| (a sweep moves w by a small fraction of itself); where |h| < |u|
// the error it can miss is below ulp(s) of a small s.  The renormalisation of
// (s, l + e) is a fast two-sum as well.
__device__ __forceinline__ void dw_add(float h, float l, float u, float& ho, __nv_bfloat16& lo)
{
    float s = h + u;
    float e = u - (s - h);
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
            if (ing && s < nz && tx > 0 && ty > 0 && !free_xy(a.bc, i == 0 || i == nx, j == 0 || j == ny)) {
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
            if (ing && j < ny && tx > 0 && !free_xz(a.bc, i == 0 || i == nx, s == 0 || s == nz)) {
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
            if (ing && i < nx && ty > 0 && !free_yz(a.bc, j == 0 || j == ny, s == 0 || s == nz)) {
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
    // this kernel is built for 8 and 16 rows
    g.ty = tile && tile[1] == 8 ? 8 : 16;
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

// ===========================================================================
// TMA variant.  Same arithmetic as k_fused, but every plane of every field a
// block needs (u, w hi, w lo, K, G, dt~/rho~) arrives by cp.async.bulk.tensor
// into a three-stage shared-memory ring, issued two planes ahead by one
// thread and completed on an mbarrier, so the loads of two planes are in
// flight while a plane is computed, and no registers are held by in-flight
// loads.  Tensor maps view a whole ping-pong buffer as a 4-D array
// (x, y, z, field slot); a box is one TY-row tile of one plane of one slot.
// The x origin of a box is rounded down to 16 bytes (4 FP32 / 8 BF16
// elements) and the row is read at an offset, as TMA requires.  Every wait
// on an mbarrier is bounded: on time-out the block sets an error flag, waits
// (bounded) for its copies in flight and returns.
// ===========================================================================
namespace ce {

namespace {

using namespace tma;

constexpr int RW = 40;     // FP32 row of a box (elements)
constexpr int RH = 48;     // BF16 row of a box (elements)
constexpr int NF32 = 11;   // u x3, w hi x3, K, G, rx, ry, rz
constexpr int NB16 = 3;    // w lo x3

template <int TY>
struct TmaGeom {
    static constexpr int F32BOX = RW * TY * 4;
    static constexpr int B16BOX = RH * TY * 2;
    static constexpr int STAGE = NF32 * F32BOX + NB16 * B16BOX;
    // FP32 w without a low part (MODE_F32): the FP32 boxes only
    static constexpr int STAGE_F32 = NF32 * F32BOX;
    // correction phase (MODE_RHS): the three FP32 right-hand-side slots
    // replace the BF16 low parts
    static constexpr int STAGE_RHS = (NF32 + 3) * F32BOX;
    template <int MODE>
    static constexpr int STAGE_OF = MODE == MODE_DW ? STAGE : MODE == MODE_F32 ? STAGE_F32 : STAGE_RHS;
};

// loads for step t of the block: load case q (position in the active list), plane s
template <int TY, int MODE>
__device__ __forceinline__ void issue_step(const TmaArgs& a, unsigned char* stage, uint64_t* bar, int q, int s,
                                           int xa, int xh, int y0, int b)
{
    using Gm = TmaGeom<TY>;
    const int base = a.case_id[q] * NFIELD;
    fence_async();
    mbar_expect_tx(bar, Gm::template STAGE_OF<MODE>);
    // FP32 boxes: u (slots 0-2), w hi (slots 6-8), then material (0-4)
    const int slots[6] = { base + F_UX, base + F_UY, base + F_UZ, base + F_WX, base + F_WY, base + F_WZ };
#pragma unroll
    for (int f = 0; f < 6; ++f) tma_load_4d(stage + f * Gm::F32BOX, &a.st32[b], xa, y0, s, slots[f], bar);
    // the blocks of one tile's load cases read the same material planes at
    // about the same time: ask L2 to keep them for the others
    const uint64_t pol = policy_evict_last();
#pragma unroll
    for (int f = 0; f < 5; ++f) tma_load_4d_hint(stage + (6 + f) * Gm::F32BOX, &a.mat, xa, y0, s, f, bar, pol);
    if constexpr (MODE == MODE_RHS) {
        // right-hand side r_x, r_y, r_z (FP32, slots 3-5)
#pragma unroll
        for (int f = 0; f < 3; ++f)
            tma_load_4d(stage + (NF32 + f) * Gm::F32BOX, &a.st32[b], xa, y0, s, base + F_RX + f, bar);
    } else if constexpr (MODE == MODE_DW) {
        // BF16 boxes: w lo x, y (slot 3 halves), z (slot 4 first half)
        unsigned char* h = stage + NF32 * Gm::F32BOX;
        tma_load_4d(h, &a.st16[b], xh, y0, s, 2 * (base + F_WLO_XY), bar);
        tma_load_4d(h + Gm::B16BOX, &a.st16[b], xh, y0, s, 2 * (base + F_WLO_XY) + 1, bar);
        tma_load_4d(h + 2 * Gm::B16BOX, &a.st16[b], xh, y0, s, 2 * (base + F_WLO_Z), bar);
    }
}

}  // namespace

}  // namespace ce

namespace ce {

namespace {

// ---------------------------------------------------------------------------
// Lagged single-plane sweep.  Step s of a load case holds only plane s of the
// old state in shared memory and forms, with the own-column values of plane
// s-1 kept in registers:
//   * the cell stresses of plane s-1 (their in-plane strains e_xx, e_yy were
//     formed at step s-1, e_zz needs w_z of planes s-1 and s),
//   * the edge stresses of plane s (xy in-plane; xz, yz from the own-column
//     z-difference and in-plane w_z neighbours),
// exchanges them once through shared memory and then updates all three face
// components of plane s-1, whose last missing flux (tau_xz, tau_yz of plane
// s) has just been formed.  In-plane flux differences of plane s are kept for
// step s+1.  So every step reads one plane, needs one block barrier, and the
// copy ring only has to hold the planes being prefetched.
//
// Boundaries are folded into per-thread factors instead of branches: every
// field is zero outside its own index range (the moduli at non-cells, w at
// non-faces, the box outside the grid), so a boundary-tangential derivative
// is f * (w(q) - w(q-1)) with f = 2 on the boundary and 1 inside (the half
// spacing to the Dirichlet value), and the edge modulus is the sum of the
// four neighbouring cells times 1/(number of existing cells) = f_a f_b / 4.
// The arithmetic is that of the general per-point formulas term by term.
template <int TY, int NST, int MODE>
struct SweepGeom {
    static constexpr int STAGE = TmaGeom<TY>::template STAGE_OF<MODE>;
    static constexpr int PL = TY * TX;                       // floats per plane of the block
    // exchange slots of a plane: T' (sxx, syy, txy, txz, tyz), then the parts
    // of T(0) (bxx, byy, bxy, bxz, byz), which the correction phase has not
    static constexpr int NS = MODE == MODE_RHS ? 5 : 10;
    static constexpr int OFF_G = NST * STAGE;                // s_G[2][PL]
    static constexpr int OFF_S = OFF_G + 2 * PL * 4;         // s_S[2][NS][PL]
    // one row of slack after the exchange planes: the edge threads' reads one
    // row past their plane (values no own point uses) stay in the block's memory
    static constexpr int OFF_BAR = OFF_S + (2 * NS * PL + TX) * 4;   // mbarriers
    static constexpr int OFF_RED = OFF_BAR + 8 * NST;        // residual partials of the warps
    static constexpr int SMEM = OFF_RED + 8 * TY + 16;
    // within the block's opt-in shared memory limit (227 KB)
    static constexpr bool FITS = SMEM <= 232448;
};

template <int V>
struct Par {
    static constexpr int value = V;
};

// The block sweeps the entries m0 <= m < m1 of the active list one after
// another through one copy ring (the single-image sweep gives every block one
// load case; the batched sweep gives it all of them).  MODE:
//   MODE_DW   w = FP32 high + BF16 low part (double word), load T(0) = C : ebar;
//   MODE_F32  w in FP32 alone, load T(0): the first phase of a refined solve,
//             which only has to bring the residual down by REFINE_STEP;
//   MODE_RHS  the correction phase of a refined solve: w is replaced by the
//             FP32 correction dw, T(0) by the stored right-hand side
//             r = div sigma(ebar.x + w_base), and the force at a face is
//             r + div C : eps(dw).
template <int TY, int NST, bool CHECK, int MODE>
__device__ __forceinline__ void sweep_body(const TmaArgs& a, int zc, int bxi, int byi, int bzi, int bid,
                                           int pstride, double* part, int bufo, int m0, int m1)
{
    constexpr bool RHS = MODE == MODE_RHS;   // right-hand side r instead of T(0)
    constexpr bool LOW = MODE == MODE_DW;    // w has a BF16 low part
    using Gm = TmaGeom<TY>;
    using Sg = SweepGeom<TY, NST, MODE>;
    constexpr int PL = Sg::PL;
    // one warp reduces the rows' residual partials
    static_assert(Sg::FITS && TY <= 32, "launch shape out of range");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float* const s_G = reinterpret_cast<float*>(smem + Sg::OFF_G);
    float* const s_S = reinterpret_cast<float*>(smem + Sg::OFF_S);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(smem + Sg::OFF_BAR);
    double* const s_red = reinterpret_cast<double*>(smem + Sg::OFF_RED);
    int* const s_abort = reinterpret_cast<int*>(smem + Sg::OFF_RED + 8 * TY);

    const Layout& L = a.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = bxi * (TX - 2) - 1, y0 = byi * (TY - 2) - 1;
    const int xa = (x0 >> 2) << 2, xh = (x0 >> 3) << 3;   // 16-byte aligned box origins
    const int cf = tx + (x0 - xa), ch = tx + (x0 - xh);   // this thread's column in a box row
    // neighbour columns and rows.  At the block edge (tx = 0, ty = 0,
    // ty = TY - 1) they fall one element or one row outside the thread's box
    // row; the shared-memory layout keeps every such address inside the
    // block's allocation (a neighbouring field, stage or the ring's end), and
    // no value an own point consumes is formed from them, so they need no
    // clamping (which would cost address registers).
    const int cfm = cf - 1, chm = ch - 1;
    const int tym = ty - 1, typ = ty + 1;
    const int txm = tx - 1;
    const int i = x0 + tx, j = y0 + ty;
    const int k0 = L.kz0 + bzi * zc;
    const int k1 = min(k0 + zc, L.kz1);
    const bool ing = i >= 0 && i <= nx && j >= 0 && j <= ny;
    const bool own = ing && tx >= 1 && tx <= TX - 2 && ty >= 1 && ty <= TY - 2;
    const bool upd_x = own && i > 0 && i < nx && j < ny;
    const bool upd_y = own && i < nx && j > 0 && j < ny;
    const bool upd_z = own && i < nx && j < ny;
    const int bc = a.bc;
    const bool bx_ = i == 0 || i == nx, by_ = j == 0 || j == ny;
    const float fx = bx_ ? 2.f : 1.f, fy = by_ ? 2.f : 1.f;
    // edge factors: zero where the boundary mode frees the shear stress
    const float cxy = free_xy(bc, bx_, by_) ? 0.f : 0.25f * fx * fy;
    // xz and yz edge factors inside and on a z boundary (f_z = 2 there)
    const float cxz_in = free_xz(bc, bx_, false) ? 0.f : 0.25f * fx;
    const float cxz_bd = free_xz(bc, bx_, true) ? 0.f : 0.5f * fx;
    const float cyz_in = free_yz(bc, by_, false) ? 0.f : 0.25f * fy;
    const float cyz_bd = free_yz(bc, by_, true) ? 0.f : 0.5f * fy;
    const long long fs = L.fsize;
    const long long col = ing ? (long long)j * L.pitch + i : 0;
    const float ra = a.a, rb = 1.f - a.a;
    const int s_begin = k0 > 0 ? k0 - 1 : 0;
    const int s_end = k1 <= nz ? k1 : nz;
    const bool leader = tx == 0 && ty == 0;
    const int me = ty * TX + tx;
    auto bufof = [&](int q) { return bufo >= 0 ? bufo : a.buf[q]; };

    // the copy ring: step (im, is) is the next one to issue, (q, ph) the
    // stage and phase parity of the step being consumed.  Issue number t goes
    // to stage t % NST and completes phase (t / NST) & 1 of its mbarrier;
    // nissued (leader only) counts the issues.
    int im = m0, is = s_begin, q = 0, nissued = 0;
    unsigned ph = 0;
    auto issue_next = [&](int stage) {
        issue_step<TY, MODE>(a, ring + stage * Sg::STAGE, &bar[stage], im, is, xa, xh, y0, bufof(im));
        ++nissued;
        if (++is > s_end) {
            is = s_begin;
            ++im;
        }
    };
    if (leader) {
        for (int t = 0; t < NST; ++t) mbar_init(&bar[t], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int t = 0; t < NST && im < m1; ++t) issue_next(t);
    }
    s_G[me] = 0.f;
    s_G[PL + me] = 0.f;
    __syncthreads();
    bool ok = true;

    for (int m = m0; m < m1; ++m) {
        const Ebar<float> eb = a.eb[m];
        const float trb = eb.xx + eb.yy + eb.zz;
        const bool bn_rt = eb.xx != 0.f || eb.yy != 0.f || eb.zz != 0.f;
        const bool bxy_rt = eb.xy != 0.f, bxz_rt = eb.xz != 0.f, byz_rt = eb.yz != 0.f;
        // the parts of T(0) = C : ebar this load case has: 1 normal, 2 xy,
        // 4 xz, 8 yz for a case with one part only (the six unit cases),
        // else 0 (decided at run time)
        const int nparts = (int)bn_rt + (int)bxy_rt + (int)bxz_rt + (int)byz_rt;
        const int kind = RHS ? 16 : nparts != 1 ? 0 : bn_rt ? 1 : bxy_rt ? 2 : bxz_rt ? 4 : 8;
        const float exy2 = 2.f * eb.xy, exz2 = 2.f * eb.xz, eyz2 = 2.f * eb.yz;
        float* const ob = a.base[1 - bufof(m)] + (size_t)a.case_id[m] * NFIELD * fs;
        __nv_bfloat16* const lxy = reinterpret_cast<__nv_bfloat16*>(ob + F_WLO_XY * fs);   // x lo, then y lo
        __nv_bfloat16* const lz = reinterpret_cast<__nv_bfloat16*>(ob + F_WLO_Z * fs);
        double acc = 0.0;

        // the case's sweep through the planes, with the parts of T(0) known at
        // compile time (KD != 0) or read from the flags (KD == 0).  A part
        // that is absent only ever adds zeros, so leaving it out changes no
        // value (at most the sign of a zero).  KD = 16: no T(0) at all (the
        // correction phase, whose load is the stored r)
        auto run = [&](auto kd) {
            constexpr int KD = decltype(kd)::value;
            static_assert(!RHS || KD == 16, "the correction phase has no T(0)");
            const bool bn = KD ? (KD & 1) != 0 : bn_rt;
            const bool bxyo = KD ? (KD & 2) != 0 : bxy_rt;
            const bool bxzo = KD ? (KD & 4) != 0 : bxz_rt;
            const bool byzo = KD ? (KD & 8) != 0 : byz_rt;
            // own-column values of plane s-1 and in-plane flux differences of plane s-1
            float wxh_p = 0.f, wxl_p = 0.f, wyh_p = 0.f, wyl_p = 0.f, wzh_p = 0.f, wzl_p = 0.f;
            float exx_p = 0.f, eyy_p = 0.f, K_p = 0.f, G_p = 0.f;
            float ux_p = 0.f, uy_p = 0.f, uz_p = 0.f, rx_p = 0.f, ry_p = 0.f, rz_p = 0.f;
            float fx_p = 0.f, fy_p = 0.f, fz_p = 0.f;   // right-hand side of plane s-1 (RHS)
            float szz_pp = 0.f, bzz_pp = 0.f, txz_p = 0.f, tyz_p = 0.f, bxz_p = 0.f, byz_p = 0.f;
            float dxy_x = 0.f, dxy_y = 0.f, dxz_z = 0.f, dyz_z = 0.f;
            float bxy_x = 0.f, bxy_y = 0.f, bxz_z = 0.f, byz_z = 0.f;

            // one step: plane s of this load case; PAR selects the exchange planes
            auto step = [&](auto par, int s) {
                constexpr int PAR = decltype(par)::value;
                if (ok && !*s_abort) {
                    ok = mbar_wait_all(&bar[q], ph);
                    if (!ok) *s_abort = 1;
                }
                const unsigned char* stg = ring + q * Sg::STAGE;
                const float(*F)[TY][RW] = reinterpret_cast<const float(*)[TY][RW]>(stg);
                [[maybe_unused]] const __nv_bfloat16(*H)[TY][RH] =
                    reinterpret_cast<const __nv_bfloat16(*)[TY][RH]>(stg + NF32 * Gm::F32BOX);
                const float* const gprev = s_G + (1 - PAR) * PL;
                float* const S = s_S + PAR * Sg::NS * PL;

                // low part of w at a box position (none without LOW)
                auto LO = [&](int f, int row, int c) -> float {
                    if constexpr (!LOW) return 0.f;
                    else return __bfloat162float(H[f][row][c]);
                };
                // (high difference) + (low difference)
                auto dsum = [](float dh, float dl) -> float {
                    if constexpr (!LOW) return dh;
                    else return dh + dl;
                };
                const float wxh = F[3][ty][cf], wyh = F[4][ty][cf], wzh = F[5][ty][cf];
                const float wxl = LO(0, ty, ch), wyl = LO(1, ty, ch);
                const float wzl = LO(2, ty, ch);
                const float Kc = F[6][ty][cf], Gc = F[7][ty][cf];
                s_G[PAR * PL + me] = Gc;
                const bool zb = s == 0 || s == nz;

                // cell stresses of plane s-1 (T' and T(0))
                float sxx, syy, szz, bxx = 0.f, byy = 0.f, bzz = 0.f, exx_n, eyy_n;
                {
                    const float ezz = dsum(wzh - wzh_p, wzl - wzl_p);
                    const float lk = K_p - (2.f / 3.f) * G_p;
                    const float g2 = 2.f * G_p;
                    const float lam = lk * ((exx_p + eyy_p) + ezz);
                    sxx = lam + g2 * exx_p;
                    syy = lam + g2 * eyy_p;
                    szz = lam + g2 * ezz;
                    if (bn) {
                        const float lb = lk * trb;
                        bxx = lb + g2 * eb.xx;
                        byy = lb + g2 * eb.yy;
                        bzz = lb + g2 * eb.zz;
                    }
                    // in-plane strains of the cell of plane s (for step s+1)
                    exx_n = dsum(F[3][ty][cf + 1] - wxh, LO(0, ty, ch + 1) - wxl);
                    eyy_n = dsum(F[4][typ][cf] - wyh, LO(1, typ, ch) - wyl);
                }
                // edge stresses of plane s; G of plane s-1 is zero before the
                // first plane (the exchange plane is cleared for it)
                float txy, txz, tyz, bxy, bxz, byz;
                {
                    const float fz = zb ? 2.f : 1.f;
                    const float cxz = zb ? cxz_bd : cxz_in, cyz = zb ? cyz_bd : cyz_in;
                    const float gpm = gprev[ty * TX + txm];     // G(i-1, j, s-1)
                    const float gp0 = gprev[me];                // G(i, j, s-1)
                    const float gpj = gprev[tym * TX + tx];     // G(i, j-1, s-1)
                    const float g_mm = F[7][tym][cfm], g_m0 = F[7][ty][cfm], g_0m = F[7][tym][cf];
                    const float gxy = ((g_mm + g_0m) + (g_m0 + Gc)) * cxy;
                    const float gxz = ((gpm + gp0) + (g_m0 + Gc)) * cxz;
                    const float gyz = ((gpj + gp0) + (g_0m + Gc)) * cyz;
                    const float dyx = fy * dsum(wxh - F[3][tym][cf], wxl - LO(0, tym, ch));
                    const float dxy = fx * dsum(wyh - F[4][ty][cfm], wyl - LO(1, ty, chm));
                    const float dzx = fz * dsum(wxh - wxh_p, wxl - wxl_p);
                    const float dxz = fx * dsum(wzh - F[5][ty][cfm], wzl - LO(2, ty, chm));
                    const float dzy = fz * dsum(wyh - wyh_p, wyl - wyl_p);
                    const float dyz = fy * dsum(wzh - F[5][tym][cf], wzl - LO(2, tym, ch));
                    txy = gxy * (dyx + dxy);
                    txz = gxz * (dzx + dxz);
                    tyz = gyz * (dzy + dyz);
                    bxy = gxy * exy2;
                    bxz = gxz * exz2;
                    byz = gyz * eyz2;
                }
                // the own values the updates of plane s need at step s+1
                const float ux = F[0][ty][cf], uy = F[1][ty][cf], uz = F[2][ty][cf];
                const float rx = F[8][ty][cf], ry = F[9][ty][cf], rz = F[10][ty][cf];
                float fxr = 0.f, fyr = 0.f, fzr = 0.f;
                if constexpr (RHS) {
                    fxr = F[NF32][ty][cf];
                    fyr = F[NF32 + 1][ty][cf];
                    fzr = F[NF32 + 2][ty][cf];
                }

                S[0 * PL + me] = sxx;
                S[1 * PL + me] = syy;
                S[2 * PL + me] = txy;
                S[3 * PL + me] = txz;
                S[4 * PL + me] = tyz;
                if (bn) {
                    S[5 * PL + me] = bxx;
                    S[6 * PL + me] = byy;
                }
                if (bxyo) S[7 * PL + me] = bxy;
                if (bxzo) S[8 * PL + me] = bxz;
                if (byzo) S[9 * PL + me] = byz;
                __syncthreads();
                // every read of this stage is done: refill it
                if (leader && im < m1 && !*s_abort) issue_next(q);
                if (++q == NST) {
                    q = 0;
                    ph ^= 1u;
                }

                if (own) {
                    // updates of the faces of plane p = s - 1 (p < k1 and p < nz
                    // hold at every step: s ends at min(k1, nz))
                    const int p = s - 1;
                    if (p >= k0) {
                        const long long qo = (long long)p * L.plane + col;
                        float* const o = ob + qo;

                        if (upd_z && p > 0) {
                            const float dt = (dxz_z + dyz_z) + (szz - szz_pp);
                            float d;
                            if constexpr (RHS) d = dt + fz_p;
                            else if constexpr (KD == 0) d = dt + ((bxz_z + byz_z) + (bzz - bzz_pp));
                            else if constexpr (KD == 1) d = dt + (bzz - bzz_pp);
                            else if constexpr (KD == 2) d = dt;
                            else if constexpr (KD == 4) d = dt + bxz_z;
                            else d = dt + byz_z;
                            const float un = rb * uz_p + ra * rz_p * d;
                            o[F_UZ * fs] = un;
                            if constexpr (!LOW) {
                                o[F_WZ * fs] = wzh_p + un;
                            } else {
                                float hh;
                                __nv_bfloat16 ll;
                                dw_add(wzh_p, wzl_p, un, hh, ll);
                                o[F_WZ * fs] = hh;
                                lz[qo] = ll;
                            }
                            if (CHECK) acc += (double)d * (double)d;
                        }
                        const float sxxm = S[0 * PL + me - 1], syym = S[1 * PL + me - TX];
                        [[maybe_unused]] const float bxxm = bn ? S[5 * PL + me - 1] : 0.f;
                        [[maybe_unused]] const float byym = bn ? S[6 * PL + me - TX] : 0.f;
                        if (upd_x) {
                            const float dt = ((sxx - sxxm) + dxy_x) + (txz - txz_p);
                            float d;
                            if constexpr (RHS) d = dt + fx_p;
                            else if constexpr (KD == 0) d = dt + (((bxx - bxxm) + bxy_x) + (bxz - bxz_p));
                            else if constexpr (KD == 1) d = dt + (bxx - bxxm);
                            else if constexpr (KD == 2) d = dt + bxy_x;
                            else if constexpr (KD == 4) d = dt + (bxz - bxz_p);
                            else d = dt;
                            const float un = rb * ux_p + ra * rx_p * d;
                            o[F_UX * fs] = un;
                            if constexpr (!LOW) {
                                o[F_WX * fs] = wxh_p + un;
                            } else {
                                float hh;
                                __nv_bfloat16 ll;
                                dw_add(wxh_p, wxl_p, un, hh, ll);
                                o[F_WX * fs] = hh;
                                lxy[qo] = ll;
                            }
                            if (CHECK) acc += (double)d * (double)d;
                        }
                        if (upd_y) {
                            const float dt = (dxy_y + (syy - syym)) + (tyz - tyz_p);
                            float d;
                            if constexpr (RHS) d = dt + fy_p;
                            else if constexpr (KD == 0) d = dt + ((bxy_y + (byy - byym)) + (byz - byz_p));
                            else if constexpr (KD == 1) d = dt + (byy - byym);
                            else if constexpr (KD == 2) d = dt + bxy_y;
                            else if constexpr (KD == 4) d = dt;
                            else d = dt + (byz - byz_p);
                            const float un = rb * uy_p + ra * ry_p * d;
                            o[F_UY * fs] = un;
                            if constexpr (!LOW) {
                                o[F_WY * fs] = wyh_p + un;
                            } else {
                                float hh;
                                __nv_bfloat16 ll;
                                dw_add(wyh_p, wyl_p, un, hh, ll);
                                o[F_WY * fs] = hh;
                                lxy[fs + qo] = ll;
                            }
                            if (CHECK) acc += (double)d * (double)d;
                        }
                    }
                    // in-plane flux differences of plane s, for step s+1
                    dxy_x = S[2 * PL + me + TX] - txy;
                    dxy_y = S[2 * PL + me + 1] - txy;
                    dxz_z = S[3 * PL + me + 1] - txz;
                    dyz_z = S[4 * PL + me + TX] - tyz;
                    bxy_x = bxyo ? S[7 * PL + me + TX] - bxy : 0.f;
                    bxy_y = bxyo ? S[7 * PL + me + 1] - bxy : 0.f;
                    bxz_z = bxzo ? S[8 * PL + me + 1] - bxz : 0.f;
                    byz_z = byzo ? S[9 * PL + me + TX] - byz : 0.f;
                }
                wxh_p = wxh;
                wxl_p = wxl;
                wyh_p = wyh;
                wyl_p = wyl;
                wzh_p = wzh;
                wzl_p = wzl;
                exx_p = exx_n;
                eyy_p = eyy_n;
                K_p = Kc;
                G_p = Gc;
                ux_p = ux;
                uy_p = uy;
                uz_p = uz;
                rx_p = rx;
                ry_p = ry;
                rz_p = rz;
                fx_p = fxr;
                fy_p = fyr;
                fz_p = fzr;
                szz_pp = szz;
                bzz_pp = bzz;
                txz_p = txz;
                tyz_p = tyz;
                bxz_p = bxz;
                byz_p = byz;
            };

            for (int s = s_begin; s <= s_end; s += 2) {
                step(Par<0>{}, s);
                if (s + 1 <= s_end) step(Par<1>{}, s + 1);
            }
        };
        if constexpr (RHS) {
            run(Par<16>{});
        } else {
            switch (kind) {
            case 1: run(Par<1>{}); break;
            case 2: run(Par<2>{}); break;
            case 4: run(Par<4>{}); break;
            case 8: run(Par<8>{}); break;
            default: run(Par<0>{}); break;
            }
        }
        if (CHECK) {
            for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o2);
            if (tx == 0) s_red[ty] = acc;
            __syncthreads();
            if (ty == 0) {
                double tt = tx < TY ? s_red[tx] : 0.0;
                for (int o2 = 16; o2 > 0; o2 >>= 1) tt += __shfl_down_sync(0xffffffffu, tt, o2);
                if (tx == 0) part[(size_t)m * pstride + bid] = tt;
            }
        }
        // the next load case starts again with exchange planes 0; a chunk
        // that starts at plane 0 reads plane 1's G exchange as "plane -1"
        if (s_begin == 0) s_G[PL + me] = 0.f;
        __syncthreads();
    }
    if (*s_abort) {
        if (leader) {
            atomicExch(a.err, 1);
            // let the copies still in flight land before the block's memory
            // goes away.  No issue follows the barrier after the first failed
            // wait, and a stage is refilled only after the step before it in
            // that stage was consumed, so only the last NST issues can still
            // be in flight: wait (bounded) for each with its own stage and
            // parity
            for (int t = nissued > NST ? nissued - NST : 0; t < nissued; ++t)
                mbar_wait(&bar[t % NST], (unsigned)(t / NST) & 1u);
        }
        __syncthreads();
    }
}

// one image: block x index = entry + ncase * (tile column), so the blocks of
// one tile's load cases are neighbours in launch order, run at the same time
// and share the tile's material planes through L2 (read from DRAM about once
// per sweep); the residual partial of entry m and tile b is at m * tiles + b
template <int TY, int NST, int MINB, bool CHECK, int MODE>
__global__ void __launch_bounds__(TX* TY, MINB) k_sweep_tma(const __grid_constant__ TmaArgs a, int zc)
{
    const int m = (int)blockIdx.x % a.ncase;
    const int bx = (int)blockIdx.x / a.ncase;
    const int nbx = (int)gridDim.x / a.ncase;
    const int bid = ((int)blockIdx.z * (int)gridDim.y + (int)blockIdx.y) * nbx + bx;
    const int nblk = nbx * (int)gridDim.y * (int)gridDim.z;
    sweep_body<TY, NST, CHECK, MODE>(a, zc, bx, blockIdx.y, blockIdx.z, bid, nblk, a.partials, -1, m, m + 1);
}

// batched solve: one launch over the tiles of every active sample.  Block b
// belongs to the sample s with off[s] <= b < off[s+1] and sweeps load case
// (b - off[s]) % 6 of tile (b - off[s]) / 6; the sample reads the buffer
// (parity[s] + k) & 1 at the k-th sweep of the current check interval.
// The maps live in global memory, written by a copy before the launch: the
// acquire fence orders that write before the tensor-map reads of the copies.
template <int TY, int NST, bool CHECK, int MODE>
__global__ void __launch_bounds__(TX* TY, TY == 8 ? 2 : 1) k_sweep_tma_batch(const BatchEntry* __restrict__ ents, int nsamp,
                                                             const int* __restrict__ active,
                                                             const int* __restrict__ parity, int k, double* part,
                                                             int pstride)
{
    int s = 0;
    while (s + 1 < nsamp && (int)blockIdx.x >= ents[s + 1].off) ++s;
    if (!active[s]) return;
    const BatchEntry& e = ents[s];
    const int lb = (int)blockIdx.x - e.off;
    // one load case per block, the cases of a tile adjacent (as k_sweep_tma)
    const int nc = e.a.ncase;
    if (lb < 0 || nc < 1 || lb >= e.nbx * e.nby * e.nch * nc || (reinterpret_cast<uintptr_t>(&e) & 63) != 0) {
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(e.a.err, 2);
        return;
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const CUtensorMap* maps[5] = { &e.a.st32[0], &e.a.st32[1], &e.a.st16[0], &e.a.st16[1], &e.a.mat };
#pragma unroll
        for (int q = 0; q < 5; ++q)
            asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(maps[q]) : "memory");
    }
    const int m = lb % nc, t = lb / nc;
    const int bx = t % e.nbx, by = (t / e.nbx) % e.nby, bz = t / (e.nbx * e.nby);
    sweep_body<TY, NST, CHECK, MODE>(e.a, e.zc, bx, by, bz, t, pstride,
                                      part + (size_t)s * CE_MAX_CASES * pstride, (parity[s] + k) & 1, m, m + 1);
}

struct TGeo {
    int ty, zc, nbx, nby, nch;
};

TGeo tgeometry(const Layout& L, const int tile[4])
{
    // (rows per block: sweep_rows)
    TGeo g;
    g.ty = sweep_rows(tile);
    g.nbx = (L.nx + 1 + TX - 3) / (TX - 2);
    g.nby = (L.ny + 1 + g.ty - 3) / (g.ty - 2);
    // z-chunks of 32 planes (measured best at 191^3 among 32, 48 and one
    // chunk per three blocks per SM)
    g.zc = tile && tile[2] > 0 ? tile[2] : 32;
    g.nch = (L.kz1 - L.kz0 + g.zc - 1) / g.zc;
    return g;
}

}  // namespace

int sweep_rows(const int tile[4])
{
    if (tile && tile[3] == 2) return tile[1] == 16 ? 16 : 8;
    if (!tile) return 16;
    return tile[1] == 8 ? 8 : tile[1] == 24 ? 24 : 16;
}

void batch_geometry(const Layout& L, const int tile[4], int* nbx, int* nby, int* nch, int* zc)
{
    if (tile && tile[3] == 2) {
        int ty, nst;
        pair_geometry(L, tile, &ty, &nst, nbx, nby, nch, zc);
        return;
    }
    TGeo g = tgeometry(L, tile);
    *nbx = g.nbx;
    *nby = g.nby;
    *nch = g.nch;
    *zc = g.zc;
}

// the batched sweep kernel for box height ty with or without the residual
// check, in the double-word mode or the FP32-w mode of a first phase, its
// dynamic shared memory raised to what it needs (once per device)
template <int TY, int NST, bool CHECK, int MODE>
const void* batch_kernel_t(int* smem)
{
    static std::atomic<unsigned long long> done{ 0 };
    *smem = SweepGeom<TY, NST, MODE>::SMEM;
    if (!ensure_dynamic_smem(k_sweep_tma_batch<TY, NST, CHECK, MODE>, SweepGeom<TY, NST, MODE>::SMEM, done))
        return nullptr;
    return reinterpret_cast<const void*>(k_sweep_tma_batch<TY, NST, CHECK, MODE>);
}

template <int TY, int MODE>
const void* batch_kernel_n(int nst, bool check, int* smem)
{
    if (nst == 2) return check ? batch_kernel_t<TY, 2, true, MODE>(smem) : batch_kernel_t<TY, 2, false, MODE>(smem);
    return check ? batch_kernel_t<TY, 3, true, MODE>(smem) : batch_kernel_t<TY, 3, false, MODE>(smem);
}

template <int MODE>
const void* batch_kernel_m(int ty, int nst, bool check, int* smem)
{
    if (ty == 24) return batch_kernel_n<24, MODE>(nst, check, smem);
    if (ty == 16) return batch_kernel_n<16, MODE>(nst, check, smem);
    return batch_kernel_n<8, MODE>(nst, check, smem);
}

const void* batch_kernel(int ty, int nst, bool check, int mode, int* smem)
{
    return mode == MODE_F32 ? batch_kernel_m<MODE_F32>(ty, nst, check, smem)
                            : batch_kernel_m<MODE_DW>(ty, nst, check, smem);
}

namespace {
// chunks per case a launch may use (twice the tile's, and one): bounds the
// residual partials fused_tma_blocks makes room for
int chunk_cap(const TGeo& g) { return 2 * g.nch + 1; }
}  // namespace

int fused_tma_blocks(const Layout& L, const int tile[4])
{
    if (tile && tile[3] == 2) {
        int ty, nst, nbx, nby, nch, zc;
        pair_geometry(L, tile, &ty, &nst, &nbx, &nby, &nch, &zc);
        return nbx * nby * nch;
    }
    // room for the residual partials of a launch whose chunks fused_tma_chunk
    // shortened: n cases x at most 6 chunk_cap / n chunks
    TGeo g = tgeometry(L, tile);
    return g.nbx * g.nby * chunk_cap(g);
}

// z-planes per block for a launch over n of the six load cases.  The tile's
// chunk is sized for six; with fewer cases the grid has fewer blocks and its
// last wave can leave SMs idle (191^3, 24-row blocks, 96-plane chunks: 378
// blocks for three cases, 2.5 waves of 152).  So the chunk is shortened
// (down to 16 planes, to at most 6 chunk_cap / n chunks per case)
// to the one of least predicted time, ceil(blocks / (SMs x blocks per SM))
// waves of (chunk + 4) planes (4: a chunk's extra plane and ring fill, fitted
// to launch times at 191^3), if that is at least 5 % below the tile's chunk.
// Measured at 191^3 with 2..5 cases the rule picks the fastest chunk or one
// within 1 % of it (7-14 % shorter launches); with one case and on large
// grids (many waves) it keeps the tile's chunk.
int fused_tma_chunk(const Layout& L, const int tile[4], int n, int nsm)
{
    TGeo g = tgeometry(L, tile);
    if ((tile && tile[3] == 2) || n <= 0 || n >= CE_MAX_CASES || nsm <= 0) return g.zc;
    const int span = L.kz1 - L.kz0;
    const long long cols = (long long)g.nbx * g.nby;
    const long long slots = (long long)nsm * (g.ty == 8 ? 2 : 1);
    const int hi = chunk_cap(g) * CE_MAX_CASES / n;
    auto cost = [&](int zc) {
        const long long nb = (long long)n * cols * ((span + zc - 1) / zc);
        return ((nb + slots - 1) / slots) * (zc + 4);
    };
    const long long base = cost(g.zc);
    int best = g.zc;
    long long best_cost = base;
    for (int nch = g.nch + 1; nch <= hi; ++nch) {
        const int zc = (span + nch - 1) / nch;
        if (zc < 16) break;
        if (cost(zc) < best_cost) {
            best_cost = cost(zc);
            best = zc;
        }
    }
    return 20 * best_cost <= 19 * base ? best : g.zc;
}

namespace {

template <int TY, int NST, int MINB, bool CHECK, int MODE>
void launch_sweep_t(const TmaArgs& a, const TGeo& g, cudaStream_t st)
{
    using Sg = SweepGeom<TY, NST, MODE>;
    static std::atomic<unsigned long long> done{ 0 };
    ensure_dynamic_smem(k_sweep_tma<TY, NST, MINB, CHECK, MODE>, Sg::SMEM, done);
    dim3 grid(g.nbx * a.ncase, g.nby, g.nch);
    k_sweep_tma<TY, NST, MINB, CHECK, MODE><<<grid, dim3(TX, TY), Sg::SMEM, st>>>(a, g.zc);
}

template <int TY, int NST, int MINB, int MODE>
void launch_sweep_m(const TmaArgs& a, const TGeo& g, cudaStream_t st)
{
    if (a.partials) launch_sweep_t<TY, NST, MINB, true, MODE>(a, g, st);
    else launch_sweep_t<TY, NST, MINB, false, MODE>(a, g, st);
}

template <int TY, int NST, int MINB>
void launch_sweep_c(const TmaArgs& a, const TGeo& g, cudaStream_t st)
{
    if (a.mode == MODE_RHS) launch_sweep_m<TY, NST, MINB, MODE_RHS>(a, g, st);
    else if (a.mode == MODE_F32) launch_sweep_m<TY, NST, MINB, MODE_F32>(a, g, st);
    else launch_sweep_m<TY, NST, MINB, MODE_DW>(a, g, st);
}

}  // namespace

int launch_fused_tma(const TmaArgs& a, const int tile[4], cudaStream_t st)
{
    if (a.cols == 2) return launch_pair_tma(a, tile, st);
    TGeo g = tgeometry(a.L, tile);
    const int nst = tile && tile[0] == 2 ? 2 : 3;
    if (g.ty == 8) {
        if (nst == 2) launch_sweep_c<8, 2, 2>(a, g, st);
        else launch_sweep_c<8, 3, 2>(a, g, st);
    } else if (g.ty == 24) {
        // 768 threads: 24 warps per SM, at most 85 registers a thread (the
        // sweep fits in 80 without spilling in the FP32 and correction modes).
        // Measured 10 % faster than 16 rows at 191^3 and 479^3; 28 and 32 rows
        // (72 and 64 registers) spill and measured slower
        if (nst == 2) launch_sweep_c<24, 2, 1>(a, g, st);
        else launch_sweep_c<24, 3, 1>(a, g, st);
    } else {
        if (nst == 2) launch_sweep_c<16, 2, 1>(a, g, st);
        else launch_sweep_c<16, 3, 1>(a, g, st);
    }
    return g.nbx * g.nby * g.nch;
}

bool encode_tma_maps(TmaArgs& a, const Layout& L, void* state0, void* state1, void* mat, int ty, int cols)
{
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult qr;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr)
                != cudaSuccess
            || qr != cudaDriverEntryPointSuccess || !fn)
            return false;
        enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    if (ty != 8 && ty != 16 && !(ty == 24 && cols != 2)) return false;
    const cuuint32_t estr[4] = { 1, 1, 1, 1 };
    auto make = [&](CUtensorMap* m, void* base, CUtensorMapDataType dt, int esz, int row, int nslot) {
        cuuint64_t dim[4] = { (cuuint64_t)L.pitch * (4 / esz), (cuuint64_t)(L.ny + 1), (cuuint64_t)(L.nz + 1),
                              (cuuint64_t)nslot };
        cuuint64_t str[3] = { (cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4, (cuuint64_t)L.fsize * 4 };
        if (esz == 2) {
            // a BF16 slot is half of a float slot: same row and plane strides in
            // bytes, twice as many slots of half the byte size
            dim[0] = (cuuint64_t)L.pitch;
            str[0] = (cuuint64_t)L.pitch * 2;
            str[1] = (cuuint64_t)L.plane * 2;
            str[2] = (cuuint64_t)L.fsize * 2;
        }
        cuuint32_t box[4] = { (cuuint32_t)row, (cuuint32_t)ty, 1, 1 };
        return enc(m, dt, 4, base, dim, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const int nst = CE_MAX_CASES * NFIELD;
    a.base[0] = (float*)state0;
    a.base[1] = (float*)state1;
    a.matp = (const float*)mat;
    a.cols = cols == 2 ? 2 : 1;
    // box rows: 40 FP32 / 48 BF16 elements cover the 32 columns of a warp
    // with one column of halo from any 16-byte aligned origin; 72 cover the
    // 64 columns of the paired-column warp
    const int rw = a.cols == 2 ? 72 : RW, rh = a.cols == 2 ? 72 : RH;
    bool ok = make(&a.st32[0], state0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rw, nst)
           && make(&a.st32[1], state1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rw, nst)
           && make(&a.st16[0], state0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, rh, 2 * nst)
           && make(&a.st16[1], state1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, rh, 2 * nst)
           && make(&a.mat, mat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rw, 5);
    return ok;
}

}  // namespace ce
