// Paired-column TMA sweep: the same pseudo-time step as the single-column
// sweep (velocity form, double-word w, T = T(0) + T'(w), residual partials
// on check sweeps), with every thread owning two adjacent index-grid columns
// (i, i+1) of its row.  The pair is processed with packed FP32 instructions
// (f32x2 add/sub/mul/fma) and 64-bit shared-memory loads, so the arithmetic
// and shared-memory load instructions per point are halved; the results are
// bitwise those of the single-column sweep.  It is one of the launch shapes
// the autotuner times (tile[3] = 2).  At 191^3 it measured slower than the
// single-column sweep (1.14 against 0.93 ms per six-case sweep): its 124
// registers leave two blocks of 8 warps per SM, and the point-wise global
// loads of u, dt~/rho~ and K wait on memory.
//
// Step s of a load case holds planes s and s+1 of w and G in the copy ring
// and forms
//   * the cell stresses of plane s (e_zz needs w_z of plane s+1),
//   * the edge stresses tau_xy of plane s and tau_xz, tau_yz of plane s+1,
// exchanges them once through shared memory, and updates all three face
// components of plane s.  tau_xz, tau_yz of plane s and sigma_zz of plane s-1
// come from step s-1 in registers.  u, dt~/rho~ and K are read point-wise
// straight from global memory (coalesced 8-byte loads), so the ring holds
// only what has neighbours: w (hi, lo) and G.
//
// Tiles: a warp covers 64 columns of one row, of which 60 are owned (one
// column of halo on each side is needed, one more on each side keeps every
// pair 8-byte aligned); a block of 32 x TY threads owns TY-2 rows.  Boundary
// rules are per-point factors (every field is zero outside its faces), as in
// the single-column sweep.
#include <cuda_bf16.h>

#include "ce_internal.h"
#include "tma_util.cuh"

namespace ce {

namespace {

using namespace tma;

constexpr int PX = 32;     // threads per row
constexpr int PW = 72;     // box row (elements), FP32 and BF16
constexpr int OWN = 60;    // owned columns per row

// ------------------------------------------------------------ packed pairs
// two adjacent columns in one 64-bit register pair, computed with the
// sm_100-family packed FP32 instructions (IEEE single rounding per element,
// so a pair gives bitwise the results of two scalar evaluations)
using f2 = float2;

__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
// a * b + c, one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ f2 bc(float v) { return { v, v }; }

__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// two BF16 values (one 32-bit word) widened to FP32
__device__ __forceinline__ f2 ldh2(const __nv_bfloat16* p)
{
    const unsigned v = *reinterpret_cast<const unsigned*>(p);
    return { __uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u) };
}

__device__ __forceinline__ float ldh1(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// (a_hi + a_lo) - (b_hi + b_lo) formed part by part
__device__ __forceinline__ f2 dwdiff(f2 ah, f2 al, f2 bh, f2 bl) { return add2(sub2(ah, bh), sub2(al, bl)); }

// w + u for a double-word w (hi FP32, lo BF16), the same fast two-sums as
// the single-column sweep
__device__ __forceinline__ void dw_add2(f2 h, f2 l, f2 u, f2& ho, unsigned& lo)
{
    const f2 s = add2(h, u);
    const f2 e = sub2(u, sub2(s, h));
    const f2 l2 = add2(l, e);
    const f2 h2 = add2(s, l2);
    const f2 l3 = sub2(l2, sub2(h2, s));
    ho = h2;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(l3.y), "f"(l3.x));
}

template <int TY>
struct PairGeom {
    static constexpr int F32BOX = PW * TY * 4;
    static constexpr int B16BOX = PW * TY * 2;
    static constexpr int STAGE = 4 * F32BOX + 3 * B16BOX;   // w hi x3, G; w lo x3
    static constexpr int PL = TY * 64;                      // floats per exchange plane
};

template <int TY, int NST>
struct PairSmem {
    static constexpr int OFF_S = NST * PairGeom<TY>::STAGE;              // s_S[2][10][PL]
    static constexpr int OFF_BAR = OFF_S + 2 * 10 * PairGeom<TY>::PL * 4;
    static constexpr int OFF_RED = OFF_BAR + 8 * NST;
    static constexpr int SMEM = OFF_RED + 8 * TY + 16;
};

// the copies of one plane: w (hi, lo) of load case q from buffer b and G
template <int TY>
__device__ __forceinline__ void issue_plane(const TmaArgs& a, unsigned char* stage, uint64_t* bar, int q, int s,
                                            int xa, int xh, int y0, int b)
{
    using Gm = PairGeom<TY>;
    const int base = a.case_id[q] * NFIELD;
    fence_async();
    mbar_expect_tx(bar, Gm::STAGE);
    tma_load_4d(stage, &a.st32[b], xa, y0, s, base + F_WX, bar);
    tma_load_4d(stage + Gm::F32BOX, &a.st32[b], xa, y0, s, base + F_WY, bar);
    tma_load_4d(stage + 2 * Gm::F32BOX, &a.st32[b], xa, y0, s, base + F_WZ, bar);
    tma_load_4d_hint(stage + 3 * Gm::F32BOX, &a.mat, xa, y0, s, 1, bar, policy_evict_last());
    unsigned char* h = stage + 4 * Gm::F32BOX;
    tma_load_4d(h, &a.st16[b], xh, y0, s, 2 * (base + F_WLO_XY), bar);
    tma_load_4d(h + Gm::B16BOX, &a.st16[b], xh, y0, s, 2 * (base + F_WLO_XY) + 1, bar);
    tma_load_4d(h + 2 * Gm::B16BOX, &a.st16[b], xh, y0, s, 2 * (base + F_WLO_Z), bar);
}

// store one pair of a field, each point only where it is updated
__device__ __forceinline__ void put2(float* p, f2 v, bool m0, bool m1)
{
    if (m0 && m1) {
        *reinterpret_cast<float2*>(p) = v;
    } else {
        if (m0) p[0] = v.x;
        if (m1) p[1] = v.y;
    }
}

__device__ __forceinline__ void puth2(__nv_bfloat16* p, unsigned v, bool m0, bool m1)
{
    if (m0 && m1) {
        *reinterpret_cast<unsigned*>(p) = v;
    } else {
        if (m0) p[0] = __ushort_as_bfloat16((unsigned short)(v & 0xffffu));
        if (m1) p[1] = __ushort_as_bfloat16((unsigned short)(v >> 16));
    }
}

template <int TY, int NST, bool CHECK>
__device__ __forceinline__ void pair_body(const TmaArgs& a, int zc, int bxi, int byi, int bzi, int bid, int pstride,
                                          double* part, int bufo)
{
    using Gm = PairGeom<TY>;
    using Sm = PairSmem<TY, NST>;
    constexpr int PL = Gm::PL;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float* const s_S = reinterpret_cast<float*>(smem + Sm::OFF_S);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(smem + Sm::OFF_BAR);
    double* const s_red = reinterpret_cast<double*>(smem + Sm::OFF_RED);
    int* const s_abort = reinterpret_cast<int*>(smem + Sm::OFF_RED + 8 * TY);

    const Layout& L = a.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = bxi * OWN - 2, y0 = byi * (TY - 2) - 1;     // x0 even
    const int xa = x0 & ~3, xh = x0 & ~7;                      // 16-byte aligned box origins
    const int lx = 2 * tx;                                     // first column of the pair in the tile
    const int cf = lx + (x0 - xa), ch = lx + (x0 - xh);        // its place in a box row (even)
    const int cfl = cf > 0 ? cf - 1 : 0, chl = ch > 0 ? ch - 1 : 0;
    const int tym = ty - (ty > 0), typ = ty + (ty < TY - 1);
    const int i0 = x0 + lx, j = y0 + ty;
    const int i1 = i0 + 1;
    const bool rowin = j >= 0 && j <= ny;
    const bool in0 = rowin && i0 >= 0 && i0 <= nx, in1 = rowin && i1 >= 0 && i1 <= nx;
    // the pair's 8-byte global loads stay inside the padded rows
    const bool ldok = rowin && i0 >= 0 && i0 < L.pitch;
    const bool ownt = tx >= 1 && tx <= PX - 2 && ty >= 1 && ty <= TY - 2;
    const bool own0 = ownt && in0, own1 = ownt && in1;
    const bool ux0 = own0 && i0 > 0 && i0 < nx && j < ny, ux1 = own1 && i1 > 0 && i1 < nx && j < ny;
    const bool uy0 = own0 && i0 < nx && j > 0 && j < ny, uy1 = own1 && i1 < nx && j > 0 && j < ny;
    const bool uz0 = own0 && i0 < nx && j < ny, uz1 = own1 && i1 < nx && j < ny;
    const int bm = a.bc;
    const bool bx0 = i0 == 0 || i0 == nx, bx1 = i1 == 0 || i1 == nx, by_ = j == 0 || j == ny;
    const f2 fx = { bx0 ? 2.f : 1.f, bx1 ? 2.f : 1.f };
    const float fy = by_ ? 2.f : 1.f;
    // edge factors: zero where the boundary mode frees the shear stress
    const f2 cxy = { free_xy(bm, bx0, by_) ? 0.f : 0.25f * fx.x * fy, free_xy(bm, bx1, by_) ? 0.f : 0.25f * fx.y * fy };
    // edge factors of the xz and yz edges inside and on a z boundary
    const f2 cxz_in = { free_xz(bm, bx0, false) ? 0.f : 0.25f * fx.x, free_xz(bm, bx1, false) ? 0.f : 0.25f * fx.y };
    const f2 cxz_bd = { free_xz(bm, bx0, true) ? 0.f : 0.5f * fx.x, free_xz(bm, bx1, true) ? 0.f : 0.5f * fx.y };
    const float cyz_in = free_yz(bm, by_, false) ? 0.f : 0.25f * fy;
    const float cyz_bd = free_yz(bm, by_, true) ? 0.f : 0.5f * fy;
    const long long fs = L.fsize;
    const long long col = (long long)j * L.pitch + i0;
    const f2 ra = bc(a.a), rb = bc(1.f - a.a);
    const int k0 = bzi * zc;
    const int k1 = min(k0 + zc, nz);
    const int s_begin = k0 - 1;
    const int P = k1 - k0 + 1;            // steps per load case (planes s_begin .. k1 - 1)
    const int ncase = a.ncase;
    const int NP = ncase * (P + 1);       // planes copied per block
    const bool leader = tx == 0 && ty == 0;
    const int me = ty * 64 + lx;          // pair's first point in an exchange plane
    auto bufof = [&](int q) { return bufo >= 0 ? bufo : a.buf[q]; };

    // copy ring: plane g (global order) lives in stage g % NST; planes are
    // issued in order, a stage is refilled once its plane is not needed
    int gi = 0, im = 0, il = 0;           // next plane to issue and its (case, plane index)
    auto issue_upto = [&](int lowest) {
        while (gi < lowest + NST && gi < NP) {
            issue_plane<TY>(a, ring + (gi % NST) * Gm::STAGE, &bar[gi % NST], im, s_begin + il, xa, xh, y0,
                            bufof(im));
            ++gi;
            if (++il > P) {
                il = 0;
                ++im;
            }
        }
    };
    if (leader) {
        for (int t = 0; t < NST; ++t) mbar_init(&bar[t], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue_upto(0);
    }
    __syncthreads();
    bool ok = true;
    // stage and phase parity of the current plane and of the next one
    int q0 = 0, g = 0;                    // g: global index of the current plane
    unsigned ph0 = 0;
    auto next_stage = [&](int q, unsigned ph, int& qn, unsigned& phn) {
        qn = q + 1 == NST ? 0 : q + 1;
        phn = qn == 0 ? ph ^ 1u : ph;
    };
    int par = 0;                          // exchange-plane parity
    // clamped neighbour offsets in an exchange plane (the clamped values are
    // only read by lanes and rows that update nothing)
    const int om1 = lx > 0 ? -1 : 0, op2 = lx < 62 ? 2 : 0;
    const int orm = ty > 0 ? -64 : 0, orp = ty < TY - 1 ? 64 : 0;
    const bool rowown = ty >= 1 && ty <= TY - 2;
    // global loads of the pair: inside the padded rows, else from column 0
    const long long colc = ldok ? col : 0;
    const float* const matq = a.matp + colc;
    const unsigned lmask = (uz0 ? 0xffffu : 0u) | (uz1 ? 0xffff0000u : 0u);
    const unsigned xmask = (ux0 ? 0xffffu : 0u) | (ux1 ? 0xffff0000u : 0u);
    const unsigned ymask = (uy0 ? 0xffffu : 0u) | (uy1 ? 0xffff0000u : 0u);
    const bool sz = uz0 || uz1, sx = ux0 || ux1, sy = uy0 || uy1;
    auto sel2 = [](bool m0, bool m1, f2 v, f2 old) { return f2{ m0 ? v.x : old.x, m1 ? v.y : old.y }; };

    for (int m = 0; m < ncase; ++m) {
        const Ebar<float> eb = a.eb[m];
        const float trb = eb.xx + eb.yy + eb.zz;
        const bool bn = eb.xx != 0.f || eb.yy != 0.f || eb.zz != 0.f;
        const bool bxyo = eb.xy != 0.f, bxzo = eb.xz != 0.f, byzo = eb.yz != 0.f;
        const f2 exy2 = bc(2.f * eb.xy), exz2 = bc(2.f * eb.xz), eyz2 = bc(2.f * eb.yz);
        const float* const ib = a.base[bufof(m)] + (size_t)a.case_id[m] * NFIELD * fs + colc;
        float* const ob = a.base[1 - bufof(m)] + (size_t)a.case_id[m] * NFIELD * fs + colc;
        __nv_bfloat16* const lxy = reinterpret_cast<__nv_bfloat16*>(ob - colc + F_WLO_XY * fs) + colc;
        __nv_bfloat16* const lz = reinterpret_cast<__nv_bfloat16*>(ob - colc + F_WLO_Z * fs) + colc;
        // carried from step s-1: sigma_zz, b_zz of plane s-1; tau_xz, tau_yz
        // (and T(0) parts) of plane s with their in-plane differences
        f2 szz_p = bc(0.f), bzz_p = bc(0.f), txz_c = bc(0.f), tyz_c = bc(0.f), bxz_c = bc(0.f), byz_c = bc(0.f);
        f2 dxz_c = bc(0.f), dyz_c = bc(0.f), dbxz_c = bc(0.f), dbyz_c = bc(0.f);
        double acc = 0.0;

        for (int l = 0; l < P; ++l) {
            const int s = s_begin + l;
            const bool upd = s >= k0;
            // point-wise values of plane s, read early (plane 0 stands in for
            // the warm-up plane -1, whose cells and faces are never used)
            const long long qs = (long long)(s > 0 ? s : 0) * L.plane;
            const f2 Kc = ld2(matq + qs);
            f2 u_x = bc(0.f), u_y = bc(0.f), u_z = bc(0.f), r_x = bc(0.f), r_y = bc(0.f), r_z = bc(0.f);
            if (upd) {
                u_x = ld2(ib + F_UX * fs + qs);
                u_y = ld2(ib + F_UY * fs + qs);
                u_z = ld2(ib + F_UZ * fs + qs);
                r_x = ld2(matq + 2 * fs + qs);
                r_y = ld2(matq + 3 * fs + qs);
                r_z = ld2(matq + 4 * fs + qs);
            }
            int q1;
            unsigned ph1;
            next_stage(q0, ph0, q1, ph1);
            // planes s and s+1 have landed
            if (ok) {
                ok = mbar_wait_all(&bar[q0], ph0) && mbar_wait_all(&bar[q1], ph1);
                if (!ok) *s_abort = 1;
            }
            const unsigned char* st0 = ring + q0 * Gm::STAGE;
            const unsigned char* st1 = ring + q1 * Gm::STAGE;
            const float(*F0)[TY][PW] = reinterpret_cast<const float(*)[TY][PW]>(st0);
            const __nv_bfloat16(*H0)[TY][PW] = reinterpret_cast<const __nv_bfloat16(*)[TY][PW]>(st0 + 4 * Gm::F32BOX);
            const float(*F1)[TY][PW] = reinterpret_cast<const float(*)[TY][PW]>(st1);
            const __nv_bfloat16(*H1)[TY][PW] = reinterpret_cast<const __nv_bfloat16(*)[TY][PW]>(st1 + 4 * Gm::F32BOX);

            // plane s
            const f2 wxh = ld2(&F0[0][ty][cf]), wyh = ld2(&F0[1][ty][cf]), wzh = ld2(&F0[2][ty][cf]);
            const unsigned wxr = *reinterpret_cast<const unsigned*>(&H0[0][ty][ch]);
            const unsigned wyr = *reinterpret_cast<const unsigned*>(&H0[1][ty][ch]);
            const unsigned wzr = *reinterpret_cast<const unsigned*>(&H0[2][ty][ch]);
            const f2 wxl = { __uint_as_float(wxr << 16), __uint_as_float(wxr & 0xffff0000u) };
            const f2 wyl = { __uint_as_float(wyr << 16), __uint_as_float(wyr & 0xffff0000u) };
            const f2 wzl = { __uint_as_float(wzr << 16), __uint_as_float(wzr & 0xffff0000u) };
            const f2 Gc = ld2(&F0[3][ty][cf]);
            const f2 Gl = { F0[3][ty][cfl], Gc.x };                       // G(i-1, j)
            const f2 Gj = ld2(&F0[3][tym][cf]);                           // G(i, j-1)
            const f2 Gjl = { F0[3][tym][cfl], Gj.x };                     // G(i-1, j-1)
            const f2 wxh_r = { wxh.y, F0[0][ty][cf + 2] }, wxl_r = { wxl.y, ldh1(&H0[0][ty][ch + 2]) };
            const f2 wxh_j = ld2(&F0[0][tym][cf]), wxl_j = ldh2(&H0[0][tym][ch]);
            const f2 wyh_l = { F0[1][ty][cfl], wyh.x }, wyl_l = { ldh1(&H0[1][ty][chl]), wyl.x };
            const f2 wyh_j = ld2(&F0[1][typ][cf]), wyl_j = ldh2(&H0[1][typ][ch]);
            // plane s+1
            const f2 wxh1 = ld2(&F1[0][ty][cf]), wxl1 = ldh2(&H1[0][ty][ch]);
            const f2 wyh1 = ld2(&F1[1][ty][cf]), wyl1 = ldh2(&H1[1][ty][ch]);
            const f2 wzh1 = ld2(&F1[2][ty][cf]), wzl1 = ldh2(&H1[2][ty][ch]);
            const f2 wzh1_l = { F1[2][ty][cfl], wzh1.x }, wzl1_l = { ldh1(&H1[2][ty][chl]), wzl1.x };
            const f2 wzh1_j = ld2(&F1[2][tym][cf]), wzl1_j = ldh2(&H1[2][tym][ch]);
            const f2 G1 = ld2(&F1[3][ty][cf]);
            const f2 G1l = { F1[3][ty][cfl], G1.x };
            const f2 G1j = ld2(&F1[3][tym][cf]);

            // cell stresses of plane s (T' and T(0)); G = 0 off the cells
            const f2 exx = dwdiff(wxh_r, wxl_r, wxh, wxl);
            const f2 eyy = dwdiff(wyh_j, wyl_j, wyh, wyl);
            const f2 ezz = dwdiff(wzh1, wzl1, wzh, wzl);
            const f2 lk = fma2(bc(-2.f / 3.f), Gc, Kc);
            const f2 g2 = add2(Gc, Gc);
            const f2 lam = mul2(lk, add2(add2(exx, eyy), ezz));
            const f2 sxx = fma2(g2, exx, lam), syy = fma2(g2, eyy, lam), szz = fma2(g2, ezz, lam);
            f2 bxx = bc(0.f), byy = bc(0.f), bzz = bc(0.f);
            if (bn) {
                const f2 lb = mul2(lk, bc(trb));
                bxx = fma2(g2, bc(eb.xx), lb);
                byy = fma2(g2, bc(eb.yy), lb);
                bzz = fma2(g2, bc(eb.zz), lb);
            }
            // edge xy of plane s
            const f2 gxy = mul2(add2(add2(Gjl, Gj), add2(Gl, Gc)), cxy);
            const f2 dyx = mul2(bc(fy), dwdiff(wxh, wxl, wxh_j, wxl_j));
            const f2 dxy = mul2(fx, dwdiff(wyh, wyl, wyh_l, wyl_l));
            const f2 txy = mul2(gxy, add2(dyx, dxy));
            const f2 bxy = mul2(gxy, exy2);
            // edges xz, yz of plane s+1
            const bool zb = s + 1 == 0 || s + 1 == nz;
            const float fz = zb ? 2.f : 1.f;
            const f2 gxz = mul2(add2(add2(Gl, Gc), add2(G1l, G1)), zb ? cxz_bd : cxz_in);
            const f2 gyz = mul2(add2(add2(Gj, Gc), add2(G1j, G1)), bc(zb ? cyz_bd : cyz_in));
            const f2 dzx = mul2(bc(fz), dwdiff(wxh1, wxl1, wxh, wxl));
            const f2 dxz = mul2(fx, dwdiff(wzh1, wzl1, wzh1_l, wzl1_l));
            const f2 dzy = mul2(bc(fz), dwdiff(wyh1, wyl1, wyh, wyl));
            const f2 dyz = mul2(bc(fy), dwdiff(wzh1, wzl1, wzh1_j, wzl1_j));
            const f2 txz = mul2(gxz, add2(dzx, dxz)), tyz = mul2(gyz, add2(dzy, dyz));
            const f2 bxz = mul2(gxz, exz2), byz = mul2(gyz, eyz2);

            float* const S = s_S + par * 10 * PL;
            auto st2 = [&](int k, f2 v) { *reinterpret_cast<float2*>(&S[k * PL + me]) = v; };
            st2(0, sxx);
            st2(1, syy);
            st2(2, txy);
            st2(3, txz);
            st2(4, tyz);
            if (bn) {
                st2(5, bxx);
                st2(6, byy);
            }
            if (bxyo) st2(7, bxy);
            if (bxzo) st2(8, bxz);
            if (byzo) st2(9, byz);
            __syncthreads();
            // plane s is done with; after a load case's last step so is s+1
            if (leader && !*s_abort) issue_upto(g + (l == P - 1 ? 2 : 1));

            if (rowown) {
                auto ld = [&](int k, int off) { return ld2(&S[k * PL + me + off]); };
                auto l1 = [&](int k, int off) { return S[k * PL + me + off]; };
                if (upd) {
                    const f2 sxxl = { l1(0, om1), sxx.x }, syyj = ld(1, orm);
                    const f2 txyj = ld(2, orp), txyr = { txy.y, l1(2, op2) };
                    f2 bxxl = bc(0.f), byyj = bc(0.f), bxyj = bc(0.f), bxyr = bc(0.f);
                    if (bn) {
                        bxxl = f2{ l1(5, om1), bxx.x };
                        byyj = ld(6, orm);
                    }
                    if (bxyo) {
                        bxyj = ld(7, orp);
                        bxyr = f2{ bxy.y, l1(7, op2) };
                    }
                    float* const o = ob + qs;
                    {
                        // z faces of plane s (plane 0 is a boundary)
                        const bool zs = sz && s > 0;
                        const f2 d = add2(add2(add2(dxz_c, dyz_c), sub2(szz, szz_p)),
                                          add2(add2(dbxz_c, dbyz_c), sub2(bzz, bzz_p)));
                        const f2 un = fma2(rb, u_z, mul2(mul2(ra, r_z), d));
                        f2 hh;
                        unsigned ll;
                        dw_add2(wzh, wzl, un, hh, ll);
                        if (zs) {
                            *reinterpret_cast<float2*>(o + F_UZ * fs) = sel2(uz0, uz1, un, u_z);
                            *reinterpret_cast<float2*>(o + F_WZ * fs) = sel2(uz0, uz1, hh, wzh);
                            *reinterpret_cast<unsigned*>(lz + qs) = (ll & lmask) | (wzr & ~lmask);
                        }
                        if (CHECK && zs) acc += (uz0 ? (double)d.x * d.x : 0.0) + (uz1 ? (double)d.y * d.y : 0.0);
                    }
                    {
                        const f2 d = add2(add2(add2(sub2(sxx, sxxl), sub2(txyj, txy)), sub2(txz, txz_c)),
                                          add2(add2(sub2(bxx, bxxl), sub2(bxyj, bxy)), sub2(bxz, bxz_c)));
                        const f2 un = fma2(rb, u_x, mul2(mul2(ra, r_x), d));
                        f2 hh;
                        unsigned ll;
                        dw_add2(wxh, wxl, un, hh, ll);
                        if (sx) {
                            *reinterpret_cast<float2*>(o + F_UX * fs) = sel2(ux0, ux1, un, u_x);
                            *reinterpret_cast<float2*>(o + F_WX * fs) = sel2(ux0, ux1, hh, wxh);
                            *reinterpret_cast<unsigned*>(lxy + qs) = (ll & xmask) | (wxr & ~xmask);
                        }
                        if (CHECK && sx) acc += (ux0 ? (double)d.x * d.x : 0.0) + (ux1 ? (double)d.y * d.y : 0.0);
                    }
                    {
                        const f2 d = add2(add2(add2(sub2(txyr, txy), sub2(syy, syyj)), sub2(tyz, tyz_c)),
                                          add2(add2(sub2(bxyr, bxy), sub2(byy, byyj)), sub2(byz, byz_c)));
                        const f2 un = fma2(rb, u_y, mul2(mul2(ra, r_y), d));
                        f2 hh;
                        unsigned ll;
                        dw_add2(wyh, wyl, un, hh, ll);
                        if (sy) {
                            *reinterpret_cast<float2*>(o + F_UY * fs) = sel2(uy0, uy1, un, u_y);
                            *reinterpret_cast<float2*>(o + F_WY * fs) = sel2(uy0, uy1, hh, wyh);
                            *reinterpret_cast<unsigned*>(lxy + fs + qs) = (ll & ymask) | (wyr & ~ymask);
                        }
                        if (CHECK && sy) acc += (uy0 ? (double)d.x * d.x : 0.0) + (uy1 ? (double)d.y * d.y : 0.0);
                    }
                }
                // in-plane differences of tau_xz, tau_yz of plane s+1, for step s+1
                dxz_c = sub2(f2{ txz.y, l1(3, op2) }, txz);
                dyz_c = sub2(ld(4, orp), tyz);
                dbxz_c = bxzo ? sub2(f2{ bxz.y, l1(8, op2) }, bxz) : bc(0.f);
                dbyz_c = byzo ? sub2(ld(9, orp), byz) : bc(0.f);
            }
            szz_p = szz;
            bzz_p = bzz;
            txz_c = txz;
            tyz_c = tyz;
            bxz_c = bxz;
            byz_c = byz;
            par ^= 1;
            q0 = q1;
            ph0 = ph1;
            ++g;
        }
        // the last step's "next" plane ends the load case
        next_stage(q0, ph0, q0, ph0);
        ++g;
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
        __syncthreads();
    }
    if (*s_abort) {
        if (leader) {
            atomicExch(a.err, 1);
            // let the copies still in flight land before the block's memory goes away
            for (int t = (gi > NST ? gi - NST : 0); t < gi; ++t) mbar_wait(&bar[t % NST], (unsigned)(t / NST) & 1u);
        }
        __syncthreads();
    }
}

template <int TY, int NST, bool CHECK>
__global__ void __launch_bounds__(PX* TY, TY == 8 ? 2 : 1) k_pair_tma(const __grid_constant__ TmaArgs a, int zc)
{
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    pair_body<TY, NST, CHECK>(a, zc, blockIdx.x, blockIdx.y, blockIdx.z, bid, nblk, a.partials, -1);
}

// batched solve: as k_sweep_tma_batch, with the paired-column body
template <int TY, int NST, bool CHECK>
__global__ void __launch_bounds__(PX* TY, TY == 8 ? 2 : 1) k_pair_tma_batch(const BatchEntry* __restrict__ ents,
                                                                         int nsamp, const int* __restrict__ active,
                                                                         const int* __restrict__ parity, int k,
                                                                         double* part, int pstride)
{
    int s = 0;
    while (s + 1 < nsamp && (int)blockIdx.x >= ents[s + 1].off) ++s;
    if (!active[s]) return;
    const BatchEntry& e = ents[s];
    const int lb = (int)blockIdx.x - e.off;
    if (lb < 0 || lb >= e.nbx * e.nby * e.nch || (reinterpret_cast<uintptr_t>(&e) & 63) != 0) {
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(e.a.err, 2);
        return;
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const CUtensorMap* maps[5] = { &e.a.st32[0], &e.a.st32[1], &e.a.st16[0], &e.a.st16[1], &e.a.mat };
#pragma unroll
        for (int q = 0; q < 5; ++q)
            asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(maps[q]) : "memory");
    }
    const int bx = lb % e.nbx, by = (lb / e.nbx) % e.nby, bz = lb / (e.nbx * e.nby);
    pair_body<TY, NST, CHECK>(e.a, e.zc, bx, by, bz, lb, pstride, part + (size_t)s * CE_MAX_CASES * pstride,
                              (parity[s] + k) & 1);
}

template <int TY, int NST, bool CHECK>
void launch_pair_t(const TmaArgs& a, int nbx, int nby, int nch, int zc, cudaStream_t st)
{
    static std::atomic<unsigned long long> done{ 0 };
    ensure_dynamic_smem(k_pair_tma<TY, NST, CHECK>, PairSmem<TY, NST>::SMEM, done);
    k_pair_tma<TY, NST, CHECK><<<dim3(nbx, nby, nch), dim3(PX, TY), PairSmem<TY, NST>::SMEM, st>>>(a, zc);
}

template <int TY, int NST>
void launch_pair_c(const TmaArgs& a, int nbx, int nby, int nch, int zc, cudaStream_t st)
{
    if (a.partials) launch_pair_t<TY, NST, true>(a, nbx, nby, nch, zc, st);
    else launch_pair_t<TY, NST, false>(a, nbx, nby, nch, zc, st);
}

template <int TY, int NST, bool CHECK>
const void* pair_batch_kernel_t(int* smem)
{
    static std::atomic<unsigned long long> done{ 0 };
    *smem = PairSmem<TY, NST>::SMEM;
    if (!ensure_dynamic_smem(k_pair_tma_batch<TY, NST, CHECK>, PairSmem<TY, NST>::SMEM, done)) return nullptr;
    return reinterpret_cast<const void*>(k_pair_tma_batch<TY, NST, CHECK>);
}

}  // namespace

void pair_geometry(const Layout& L, const int tile[4], int* ty, int* nst, int* nbx, int* nby, int* nch, int* zc)
{
    *ty = tile && tile[1] == 16 ? 16 : 8;
    *nst = tile && (tile[0] == 2 || tile[0] == 4) ? tile[0] : 3;
    *nbx = (L.nx + 1 + OWN - 1) / OWN;
    *nby = (L.ny + 1 + *ty - 3) / (*ty - 2);
    *zc = tile && tile[2] > 0 ? tile[2] : 32;
    *nch = (L.nz + *zc - 1) / *zc;
}

int launch_pair_tma(const TmaArgs& a, const int tile[4], cudaStream_t st)
{
    int ty, nst, nbx, nby, nch, zc;
    pair_geometry(a.L, tile, &ty, &nst, &nbx, &nby, &nch, &zc);
    if (ty == 16) {
        if (nst == 2) launch_pair_c<16, 2>(a, nbx, nby, nch, zc, st);
        else if (nst == 4) launch_pair_c<16, 4>(a, nbx, nby, nch, zc, st);
        else launch_pair_c<16, 3>(a, nbx, nby, nch, zc, st);
    } else {
        if (nst == 2) launch_pair_c<8, 2>(a, nbx, nby, nch, zc, st);
        else if (nst == 4) launch_pair_c<8, 4>(a, nbx, nby, nch, zc, st);
        else launch_pair_c<8, 3>(a, nbx, nby, nch, zc, st);
    }
    return nbx * nby * nch;
}

const void* pair_batch_kernel(int ty, int nst, bool check, int* smem)
{
    if (ty == 16) {
        if (nst == 4) return check ? pair_batch_kernel_t<16, 4, true>(smem) : pair_batch_kernel_t<16, 4, false>(smem);
        return check ? pair_batch_kernel_t<16, 3, true>(smem) : pair_batch_kernel_t<16, 3, false>(smem);
    }
    if (nst == 4) return check ? pair_batch_kernel_t<8, 4, true>(smem) : pair_batch_kernel_t<8, 4, false>(smem);
    return check ? pair_batch_kernel_t<8, 3, true>(smem) : pair_batch_kernel_t<8, 3, false>(smem);
}

}  // namespace ce
