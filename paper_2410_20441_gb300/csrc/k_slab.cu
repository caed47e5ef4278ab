// Halo planes of a z-slab decomposition (the multi-GPU domain decomposition
// the paper names as future work, Sec. 5.3, item 1).  A slab context updates the index
// planes [kz0, kz1) of its local grid; the sweep of plane k reads w of planes
// k - 1 and k + 1, so after every sweep the neighbours swap one plane of w:
// the slab's first and last own planes go out, the planes kz0 - 1 and kz1
// (owned by the neighbours) come in.  Nothing else crosses: the moduli of
// the ghost planes are uploaded once, and u, which only the owner of a
// plane reads, stays local.
//
// Message of one plane, per load case q (in the order of the case list):
//   words [q*4.5P, q*4.5P + 3P)        w_x, w_y, w_z high parts (FP32 planes)
//   words [q*4.5P + 3P, (q+1)*4.5P)    w_x, w_y, w_z low parts (BF16 planes)
// with P = Layout::plane elements; P is a multiple of 32, so every segment
// starts on a 16-byte boundary and the copies move 16-byte words.
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int HB = 256;

__global__ void k_halo(Layout L, HaloArgs h, int plane, uint4* __restrict__ msg, int unpack)
{
    const int q = blockIdx.y / 6, seg = blockIdx.y % 6;
    const long long P = L.plane;
    // segment length in 16-byte words: FP32 planes P/4, BF16 planes P/8
    const long long n16 = seg < 3 ? P / 4 : P / 8;
    uint4* src;
    if (seg < 3) {
        float* f = h.base[q] + (size_t)(F_WX + seg) * L.fsize + (size_t)plane * P;
        src = reinterpret_cast<uint4*>(f);
    } else {
        __nv_bfloat16* lo = seg == 5
                                ? reinterpret_cast<__nv_bfloat16*>(h.base[q] + (size_t)F_WLO_Z * L.fsize)
                                : reinterpret_cast<__nv_bfloat16*>(h.base[q] + (size_t)F_WLO_XY * L.fsize)
                                      + (seg == 4 ? L.fsize : 0);
        src = reinterpret_cast<uint4*>(lo + (size_t)plane * P);
    }
    const long long off16 = (long long)q * (P * 9 / 8) + (seg < 3 ? seg * (P / 4) : 3 * (P / 4) + (seg - 3) * (P / 8));
    uint4* m = msg + off16;
    for (long long t = (long long)blockIdx.x * HB + threadIdx.x; t < n16; t += (long long)gridDim.x * HB) {
        if (unpack) src[t] = m[t];
        else m[t] = src[t];
    }
}

}  // namespace

size_t halo_bytes(const Layout& L, int ncases) { return (size_t)ncases * (size_t)L.plane * 18; }

void launch_halo(const Layout& L, const HaloArgs& h, int ncases, int plane, void* msg, int unpack,
                 cudaStream_t st)
{
    const long long n16 = L.plane / 4;
    int bx = (int)((n16 + HB - 1) / HB);
    if (bx > 64) bx = 64;
    k_halo<<<dim3(bx, 6 * ncases), HB, 0, st>>>(L, h, plane, reinterpret_cast<uint4*>(msg), unpack);
}

}  // namespace ce
