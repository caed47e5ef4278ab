// libce C-ABI: context life cycle, the pseudo-time loop driver, volume
// averages -> C (Eq. BC:3), field export and the adjoint gradient entry.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <new>
#include <vector>

#include "ce_internal.h"

using namespace ce;

struct ce_ctx {
    Layout L{};
    ce_opts opts{};
    ce_allocator alloc{};
    bool own_alloc = true;
    cudaStream_t st = nullptr;
    // numerical parameters (Sec. 3.1)
    double theta = 0, cdr = 0;
    int n_check = 16;
    // device memory
    std::vector<std::pair<void*, size_t>> blocks;
    float* K = nullptr;           // cell moduli on the index grid
    float* G = nullptr;
    void* rx = nullptr;           // dt~/rho~ per velocity node (field type)
    void* ry = nullptr;
    void* rz = nullptr;
    void* state[2] = { nullptr, nullptr };   // [buffer][case][field] fields
    void* scratch = nullptr;      // FP64: elastic-stress scratch of one case
    double* partials = nullptr;
    double* dres = nullptr;       // per-case reduction outputs (12 doubles each)
    double* hres = nullptr;       // pinned host mirror
    int* derr = nullptr;          // device error flag of the TMA sweep
    TmaArgs* tma = nullptr;       // encoded tensor maps (FP32 fused path)
    // defect correction of refined solves (FP32 TMA path of a whole image)
    double* wb = nullptr;         // FP64 w_base, [case][component] fields
    double* s64 = nullptr;        // FP64 elastic-stress scratch of one case (6 fields)
    bool wb_valid[CE_MAX_CASES] = {};   // w_base holds the case's final w (last solve was refined)
    // batch of samples (ce_create_batch)
    std::vector<ce_ctx*> samples;
    BatchEntry* d_ents = nullptr;
    int* d_int = nullptr;         // active, parity, iters, status (4 x n)
    double* d_dbl = nullptr;      // res0, rel (2 x 6n), tol and max_iter
    double* d_part = nullptr;
    int pstride = 0, total_blocks = 0, batch_ty = 8, batch_nchk = 32;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev[4] = { nullptr, nullptr, nullptr, nullptr };   // sweep / check timing
    int nblk = 0;
    int nsm = 0;                  // SMs of the context's device
    // the first phase of a refined solve may run at its own Strouhal number
    // (ce_opts.St_first): its theta and dt~/rho~ scale, and whether the
    // node coefficients rx, ry, rz currently hold that phase's values
    double theta1 = 0.0, cdr1 = 0.0;
    bool coef_first = false;
    size_t npart = 0;
    int cur[CE_MAX_CASES] = { 0 };
    // results of the last solve
    int n_cases = 0;
    double loads[CE_MAX_CASES][6]{};
    double sig[CE_MAX_CASES][6]{}, eps[CE_MAX_CASES][6]{};
    bool have_avg = false;
    bool moduli_ok = true;        // false after a rejected ce_set_moduli
    bool have_state = false;      // a solve has left fields to warm start from
    bool unit_loads = false;
    bool slab = false;            // a z-slab of a larger grid (ce_create_slab)
    int slab_nres = 0;            // entries of the last checked slab sweep
    bool slab_pend[CE_MAX_CASES] = {};   // a split slab sweep wrote its boundary planes, interior pending
    int slab_npend = 0;
    char err[512] = "";
};

namespace {

// the fused FP32 path keeps the state in velocity form (u, double-word w)
bool vform(const ce_ctx* c) { return c->opts.prec == CE_PREC_FP32 && c->opts.kernel != CE_KERNEL_PLAIN; }
bool use_tma(const ce_ctx* c) { return vform(c) && c->opts.kernel != CE_KERNEL_FUSED_LSU; }

const char* kStatus[] = { "ok", "invalid argument", "out of device memory", "CUDA error", "not converged",
                          "diverged", "call out of order", "not implemented" };

thread_local char t_free_err[256] = "";

ce_status fail(ce_ctx* c, ce_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CK(ctx, call)                                                                                      \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return fail((ctx), CE_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,    \
                        __LINE__);                                                                         \
    } while (0)

#define CKL(ctx) CK(ctx, cudaGetLastError())

size_t esize(const ce_ctx* c) { return c->opts.prec == CE_PREC_FP64 ? sizeof(double) : sizeof(float); }

void* dev_alloc(ce_ctx* c, size_t bytes)
{
    void* p = nullptr;
    if (c->alloc.alloc) {
        p = c->alloc.alloc(bytes, (void*)c->st, c->alloc.user);
    } else if (cudaMallocAsync(&p, bytes, c->st) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->blocks.push_back({ p, bytes });
    return p;
}

void release(ce_ctx* c)
{
    for (auto& b : c->blocks) {
        if (c->alloc.free) c->alloc.free(b.first, b.second, (void*)c->st, c->alloc.user);
        else cudaFreeAsync(b.first, c->st);
    }
    c->blocks.clear();
    if (c->hres) cudaFreeHost(c->hres);
    c->hres = nullptr;
    delete c->tma;
    c->tma = nullptr;
    for (auto& e : c->ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
}

template <class T>
T* field(const ce_ctx* c, int buf, int m, int f)
{
    return (T*)c->state[buf] + ((size_t)m * NFIELD + f) * (size_t)c->L.fsize;
}

bool vform(const ce_ctx* c);

template <class T>
CaseArgs<T> case_args(const ce_ctx* c, int buf, int m)
{
    CaseArgs<T> a;
    for (int f = 0; f < NFIELD; ++f) a.f[f] = field<T>(c, buf, m, f);
    a.eb = ebar_from_voigt<T>(c->loads[m]);
    if (vform(c)) {
        const __nv_bfloat16* lxy = (const __nv_bfloat16*)field<T>(c, buf, m, F_WLO_XY);
        a.lo[0] = lxy;
        a.lo[1] = lxy + c->L.fsize;
        a.lo[2] = (const __nv_bfloat16*)field<T>(c, buf, m, F_WLO_Z);
    }
    return a;
}


bool finite_pos(const float* v, size_t n)
{
    for (size_t q = 0; q < n; ++q)
        if (!(isfinite(v[q]) && v[q] > 0.f)) return false;
    return true;
}

}  // namespace

namespace ce {
const char* free_last_error() { return t_free_err; }
void set_free_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_free_err, sizeof t_free_err, fmt, ap);
    va_end(ap);
}
}  // namespace ce

// =====================================================================
extern "C" {

void ce_default_opts(ce_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->prec = CE_PREC_FP32;
    o->bc = CE_BC_KUBC;
    o->kernel = CE_KERNEL_AUTO;
    o->St = 2.0 * M_PI * sqrt(3.0);
    o->Ct = 0.95 / sqrt(3.0);
    o->n_check = 0;
}

const char* ce_status_str(ce_status s)
{
    return (s >= 0 && s <= CE_ENOTIMPL) ? kStatus[s] : "unknown status";
}

const char* ce_last_error(const ce_ctx* c) { return c ? c->err : free_last_error(); }

// moduli (host or device, x fastest) -> padded index grid, checked positive
// and finite; then dt~/rho~ of every velocity node
static ce_status upload_moduli(ce_ctx* c, const float* K, const float* G, int moduli_on_device)
{
    const Layout& L = c->L;
    if (!moduli_on_device) {
        size_t n = (size_t)L.nx * L.ny * L.nz;
        if (!finite_pos(K, n) || !finite_pos(G, n)) return fail(c, CE_EINVAL, "moduli must be positive and finite");
        for (int which = 0; which < 2; ++which) {
            cudaMemcpy3DParms p = {};
            p.srcPtr = make_cudaPitchedPtr((void*)(which ? G : K), (size_t)L.nx * sizeof(float), L.nx, L.ny);
            p.dstPtr = make_cudaPitchedPtr((void*)(which ? c->G : c->K), (size_t)L.pitch * sizeof(float),
                                           L.pitch, L.ny + 1);
            p.extent = make_cudaExtent((size_t)L.nx * sizeof(float), L.ny, L.nz);
            p.kind = cudaMemcpyHostToDevice;
            CK(c, cudaMemcpy3DAsync(&p, c->st));
        }
    } else {
        launch_scatter_moduli(L, K, G, c->K, c->G, c->st);
        CKL(c);
    }
    int* dbad = (int*)c->dres;
    CK(c, cudaMemsetAsync(dbad, 0, sizeof(int), c->st));
    launch_validate(L, c->K, c->G, dbad, c->st);
    CKL(c);
    int hbad = 0;
    CK(c, cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (hbad) return fail(c, CE_EINVAL, "moduli must be positive and finite");
    if (c->opts.prec == CE_PREC_FP64)
        launch_node_coef<double>(L, c->K, c->G, (double*)c->rx, (double*)c->ry, (double*)c->rz, c->cdr, c->st);
    else
        launch_node_coef<float>(L, c->K, c->G, (float*)c->rx, (float*)c->ry, (float*)c->rz, c->cdr, c->st);
    CKL(c);
    CK(c, cudaStreamSynchronize(c->st));
    return CE_OK;
}

}  // extern "C"

namespace {

// z window of a slab context: local grid g (cells zoff .. zoff + g->nz - 1
// of a grid with nzg cells in z), own index planes [kz0, kz1) local
struct Window {
    int zoff, nzg, kz0, kz1;
};

// a failure with no context to hold its message (ce_last_error(NULL))
ce_status free_fail(ce_status s, const char* what)
{
    set_free_error("%s", what);
    return s;
}

ce_status create_ctx_impl(const ce_grid* g, const float* K, const float* G, int moduli_on_device,
                          const ce_opts* opts, const ce_allocator* a, void* stream, ce_ctx** out, const Window* win,
                          bool refine_mem)
{
    if (!out) return free_fail(CE_EINVAL, "create: NULL output pointer");
    *out = nullptr;
    if (!g || !K || !G) return free_fail(CE_EINVAL, "create: NULL grid or moduli");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return free_fail(CE_EINVAL, "create: grid below 2 voxels per axis");
    if ((long long)(g->nx + 1) * (g->ny + 1) * (g->nz + 1) > (1LL << 31) - 1)
        return free_fail(CE_EINVAL, "create: (nx+1)(ny+1)(nz+1) exceeds 32-bit index-grid offsets");
    ce_ctx* c = new (std::nothrow) ce_ctx();
    if (!c) return CE_ENOMEM;
    ce_default_opts(&c->opts);
    if (opts) c->opts = *opts;
    c->opts.tile[3] = c->opts.tile[3] == 2 ? 2 : 1;
    if (win) {
        // slabs run the single-column TMA sweep, the one kernel with the window
        if (c->opts.prec != CE_PREC_FP32 || c->opts.kernel == CE_KERNEL_PLAIN
            || c->opts.kernel == CE_KERNEL_FUSED_LSU) {
            delete c;
            return free_fail(CE_ENOTIMPL, "create: slabs run the FP32 TMA sweep only");
        }
        c->opts.kernel = CE_KERNEL_FUSED;
        c->opts.tile[3] = 1;
        c->slab = true;
    }
    if (c->opts.St <= 0) c->opts.St = 2.0 * M_PI * sqrt(3.0);
    if (c->opts.Ct <= 0) c->opts.Ct = 0.95 / sqrt(3.0);
    if (c->opts.prec != CE_PREC_FP32 && c->opts.prec != CE_PREC_FP64) {
        delete c;
        return free_fail(CE_EINVAL, "create: bad precision");
    }
    if (!valid_bc(c->opts.bc)) {
        delete c;
        return free_fail(CE_EINVAL, "create: bad boundary condition");
    }
    if (c->opts.kernel < CE_KERNEL_AUTO || c->opts.kernel > CE_KERNEL_FUSED_LSU) {
        delete c;
        return free_fail(CE_EINVAL, "create: bad kernel");
    }
    if (c->opts.prec == CE_PREC_FP64 && (c->opts.kernel == CE_KERNEL_FUSED || c->opts.kernel == CE_KERNEL_FUSED_LSU)) {
        delete c;
        return free_fail(CE_ENOTIMPL, "create: the fused sweeps are FP32 only");
    }
    if (a) { c->alloc = *a; c->own_alloc = false; }
    c->st = (cudaStream_t)stream;
    Layout& L = c->L;
    L.nx = g->nx; L.ny = g->ny; L.nz = g->nz;
    L.pitch = ((g->nx + 1) + 31) / 32 * 32;
    L.plane = (long long)L.pitch * (g->ny + 1);
    L.fsize = L.plane * (g->nz + 1);
    L.kz0 = win ? win->kz0 : 0;
    L.kz1 = win ? win->kz1 : g->nz + 1;
    L.zoff = win ? win->zoff : 0;
    L.nzg = win ? win->nzg : g->nz;
    c->n_check = c->opts.n_check > 0 ? c->opts.n_check : (g->nx / 4 > 16 ? g->nx / 4 : 16);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess
            || cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            c->nsm = 0;   // unknown: sweeps keep the tile's chunk
    }

    // numerical parameters, Sec. 3.1: St = Lx/(Vp~ dt), dt~ = C~ dx / Vp~,
    // dt~/rho~ = C~ dx Lx / (St H~ dt); dx = dt = 1; Lx of the whole grid
    const int nzg = L.nzg;
    double Lx = (double)(g->nx > g->ny ? (g->nx > nzg ? g->nx : nzg) : (g->ny > nzg ? g->ny : nzg));
    double Vp = Lx / c->opts.St;
    c->theta = c->opts.Ct / Vp;
    c->cdr = c->opts.Ct * Lx / c->opts.St;
    if (c->opts.St_first > 0 && c->opts.St_first != c->opts.St) {
        c->theta1 = c->opts.Ct / (Lx / c->opts.St_first);
        c->cdr1 = c->opts.Ct * Lx / c->opts.St_first;
    } else {
        c->opts.St_first = c->opts.St;
        c->theta1 = c->theta;
        c->cdr1 = c->cdr;
    }

    const size_t fb = (size_t)L.fsize;
    const size_t es = esize(c);
    if (c->opts.prec == CE_PREC_FP32) {
        // one block K, G, rx, ry, rz (the TMA path reads it as five slots)
        float* mat = (float*)dev_alloc(c, 5 * fb * sizeof(float));
        if (mat) {
            c->K = mat;
            c->G = mat + fb;
            c->rx = mat + 2 * fb;
            c->ry = mat + 3 * fb;
            c->rz = mat + 4 * fb;
        }
    } else {
        c->K = (float*)dev_alloc(c, fb * sizeof(float));
        c->G = (float*)dev_alloc(c, fb * sizeof(float));
        c->rx = dev_alloc(c, fb * es);
        c->ry = dev_alloc(c, fb * es);
        c->rz = dev_alloc(c, fb * es);
    }
    size_t nstate = (size_t)CE_MAX_CASES * NFIELD * fb * es;
    c->state[0] = dev_alloc(c, nstate);
    if (c->opts.prec == CE_PREC_FP32) c->state[1] = dev_alloc(c, nstate);
    else c->scratch = dev_alloc(c, (size_t)NFIELD * fb * es);
    c->nblk = reduce_blocks(L);
    size_t npart = (size_t)c->nblk * 12;
    if (c->opts.prec == CE_PREC_FP32) {
        size_t nf = (size_t)fused_blocks(L, c->opts.tile);
        if (nf > npart) npart = nf;
        nf = (size_t)fused_tma_blocks(L, c->opts.tile);
        if (nf > npart) npart = nf;
    }
    // refined solves: FP64 w_base of every case and one case's FP64 stresses
    const bool refine = refine_mem && !win && use_tma(c);
    if (refine) {
        c->wb = (double*)dev_alloc(c, (size_t)CE_MAX_CASES * 3 * fb * sizeof(double));
        c->s64 = (double*)dev_alloc(c, (size_t)6 * fb * sizeof(double));
        if ((size_t)rhs_blocks(L) > npart) npart = (size_t)rhs_blocks(L);
    }
    c->partials = (double*)dev_alloc(c, (size_t)CE_MAX_CASES * npart * sizeof(double));
    c->npart = npart;
    c->dres = (double*)dev_alloc(c, (size_t)CE_MAX_CASES * 12 * sizeof(double) + 256);
    bool ok = c->K && c->G && c->rx && c->ry && c->rz && c->state[0] && c->partials && c->dres
           && (c->opts.prec == CE_PREC_FP64 ? c->scratch != nullptr : c->state[1] != nullptr)
           && (!refine || (c->wb && c->s64));
    if (!ok) { ce_status s = fail(c, CE_ENOMEM, "device allocation failed"); release(c); delete c; return s; }
    if (cudaMallocHost(&c->hres, CE_MAX_CASES * 12 * sizeof(double) + 256) != cudaSuccess) {
        release(c);
        delete c;
        return CE_ENOMEM;
    }
    for (auto& e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { release(c); delete c; return CE_ECUDA; }

    auto bail = [&](ce_status s) { release(c); delete c; return s; };
#define CKC(call)                                                                                          \
    do {                                                                                                   \
        if ((call) != cudaSuccess) { cudaGetLastError(); return bail(CE_ECUDA); }                          \
    } while (0)

    CKC(cudaMemsetAsync(c->K, 0, fb * sizeof(float), c->st));
    CKC(cudaMemsetAsync(c->G, 0, fb * sizeof(float), c->st));
    CKC(cudaMemsetAsync(c->rx, 0, fb * es, c->st));
    CKC(cudaMemsetAsync(c->ry, 0, fb * es, c->st));
    CKC(cudaMemsetAsync(c->rz, 0, fb * es, c->st));
    c->derr = (int*)((char*)c->dres + CE_MAX_CASES * 12 * sizeof(double));
    CKC(cudaMemsetAsync(c->derr, 0, sizeof(int), c->st));
    if (use_tma(c)) {
        c->tma = new (std::nothrow) TmaArgs();
        if (!c->tma || !encode_tma_maps(*c->tma, L, c->state[0], c->state[1], c->K, sweep_rows(c->opts.tile),
                                        c->opts.tile[3]))
            return bail(CE_ECUDA);
    }
    CKC(cudaMemsetAsync(c->state[0], 0, nstate, c->st));
    if (c->state[1]) CKC(cudaMemsetAsync(c->state[1], 0, nstate, c->st));
    if (c->scratch) CKC(cudaMemsetAsync(c->scratch, 0, (size_t)NFIELD * fb * es, c->st));

    {
        ce_status us = upload_moduli(c, K, G, moduli_on_device);
        if (us != CE_OK) return bail(us);
    }
#undef CKC
    *out = c;
    return CE_OK;
}

// every failure leaves a message for ce_last_error(NULL)
ce_status create_ctx(const ce_grid* g, const float* K, const float* G, int moduli_on_device, const ce_opts* opts,
                     const ce_allocator* a, void* stream, ce_ctx** out, const Window* win, bool refine_mem)
{
    set_free_error("");
    ce_status s = create_ctx_impl(g, K, G, moduli_on_device, opts, a, stream, out, win, refine_mem);
    if (s != CE_OK && !free_last_error()[0])
        set_free_error("create: %s (device allocation, CUDA set-up or moduli upload)", ce_status_str(s));
    return s;
}

}  // namespace

extern "C" {

ce_status ce_create(const ce_grid* g, const float* K, const float* G, int moduli_on_device,
                    const ce_opts* opts, const ce_allocator* a, void* stream, ce_ctx** out)
{
    return create_ctx(g, K, G, moduli_on_device, opts, a, stream, out, nullptr, true);
}

void ce_destroy(ce_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (ce_ctx* s : c->samples) ce_destroy(s);
    c->samples.clear();
    release(c);
    cudaStreamSynchronize(c->st);
    delete c;
}

ce_status ce_set_moduli(ce_ctx* c, const float* K, const float* G, int moduli_on_device)
{
    if (!c || !K || !G) return CE_EINVAL;
    if (!c->samples.empty()) return fail(c, CE_ENOTIMPL, "a batch takes its moduli at ce_create_batch");
    ce_status s = upload_moduli(c, K, G, moduli_on_device);
    c->have_avg = false;
    c->moduli_ok = s == CE_OK;
    return s;
}

}  // extern "C"

// ------------------------------------------------------------ solve driver
namespace {

template <class T>
ce_status residuals(ce_ctx* c, const int* cases, int n, int zero_w, double* out_norm, ce_solve_info* info)
{
    CK(c, cudaEventRecord(c->ev[2], c->st));
    CaseArgs<T> a[CE_MAX_CASES], s[CE_MAX_CASES];
    for (int q = 0; q < n; ++q) {
        int m = cases[q];
        a[q] = case_args<T>(c, c->cur[m], m);
        if (c->opts.prec == CE_PREC_FP64) {
            for (int f = 0; f < NFIELD; ++f) s[q].f[f] = (T*)c->scratch + (size_t)f * c->L.fsize;
        } else {
            s[q] = case_args<T>(c, 1 - c->cur[m], m);
        }
        s[q].eb = a[q].eb;
    }
    // FP64 solves one case at a time, so the scratch holds one case
    const int per = c->opts.prec == CE_PREC_FP64 ? 1 : n;
    for (int q0 = 0; q0 < n; q0 += per) {
        launch_residual<T>(c->L, c->K, c->G, a + q0, s + q0, per, c->opts.bc, zero_w, c->partials, c->nblk,
                           c->dres + q0, c->st);
        CKL(c);
        info->launches += 3;
    }
    CK(c, cudaEventRecord(c->ev[3], c->st));
    CK(c, cudaMemcpyAsync(c->hres, c->dres, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
    info->check_ms += ms;
    info->checks += 1;
    for (int q = 0; q < n; ++q) out_norm[q] = sqrt(c->hres[q]);
    return CE_OK;
}

// wz0 >= 0: sweep only the local index planes [wz0, wz1) of the window (a
// part of a split slab sweep); flip = false leaves the cases' current
// buffers as they are (the caller flips once every part is done)
template <class T>
ce_status sweep(ce_ctx* c, const int* cases, int n, bool fused, bool check = false, int* nblk_out = nullptr,
                int mode = MODE_DW, int wz0 = -1, int wz1 = -1, bool flip = true)
{
    if (wz0 >= 0 && !(fused && c->tma && c->opts.tile[3] != 2))
        return fail(c, CE_ENOTIMPL, "partial sweeps need the single-column TMA sweep");
    if (mode != MODE_DW && !(fused && c->tma && c->opts.tile[3] != 2))
        return fail(c, CE_ENOTIMPL, "refined solves need the single-column TMA sweep");
    if (fused && c->tma) {
        TmaArgs& ta = *c->tma;
        ta.L = c->L;
        if (wz0 >= 0) {
            ta.L.kz0 = wz0;
            ta.L.kz1 = wz1;
        }
        ta.mode = mode;
        ta.ncase = n;
        ta.bc = c->opts.bc;
        const double th = c->coef_first ? c->theta1 : c->theta;
        ta.a = (float)(th / (1.0 + th));
        for (int q = 0; q < n; ++q) {
            int m = cases[q];
            ta.buf[q] = c->cur[m];
            ta.case_id[q] = m;
            ta.eb[q] = ebar_from_voigt<float>(c->loads[m]);
        }
        ta.partials = check ? c->partials : nullptr;
        ta.err = c->derr;
        int tile[4] = { c->opts.tile[0], c->opts.tile[1], c->opts.tile[2], c->opts.tile[3] };
        // fewer active cases than the tile was sized for: shorter chunks
        // keep the grid's waves full (whole images only)
        if (wz0 < 0 && !c->slab) tile[2] = fused_tma_chunk(ta.L, c->opts.tile, n, c->nsm);
        int nb = launch_fused_tma(ta, tile, c->st);
        if (nblk_out) *nblk_out = nb;
        CKL(c);
        if (flip)
            for (int q = 0; q < n; ++q) c->cur[cases[q]] ^= 1;
        return CE_OK;
    }
    if (fused) {
        FusedArgs fa;
        fa.L = c->L;
        fa.K = c->K; fa.G = c->G;
        fa.rx = (const float*)c->rx; fa.ry = (const float*)c->ry; fa.rz = (const float*)c->rz;
        fa.ncase = n;
        fa.bc = c->opts.bc;
        fa.a = (float)(c->theta / (1.0 + c->theta));
        for (int q = 0; q < n; ++q) {
            int m = cases[q];
            for (int f = 0; f < NFIELD; ++f) {
                fa.in[q][f] = field<float>(c, c->cur[m], m, f);
                fa.out[q][f] = field<float>(c, 1 - c->cur[m], m, f);
            }
            fa.eb[q] = ebar_from_voigt<float>(c->loads[m]);
        }
        fa.partials = check ? c->partials : nullptr;
        int nb = launch_fused_sweep(fa, c->opts.tile, c->st);
        if (nblk_out) *nblk_out = nb;
        CKL(c);
        for (int q = 0; q < n; ++q) c->cur[cases[q]] ^= 1;
        return CE_OK;
    }
    CaseArgs<T> a[CE_MAX_CASES];
    for (int q = 0; q < n; ++q) a[q] = case_args<T>(c, c->cur[cases[q]], cases[q]);
    Relax<T> rp{ (T)(c->theta / (1.0 + c->theta)) };
    launch_plain_sweep<T>(c->L, c->K, c->G, (const T*)c->rx, (const T*)c->ry, (const T*)c->rz, a, n, rp,
                          c->opts.bc, c->st);
    CKL(c);
    return CE_OK;
}

template <class T>
ce_status averages(ce_ctx* c, int n)
{
    CaseArgs<T> a[CE_MAX_CASES];
    for (int m = 0; m < n; ++m) a[m] = case_args<T>(c, c->cur[m], m);
    bool any_wb = false;
    for (int m = 0; m < n; ++m) any_wb = any_wb || c->wb_valid[m];
    if (!any_wb) {
        // the velocity form has no stored stresses: the average kernel forms the
        // elastic stress of the final w itself
        launch_average<T>(c->L, c->K, c->G, a, n, vform(c) ? 1 : 0, c->opts.bc, c->partials, c->nblk, c->dres,
                          c->st);
        CKL(c);
    } else {
        // a refined solve: the elastic stress and strain of the FP64 base
        // (FP64 strains), case by case
        const size_t fs = (size_t)c->L.fsize;
        for (int m = 0; m < n; ++m) {
            if (c->wb_valid[m]) {
                CaseArgs<double> d;
                for (int f = 0; f < NFIELD; ++f) d.f[f] = nullptr;
                for (int f = 0; f < 3; ++f) d.f[F_WX + f] = c->wb + ((size_t)m * 3 + f) * fs;
                d.eb = ebar_from_voigt<double>(c->loads[m]);
                launch_average<double>(c->L, c->K, c->G, &d, 1, 1, c->opts.bc, c->partials, c->nblk,
                                       c->dres + 12 * m, c->st);
            } else {
                launch_average<T>(c->L, c->K, c->G, a + m, 1, 1, c->opts.bc, c->partials, c->nblk, c->dres + 12 * m,
                                  c->st);
            }
            CKL(c);
        }
    }
    CK(c, cudaMemcpyAsync(c->hres, c->dres, (size_t)n * 12 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    const double V = (double)c->L.nx * c->L.ny * c->L.nz;
    for (int m = 0; m < n; ++m)
        for (int t = 0; t < 6; ++t) {
            c->sig[m][t] = c->hres[m * 12 + t] / V;
            c->eps[m][t] = c->hres[m * 12 + 6 + t] / V;
        }
    c->have_avg = true;
    return CE_OK;
}

// ------------------------------------------------------ defect correction
// A refined solve (FP32 TMA sweep of a whole image) iterates on a correction
// dw of an FP64 base w_base with the FP64 right-hand side r (k_refine.cu).
// Rebase of a case: w_base (+)= w or dw, dw = 0, r = div sigma(ebar.x +
// w_base) in FP64 into slots 3-5 of both buffers; its FP64 norm is the exact
// residual.  The first rebase of a solve switches the sweeps to the
// correction phase (all active cases at once, so every launch is of one
// kind); later rebases act on single cases.
//
// When to rebase: the first phase (FP32 w) runs until the residual fell by
// REFINE_FIRST; a correction phase until it fell by REFINE_STEP since the
// case's last rebase, or until it stagnates: over the last REFINE_WINDOW
// checks the residual fell by less than a quarter of what the phase's
// average rate would give (after at least 2 REFINE_WINDOW checks).  A
// correction phase's own FP32 floor does not shrink with the residual
// (measured: about 2e-8 of ||div sigma(0)|| on a porous 48^3 image), so short
// phases and a rebase on stagnation keep the FP64 residual falling.  The
// first phase stops on the same stagnation test once its residual is below
// REFINE_EXIT and it has run 4 REFINE_WINDOW checks (past the start-up
// transient), for images whose FP32 w alone floors above REFINE_FIRST.
constexpr double REFINE_FIRST = 1e-3;
constexpr double REFINE_STEP = 1e-2;
constexpr int REFINE_WINDOW = 4;
constexpr double REFINE_EXIT = 1e-1;

bool can_refine(const ce_ctx* c) { return c->wb && c->s64 && c->tma && c->opts.tile[3] != 2 && !c->slab; }

ce_status rebase(ce_ctx* c, const int* ms, int nm, const bool* first, bool lo_valid, double* out,
                 ce_solve_info* info)
{
    CK(c, cudaEventRecord(c->ev[2], c->st));
    const size_t fs = (size_t)c->L.fsize;
    const int nb = rhs_blocks(c->L);
    for (int q = 0; q < nm; ++q) {
        const int m = ms[q];
        const int cur = c->cur[m];
        double* wb = c->wb + (size_t)m * 3 * fs;
        RefineW rw;
        const __nv_bfloat16* lxy = (const __nv_bfloat16*)field<float>(c, cur, m, F_WLO_XY);
        const __nv_bfloat16* lz = (const __nv_bfloat16*)field<float>(c, cur, m, F_WLO_Z);
        for (int f = 0; f < 3; ++f) {
            rw.wb[f] = wb + f * fs;
            rw.hi[f] = field<float>(c, cur, m, F_WX + f);
        }
        rw.lo[0] = lo_valid ? lxy : nullptr;
        rw.lo[1] = lo_valid ? lxy + fs : nullptr;
        rw.lo[2] = lo_valid ? lz : nullptr;
        launch_rebase_w(c->L, rw, first[q] ? 1 : 0, c->st);
        CKL(c);
        CaseArgs<double> src, dst;
        for (int f = 0; f < NFIELD; ++f) src.f[f] = dst.f[f] = nullptr;
        for (int f = 0; f < 3; ++f) src.f[F_WX + f] = wb + f * fs;
        for (int f = 0; f < 6; ++f) dst.f[f] = c->s64 + f * fs;
        src.eb = dst.eb = ebar_from_voigt<double>(c->loads[m]);
        launch_elastic_stress<double>(c->L, c->K, c->G, &src, &dst, 1, c->opts.bc, c->st);
        CKL(c);
        RefineR rr;
        for (int f = 0; f < 6; ++f) rr.s[f] = c->s64 + f * fs;
        for (int f = 0; f < 3; ++f) {
            rr.r0[f] = field<float>(c, 0, m, F_RX + f);
            rr.r1[f] = field<float>(c, 1, m, F_RX + f);
        }
        launch_rhs(c->L, rr, c->partials + (size_t)q * nb, c->st);
        CKL(c);
        info->launches += 3;
    }
    launch_reduce(c->partials, nb, nm, c->dres, c->st);
    CKL(c);
    info->launches += 1;
    CK(c, cudaEventRecord(c->ev[3], c->st));
    CK(c, cudaMemcpyAsync(c->hres, c->dres, nm * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    float t_ms = 0.f;
    CK(c, cudaEventElapsedTime(&t_ms, c->ev[2], c->ev[3]));
    info->check_ms += t_ms;
    info->rebases += nm;
    for (int q = 0; q < nm; ++q) out[q] = sqrt(c->hres[q]);
    return CE_OK;
}

// back to the ordinary layout: w = w_base as a double-word value in the
// current buffer; the idle buffer's slots 3-5 (r) cleared
ce_status finalize(ce_ctx* c, int m)
{
    c->wb_valid[m] = true;
    const size_t fs = (size_t)c->L.fsize;
    const int cur = c->cur[m];
    const double* wb = c->wb + (size_t)m * 3 * fs;
    RefineF a;
    __nv_bfloat16* lxy = (__nv_bfloat16*)field<float>(c, cur, m, F_WLO_XY);
    __nv_bfloat16* lz = (__nv_bfloat16*)field<float>(c, cur, m, F_WLO_Z);
    for (int f = 0; f < 3; ++f) {
        a.wb[f] = wb + f * fs;
        a.hi[f] = field<float>(c, cur, m, F_WX + f);
    }
    a.lo[0] = lxy;
    a.lo[1] = lxy + fs;
    a.lo[2] = lz;
    a.lo_pad = lz + fs;
    a.slot5 = field<float>(c, cur, m, F_RZ);
    launch_finalize(c->L, a, c->st);
    CKL(c);
    CK(c, cudaMemsetAsync(field<float>(c, 1 - cur, m, F_RX), 0, 3 * fs * sizeof(float), c->st));
    return CE_OK;
}

// the node coefficients dt~/rho~ (and theta) of the first phase of a refined
// solve (first) or of every other sweep; recomputed only when they change
ce_status set_phase(ce_ctx* c, bool first)
{
    if (first == c->coef_first || c->opts.prec != CE_PREC_FP32) return CE_OK;
    launch_node_coef<float>(c->L, c->K, c->G, (float*)c->rx, (float*)c->ry, (float*)c->rz,
                            first ? c->cdr1 : c->cdr, c->st);
    CKL(c);
    c->coef_first = first;
    return CE_OK;
}

// leaves the context with the ordinary coefficients on every way out of a solve
struct PhaseRestore {
    ce_ctx* c;
    ~PhaseRestore() { set_phase(c, false); }
};

// the pseudo-time loop for the cases in `cases` (all advanced together)
template <class T>
ce_status run_cases(ce_ctx* c, const int* cases, int n, double tol, int max_iter, bool warm, bool fused,
                    ce_solve_info* info, unsigned flags = 0)
{
    ce_status s;
    double r0[CE_MAX_CASES], r[CE_MAX_CASES];
    // defect correction (refined solve): see rebase()
    const bool refine = fused && sizeof(T) == sizeof(float) && can_refine(c) && !(flags & CE_NO_REFINE);
    // a refined solve from the initial state starts in its first phase, at
    // that phase's Strouhal number (u_{-1} of the initial state included)
    PhaseRestore restore{ c };
    if ((s = set_phase(c, refine && !warm && c->cdr1 != c->cdr)) != CE_OK) return s;
    if (fused) {
        // velocity form: buffer 1 first holds sigma(ebar) = T(0), from which u
        // of buffer 0 becomes r div T(0); w = 0 and lo = 0 in both buffers,
        // u = 0 in buffer 1 where the sweep never writes it
        if (!warm) {
            CaseArgs<T> a[CE_MAX_CASES], b[CE_MAX_CASES];
            for (int q = 0; q < n; ++q) {
                c->cur[cases[q]] = 0;
                a[q] = case_args<T>(c, 0, cases[q]);
                b[q] = case_args<T>(c, 1, cases[q]);
            }
            launch_init<T>(c->L, c->K, c->G, a, n, c->opts.bc, c->st);
            CKL(c);
            launch_init<T>(c->L, c->K, c->G, b, n, c->opts.bc, c->st);
            CKL(c);
            launch_uinit<T>(c->L, (const T*)c->rx, (const T*)c->ry, (const T*)c->rz, b, a, n, c->st);
            CKL(c);
            info->launches += 3;
            for (int q = 0; q < n; ++q)
                CK(c, cudaMemsetAsync((void*)a[q].f[F_WLO_XY], 0, 2 * (size_t)c->L.fsize * sizeof(T), c->st));
        }
        // residual norms use the idle buffer's first six slots as scratch
        if ((s = residuals<T>(c, cases, n, 1, r0, info)) != CE_OK) return s;
        if (warm) {
            if ((s = residuals<T>(c, cases, n, 0, r, info)) != CE_OK) return s;
        } else {
            for (int q = 0; q < n; ++q) r[q] = r0[q];
        }
        for (int q = 0; q < n; ++q) {
            CaseArgs<T> idle = case_args<T>(c, 1 - c->cur[cases[q]], cases[q]);
            CK(c, cudaMemsetAsync((void*)idle.f[F_UX], 0, 5 * (size_t)c->L.fsize * sizeof(T), c->st));
        }
    } else {
        if (!warm) {
            CaseArgs<T> a[CE_MAX_CASES];
            for (int q = 0; q < n; ++q) {
                c->cur[cases[q]] = 0;
                a[q] = case_args<T>(c, 0, cases[q]);
            }
            launch_init<T>(c->L, c->K, c->G, a, n, c->opts.bc, c->st);
            CKL(c);
            info->launches += 1;
        }
        if ((s = residuals<T>(c, cases, n, 1, r0, info)) != CE_OK) return s;
        if ((s = residuals<T>(c, cases, n, 0, r, info)) != CE_OK) return s;
    }
    int active[CE_MAX_CASES], na = 0;
    for (int q = 0; q < n; ++q) {
        int m = cases[q];
        info->res0[m] = r0[q];
        info->rel_res[m] = r0[q] > 0 ? r[q] / r0[q] : 0.0;
        info->iters[m] = 0;
        if (info->rel_res[m] <= tol) info->status[m] = CE_OK;
        else { info->status[m] = CE_ENOTCONV; active[na++] = m; }
    }
    const bool each = (flags & CE_REFINE_EACH_CHECK) != 0;
    bool rhs = false;                      // sweeps in the correction phase
    bool based[CE_MAX_CASES] = {};         // the case has a w_base
    for (int q = 0; q < n; ++q) c->wb_valid[cases[q]] = false;
    double ref[CE_MAX_CASES];              // relative residual at its last rebase
    double hist[CE_MAX_CASES][REFINE_WINDOW + 1];   // residuals of the last checks since it
    int nhist[CE_MAX_CASES] = {};
    int nchk[CE_MAX_CASES] = {};           // checks since its last rebase
    for (int m = 0; m < CE_MAX_CASES; ++m) ref[m] = 1.0;
    if (refine && warm && na > 0) {
        // a warm start keeps its double-word w: rebase at once (the first
        // phase runs on FP32 w alone and would drop the low part)
        bool first[CE_MAX_CASES];
        double r64[CE_MAX_CASES];
        for (int q = 0; q < na; ++q) first[q] = true;
        if ((s = rebase(c, active, na, first, true, r64, info)) != CE_OK) return s;
        int keep[CE_MAX_CASES], nk = 0;
        for (int q = 0; q < na; ++q) {
            const int m = active[q];
            const double rl = info->res0[m] > 0 ? r64[q] / info->res0[m] : 0.0;
            info->rel_res[m] = rl;
            ref[m] = rl;
            based[m] = true;
            if (!isfinite(rl) || rl > 1e10) info->status[m] = CE_EDIVERGED;
            else if (rl <= tol) info->status[m] = CE_OK;
            else { keep[nk++] = m; continue; }
            if ((s = finalize(c, m)) != CE_OK) return s;
        }
        na = nk;
        for (int q = 0; q < nk; ++q) active[q] = keep[q];
        rhs = true;
    }
    int it = 0;
    while (na > 0 && it < max_iter) {
        int ns = max_iter - it < c->n_check ? max_iter - it : c->n_check;
        CK(c, cudaEventRecord(c->ev[0], c->st));
        int nb = 0;
        for (int q = 0; q < ns; ++q) {
            // the fused path measures the residual inside its last sweep
            bool chk = fused && q == ns - 1;
            const int mode = !refine ? MODE_DW : rhs ? MODE_RHS : MODE_F32;
            if ((s = sweep<T>(c, active, na, fused, chk, &nb, mode)) != CE_OK) return s;
        }
        CK(c, cudaEventRecord(c->ev[1], c->st));
        it += ns;
        info->sweeps += ns;
        info->case_sweeps += (long long)ns * na;
        {
            const double vox = (double)c->L.nx * c->L.ny * c->L.nz;
            // the first phase of a refined solve keeps w in FP32 alone (48 B)
            const double per_case = (refine && !rhs) ? 48.0 : 60.0;
            const double per = fused ? per_case * na + 8.0 : (c->opts.prec == CE_PREC_FP64 ? 160.0 : 80.0) * na;
            info->teff_gbs += (double)ns * per * vox;   // bytes for now; divided by the time at the end
        }
        info->launches += ns * (fused ? 1 : 2);
        if (fused) {
            // residual of the state before the last sweep: ||div T(w)|| per case
            launch_reduce(c->partials, nb, na, c->dres, c->st);
            CKL(c);
            info->launches += 1;
            info->checks += 1;
            CK(c, cudaMemcpyAsync(c->hres, c->dres, CE_MAX_CASES * 12 * sizeof(double) + sizeof(int),
                                  cudaMemcpyDeviceToHost, c->st));
            CK(c, cudaStreamSynchronize(c->st));
            if (*(int*)(c->hres + CE_MAX_CASES * 12))
                return fail(c, CE_ECUDA, "a TMA wait of the fused sweep timed out");
            for (int q = 0; q < na; ++q) r[q] = sqrt(c->hres[q]);
        } else {
            if ((s = residuals<T>(c, active, na, 0, r, info)) != CE_OK) return s;
        }
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        info->sweep_ms += ms;
        if (rhs) {
            info->sweeps_corr += ns;
            info->case_sweeps_corr += (long long)ns * na;
            info->sweep_ms_corr += ms;
        }
        double rel[CE_MAX_CASES];
        for (int q = 0; q < na; ++q) {
            int m = active[q];
            rel[q] = info->res0[m] > 0 ? r[q] / info->res0[m] : 0.0;
            info->rel_res[m] = rel[q];
            info->iters[m] = it;
        }
        if (refine) {
            // rebase the cases whose residual fell by REFINE_STEP since their
            // last rebase, or reached tol; the first rebase takes every
            // active case into the correction phase.  Convergence is then
            // decided by the FP64 residual of the rebased state.
            auto sane = [](double v) { return isfinite(v) && v <= 1e10; };
            for (int q = 0; q < na; ++q) {
                int m = active[q];
                if (nhist[m] == REFINE_WINDOW + 1) {
                    for (int k = 0; k < REFINE_WINDOW; ++k) hist[m][k] = hist[m][k + 1];
                    --nhist[m];
                }
                hist[m][nhist[m]++] = rel[q];
                ++nchk[m];
            }
            auto due = [&](int q) {
                const int m = active[q];
                if (each || rel[q] <= fmax(tol, (rhs ? REFINE_STEP : REFINE_FIRST) * ref[m])) return true;
                // a phase that stopped gaining (the first one only past its
                // start-up transient)
                if (!(rel[q] < ref[m]) || !(rel[q] > 0.0)) return false;
                if (rhs ? nchk[m] < 2 * REFINE_WINDOW : (nchk[m] < 4 * REFINE_WINDOW || rel[q] > REFINE_EXIT))
                    return false;
                const double avg = log(ref[m] / rel[q]) / nchk[m];       // per check since the rebase
                const double last = log(hist[m][0] / rel[q]);            // over the last REFINE_WINDOW checks
                return last < 0.25 * REFINE_WINDOW * avg;
            };
            bool any = false;
            for (int q = 0; q < na; ++q) any = any || (sane(rel[q]) && due(q));
            int wq[CE_MAX_CASES], ms[CE_MAX_CASES], nw = 0;
            bool first[CE_MAX_CASES];
            double r64[CE_MAX_CASES];
            for (int q = 0; q < na; ++q)
                if (sane(rel[q]) && (due(q) || (!rhs && any))) {
                    wq[nw] = q;
                    ms[nw] = active[q];
                    first[nw] = !based[active[q]];
                    ++nw;
                }
            if (nw > 0) {
                // (the first phase keeps no low part of w)
                if ((s = rebase(c, ms, nw, first, false, r64, info)) != CE_OK) return s;
                for (int k = 0; k < nw; ++k) {
                    const int m = ms[k];
                    const double rl = info->res0[m] > 0 ? r64[k] / info->res0[m] : 0.0;
                    rel[wq[k]] = rl;
                    info->rel_res[m] = rl;
                    ref[m] = rl;
                    based[m] = true;
                    nhist[m] = 0;
                    nchk[m] = 0;
                }
                rhs = true;
                // the correction phases run at the ordinary Strouhal number
                if ((s = set_phase(c, false)) != CE_OK) return s;
            }
        }
        int keep[CE_MAX_CASES], nk = 0;
        for (int q = 0; q < na; ++q) {
            int m = active[q];
            bool done = true;
            if (!isfinite(rel[q]) || rel[q] > 1e10) info->status[m] = CE_EDIVERGED;
            else if (rel[q] <= tol) info->status[m] = CE_OK;
            else { keep[nk++] = m; done = false; }
            if (done && based[m] && (s = finalize(c, m)) != CE_OK) return s;
        }
        na = nk;
        for (int q = 0; q < nk; ++q) active[q] = keep[q];
    }
    // cases still running at max_iter: back to the ordinary layout too
    for (int q = 0; q < na; ++q)
        if (based[active[q]] && (s = finalize(c, active[q])) != CE_OK) return s;
    return CE_OK;
}

}  // namespace

extern "C" ce_status ce_solve(ce_ctx* c, const double* loads, int n_cases, double tol, int max_iter,
                              unsigned flags, ce_solve_info* info)
{
    if (!c) return CE_EINVAL;
    if (c->slab) return fail(c, CE_ENOTIMPL, "a slab context is driven by the ce_slab_* calls");
    if (n_cases < 1 || n_cases > CE_MAX_CASES || max_iter < 0 || !(tol >= 0))
        return fail(c, CE_EINVAL, "bad n_cases, max_iter or tol");
    if (!loads && n_cases != 6) return fail(c, CE_EINVAL, "loads == NULL needs n_cases == 6");
    const bool warm = (flags & CE_WARM_START) != 0;
    if (!c->moduli_ok) return fail(c, CE_ESTATE, "the moduli were rejected; set valid ones first");
    if (warm && (!c->have_state || c->n_cases != n_cases))
        return fail(c, CE_ESTATE, "warm start without a prior solve of as many cases");
    auto t0 = std::chrono::steady_clock::now();
    for (int m = 0; m < n_cases; ++m)
        for (int t = 0; t < 6; ++t) {
            double v = loads ? loads[m * 6 + t] : (m == t ? 1.0 : 0.0);
            if (!isfinite(v)) return fail(c, CE_EINVAL, "non-finite load");
            c->loads[m][t] = v;
        }
    c->unit_loads = n_cases == 6;
    for (int m = 0; m < n_cases && c->unit_loads; ++m)
        for (int t = 0; t < 6; ++t)
            if (c->loads[m][t] != (m == t ? 1.0 : 0.0)) c->unit_loads = false;
    c->n_cases = n_cases;
    c->have_avg = false;
    ce_solve_info inf;
    memset(&inf, 0, sizeof inf);
    inf.n_cases = n_cases;
    ce_status s = CE_OK;
    if (c->opts.prec == CE_PREC_FP64) {
        for (int m = 0; m < n_cases && s == CE_OK; ++m)
            s = run_cases<double>(c, &m, 1, tol, max_iter, warm, false, &inf);
        if (s == CE_OK) s = averages<double>(c, n_cases);
        inf.launches += 2;
    } else {
        int all[CE_MAX_CASES];
        for (int m = 0; m < n_cases; ++m) all[m] = m;
        bool fused = c->opts.kernel != CE_KERNEL_PLAIN;
        if (!fused && warm)
            for (int m = 0; m < n_cases; ++m)
                if (c->cur[m] != 0) return fail(c, CE_ESTATE, "warm start across kernel kinds");
        s = run_cases<float>(c, all, n_cases, tol, max_iter, warm, fused, &inf, flags);
        if (s == CE_OK) s = averages<float>(c, n_cases);
        inf.launches += 2;
    }
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inf.teff_gbs = inf.sweep_ms > 0 ? inf.teff_gbs / (inf.sweep_ms * 1e-3) / 1e9 : 0.0;
    if (info) *info = inf;
    if (s != CE_OK) return s;
    c->have_state = true;
    ce_status worst = CE_OK;
    for (int m = 0; m < n_cases; ++m) {
        if (inf.status[m] == CE_EDIVERGED) worst = CE_EDIVERGED;
        else if (inf.status[m] == CE_ENOTCONV && worst == CE_OK) worst = CE_ENOTCONV;
    }
    if (worst == CE_ENOTCONV) fail(c, worst, "max_iter reached before tol");
    if (worst == CE_EDIVERGED) fail(c, worst, "residual not finite or above 1e10");
    return worst;
}

namespace {

bool invert6(const double* A, double* Ai)
{
    double M[6][12];
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 12; ++q) M[r][q] = q < 6 ? A[r * 6 + q] : (q - 6 == r ? 1.0 : 0.0);
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        for (int r = col + 1; r < 6; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (!(fabs(M[piv][col]) > 1e-300)) return false;
        if (piv != col)
            for (int q = 0; q < 12; ++q) { double t = M[col][q]; M[col][q] = M[piv][q]; M[piv][q] = t; }
        double d = M[col][col];
        for (int q = 0; q < 12; ++q) M[col][q] /= d;
        for (int r = 0; r < 6; ++r)
            if (r != col) {
                double f = M[r][col];
                for (int q = 0; q < 12; ++q) M[r][q] -= f * M[col][q];
            }
    }
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) Ai[r * 6 + q] = M[r][q + 6];
    return true;
}

}  // namespace

// C = S E^-1 from the per-case sums of ce_slab_sums added over the slabs
// (or ranks) of one grid: the averages are the sums over nx ny nz.
extern "C" ce_status ce_ceff_from_sums(const double* sums, int n_cases, const ce_grid* g, double C[36])
{
    if (!sums || !g || !C) return free_fail(CE_EINVAL, "ceff_from_sums: NULL argument");
    if (n_cases != 6) return free_fail(CE_EINVAL, "ceff_from_sums: needs the sums of six load cases");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return free_fail(CE_EINVAL, "ceff_from_sums: bad grid");
    const double V = (double)g->nx * g->ny * g->nz;
    double S[36], E[36], Ei[36];
    for (int r = 0; r < 6; ++r)
        for (int m = 0; m < 6; ++m) {
            S[r * 6 + m] = sums[m * 12 + r] / V;       // column m: <sigma> of case m
            E[r * 6 + m] = sums[m * 12 + 6 + r] / V;   // column m: <eps> of case m
        }
    if (!invert6(E, Ei)) return free_fail(CE_EINVAL, "ceff_from_sums: the strain averages are singular");
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) {
            double v = 0.0;
            for (int k = 0; k < 6; ++k) v += S[r * 6 + k] * Ei[k * 6 + q];
            C[r * 6 + q] = v;
        }
    return CE_OK;
}

extern "C" ce_status ce_ceff(const ce_ctx* c, double C[36])
{
    if (!c || !C) return CE_EINVAL;
    if (!c->have_avg || c->n_cases != 6) return CE_ESTATE;
    // S and E with columns <sigma>^m, <eps>^m; C = S E^-1
    double S[36], E[36], Ei[36];
    for (int r = 0; r < 6; ++r)
        for (int m = 0; m < 6; ++m) {
            S[r * 6 + m] = c->sig[m][r];
            E[r * 6 + m] = c->eps[m][r];
        }
    if (!invert6(E, Ei)) return CE_EINVAL;
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) {
            double t = 0;
            for (int m = 0; m < 6; ++m) t += S[r * 6 + m] * Ei[m * 6 + q];
            C[r * 6 + q] = t;
        }
    return CE_OK;
}

// The paper's direct tests (Appendix A.1 and A.3): C11, C22, C33 from the
// three single-axis normal tests (Eq. eq:4) and C12, C13, C23 from the
// combined test by Eqs. D1-D5.
extern "C" ce_status ce_direct_tests(const ce_ctx* c, double out[6])
{
    if (!c || !out) return CE_EINVAL;
    if (!c->have_avg || c->n_cases != 4)
        return fail(const_cast<ce_ctx*>(c), CE_ESTATE, "ce_direct_tests needs a solve of the four direct-test loads");
    for (int q = 0; q < 4; ++q)
        for (int t = 0; t < 6; ++t) {
            const bool on = q < 3 ? t == q : t < 3;
            if ((c->loads[q][t] != 0.0) != on)
                return fail(const_cast<ce_ctx*>(c), CE_ESTATE,
                            "ce_direct_tests: loads must be e1, e2, e3 and e1 + e2 + e3 (any nonzero scale)");
        }
    double cd[3], sb[3], eb[3];
    for (int q = 0; q < 3; ++q) {
        if (!(fabs(c->eps[q][q]) > 0.0)) return fail(const_cast<ce_ctx*>(c), CE_EINVAL, "zero normal strain");
        cd[q] = c->sig[q][q] / c->eps[q][q];                          // Eq. eq:4
    }
    for (int i = 0; i < 3; ++i) {
        eb[i] = c->eps[3][i];                                          // Eq. D2
        sb[i] = c->sig[3][i] - cd[i] * eb[i];                          // Eq. D1
        if (!(fabs(eb[i]) > 0.0)) return fail(const_cast<ce_ctx*>(c), CE_EINVAL, "zero strain in the combined test");
    }
    out[0] = cd[0];
    out[1] = cd[1];
    out[2] = cd[2];
    out[3] = (eb[0] * sb[0] + eb[1] * sb[1] - eb[2] * sb[2]) / (2.0 * eb[0] * eb[1]);   // C12, Eq. D3
    out[4] = (eb[0] * sb[0] - eb[1] * sb[1] + eb[2] * sb[2]) / (2.0 * eb[0] * eb[2]);   // C13, Eq. D4
    out[5] = (-eb[0] * sb[0] + eb[1] * sb[1] + eb[2] * sb[2]) / (2.0 * eb[1] * eb[2]);  // C23, Eq. D5
    return CE_OK;
}

extern "C" ce_status ce_averages(const ce_ctx* c, double* sig, double* eps)
{
    if (!c || !sig || !eps) return CE_EINVAL;
    if (!c->have_avg) return CE_ESTATE;
    for (int m = 0; m < c->n_cases; ++m)
        for (int t = 0; t < 6; ++t) {
            sig[m * 6 + t] = c->sig[m][t];
            eps[m * 6 + t] = c->eps[m][t];
        }
    return CE_OK;
}

extern "C" ce_status ce_get_field(const ce_ctx* cc, int m, int f, double* host_out)
{
    ce_ctx* c = const_cast<ce_ctx*>(cc);
    if (!c || !host_out || m < 0 || m >= CE_MAX_CASES || f < 0 || f >= NFIELD + 3) return CE_EINVAL;
    if (f >= NFIELD && !vform(c)) return fail(c, CE_EINVAL, "fields 9-11 exist in the velocity form only");
    const Layout& L = c->L;
    size_t n = (size_t)(L.nx + 1) * (L.ny + 1) * (L.nz + 1);
    double* d = (double*)c->partials;   // reuse the reduction scratch when it is large enough
    size_t cap = (size_t)CE_MAX_CASES * c->nblk * 12;
    bool tmp = n > cap;
    if (tmp) {
        if (cudaMallocAsync((void**)&d, n * sizeof(double), c->st) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CE_ENOMEM, "no room for the field copy");
        }
    }
    if (c->opts.prec == CE_PREC_FP64) {
        launch_gather_field<double>(L, field<double>(c, c->cur[m], m, f), d, c->st);
    } else if (!vform(c)) {
        launch_gather_field<float>(L, field<float>(c, c->cur[m], m, f), d, c->st);
    } else {
        launch_gather_vform(L, c->K, c->G, case_args<float>(c, c->cur[m], m), f, c->opts.bc, d, c->st);
    }
    CKL(c);
    CK(c, cudaMemcpyAsync(host_out, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (tmp) {
        cudaFreeAsync(d, c->st);
        cudaStreamSynchronize(c->st);
    }
    return CE_OK;
}

extern "C" ce_status ce_grad(ce_ctx* c, const double w[36], float* dJdK, float* dJdG, int out_on_device)
{
    if (!c || !w || !dJdK || !dJdG) return CE_EINVAL;
    if (c->slab) return fail(c, CE_ENOTIMPL, "ce_grad acts on whole-grid contexts");
    if (!c->have_avg || !c->unit_loads) return fail(c, CE_ESTATE, "ce_grad needs a solve of the six unit cases");
    const Layout& L = c->L;
    const size_t n = (size_t)L.nx * L.ny * L.nz;
    double ws[36];
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) ws[a * 6 + b] = 0.5 * (w[a * 6 + b] + w[b * 6 + a]);
    float *dK = dJdK, *dG = dJdG;
    double* dw = c->dres;   // 36 doubles fit in the reduction output block
    if (!out_on_device) {
        if (cudaMallocAsync((void**)&dK, 2 * n * sizeof(float), c->st) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CE_ENOMEM, "no room for the gradient");
        }
        dG = dK + n;
    }
    CK(c, cudaMemcpyAsync(dw, ws, sizeof ws, cudaMemcpyHostToDevice, c->st));
    CaseArgs<float> a32[CE_MAX_CASES];
    CaseArgs<double> a64[CE_MAX_CASES];
    // a refined FP32 solve keeps its final w in the FP64 base: FP64 strains
    bool wb = c->wb != nullptr;
    for (int m = 0; m < 6; ++m) wb = wb && c->wb_valid[m];
    const bool f64 = c->opts.prec == CE_PREC_FP64 || wb;
    for (int m = 0; m < 6; ++m) {
        if (c->opts.prec == CE_PREC_FP64) {
            a64[m] = case_args<double>(c, c->cur[m], m);
        } else if (wb) {
            for (int f = 0; f < NFIELD; ++f) a64[m].f[f] = nullptr;
            for (int f = 0; f < 3; ++f) a64[m].f[F_WX + f] = c->wb + ((size_t)m * 3 + f) * (size_t)L.fsize;
            a64[m].eb = ebar_from_voigt<double>(c->loads[m]);
        } else {
            a32[m] = case_args<float>(c, c->cur[m], m);
        }
    }
    launch_grad(L, c->K, c->G, f64 ? nullptr : a32, f64 ? a64 : nullptr, dw, dK, dG, c->opts.bc, c->st);
    CKL(c);
    if (!out_on_device) {
        CK(c, cudaMemcpyAsync(dJdK, dK, n * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        CK(c, cudaMemcpyAsync(dJdG, dG, n * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        CK(c, cudaStreamSynchronize(c->st));
        cudaFreeAsync(dK, c->st);
    }
    CK(c, cudaStreamSynchronize(c->st));
    return CE_OK;
}

// -------------------------------------------------------------- autotuner
// Grid search over the TMA sweep's launch shapes for this context: copy
// stages x rows per block x z-planes per block.  Each candidate runs a few
// sweeps of all six unit load cases from the current state (the next
// non-warm ce_solve starts afresh, so the state's values do not matter) and
// is timed with events on the context's stream; the fastest becomes the
// context's tile.
extern "C" ce_status ce_autotune_for(ce_ctx* c, int sweeps, int solves, int* tile_out, double* ms_out)
{
    if (!c) return CE_EINVAL;
    if (solves != CE_TUNE_AUTO && solves != CE_TUNE_PLAIN && solves != CE_TUNE_REFINED)
        return fail(c, CE_EINVAL, "solves must be CE_TUNE_AUTO, CE_TUNE_PLAIN or CE_TUNE_REFINED");
    if (!c->samples.empty() || c->slab) return fail(c, CE_ENOTIMPL, "autotune acts on single-image contexts");
    if (!use_tma(c)) return fail(c, CE_ENOTIMPL, "autotune needs the FP32 TMA sweep");
    if (sweeps < 1 || sweeps > 1000) return fail(c, CE_EINVAL, "sweeps must be 1..1000");
    // longer chunks cost fewer warm-up planes and ring fills per sweep
    // (measured at 191^3: 128 planes 2 % faster than 64)
    static const int kPlanes[9] = { 16, 24, 32, 48, 64, 96, 128, 192, 256 };
    // (columns per thread, copy stages) pairs, times rows {8, 16} and, for
    // the single-column sweep, 24
    static const int kKind[5][2] = { { 1, 3 }, { 1, 2 }, { 2, 3 }, { 2, 4 }, { 2, 2 } };
    for (int m = 0; m < CE_MAX_CASES; ++m)
        for (int t = 0; t < 6; ++t) c->loads[m][t] = m == t ? 1.0 : 0.0;
    c->n_cases = CE_MAX_CASES;
    c->unit_loads = true;
    c->have_avg = false;
    int all[CE_MAX_CASES] = { 0, 1, 2, 3, 4, 5 };
    const int keep[4] = { c->opts.tile[0], c->opts.tile[1], c->opts.tile[2], c->opts.tile[3] };
    int best[4] = { 0, 0, 0, 0 };
    float best_ms = 0.f;
    // refined solves are timed in their two sweep modes (first phase and
    // correction phase, half the sweeps each), and only on the single-column
    // sweep, the one they run on; the others in the double-word mode
    const bool can = c->wb && c->s64 && !c->slab;
    if (solves == CE_TUNE_REFINED && !can) return fail(c, CE_ENOTIMPL, "this context runs no refined solves");
    const bool refined = solves == CE_TUNE_REFINED || (solves == CE_TUNE_AUTO && can);
    for (int a = 0; a < 5; ++a) {
        if (refined && kKind[a][0] != 1) continue;
        for (int rows = 8; rows <= (kKind[a][0] == 1 ? 24 : 16); rows += 8) {
            if (!encode_tma_maps(*c->tma, c->L, c->state[0], c->state[1], c->K, rows, kKind[a][0]))
                return fail(c, CE_ECUDA, "tensor map encoding failed");
            for (int z = 0; z < 9; ++z) {
                c->opts.tile[0] = kKind[a][1];
                c->opts.tile[1] = rows;
                c->opts.tile[2] = kPlanes[z];
                c->opts.tile[3] = kKind[a][0];
                for (int w = 0; w < 2; ++w) {
                    ce_status st = sweep<float>(c, all, CE_MAX_CASES, true, false, nullptr,
                                                refined ? MODE_F32 : MODE_DW);
                    if (st != CE_OK) return st;
                }
                CK(c, cudaEventRecord(c->ev[2], c->st));
                for (int w = 0; w < sweeps; ++w) {
                    const int mode = !refined ? MODE_DW : 2 * w < sweeps ? MODE_F32 : MODE_RHS;
                    ce_status st = sweep<float>(c, all, CE_MAX_CASES, true, false, nullptr, mode);
                    if (st != CE_OK) return st;
                }
                CK(c, cudaEventRecord(c->ev[3], c->st));
                CK(c, cudaEventSynchronize(c->ev[3]));
                float ms = 0.f;
                CK(c, cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
                ms /= (float)sweeps;
                if (best[0] == 0 || ms < best_ms) {
                    best_ms = ms;
                    for (int q = 0; q < 4; ++q) best[q] = c->opts.tile[q];
                }
            }
        }
    }
    int hostflag = 0;
    CK(c, cudaMemcpy(&hostflag, c->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (hostflag) {
        for (int q = 0; q < 4; ++q) c->opts.tile[q] = keep[q];
        encode_tma_maps(*c->tma, c->L, c->state[0], c->state[1], c->K, sweep_rows(keep), keep[3]);
        return fail(c, CE_ECUDA, "a TMA wait of the sweep timed out while tuning");
    }
    // the chosen shape may need more residual partials than were allocated
    size_t nb = (size_t)fused_tma_blocks(c->L, best);
    if (nb > c->npart) {
        double* p = (double*)dev_alloc(c, (size_t)CE_MAX_CASES * nb * sizeof(double));
        if (!p) return fail(c, CE_ENOMEM, "device allocation failed");
        c->partials = p;
        c->npart = nb;
    }
    for (int q = 0; q < 4; ++q) c->opts.tile[q] = best[q];
    if (!encode_tma_maps(*c->tma, c->L, c->state[0], c->state[1], c->K, sweep_rows(best), best[3]))
        return fail(c, CE_ECUDA, "tensor map encoding failed");
    for (int m = 0; m < CE_MAX_CASES; ++m) c->cur[m] = 0;
    c->have_state = false;   // the timing sweeps overwrote the fields
    if (tile_out)
        for (int q = 0; q < 4; ++q) tile_out[q] = best[q];
    if (ms_out) *ms_out = best_ms;
    return CE_OK;
}

extern "C" ce_status ce_autotune(ce_ctx* c, int sweeps, int* tile_out, double* ms_out)
{
    return ce_autotune_for(c, sweeps, CE_TUNE_AUTO, tile_out, ms_out);
}

extern "C" ce_status ce_set_tile(ce_ctx* c, const int tile[4])
{
    if (!c || !tile) return CE_EINVAL;
    if (!c->samples.empty()) return fail(c, CE_ENOTIMPL, "set the tile of a batch at ce_create_batch");
    int t[4] = { tile[0], tile[1], tile[2], tile[3] == 2 ? 2 : 1 };
    const bool pair = t[3] == 2;
    if (pair && c->slab) return fail(c, CE_ENOTIMPL, "slabs run the single-column sweep");
    if ((t[0] != 0 && t[0] != 2 && t[0] != 3 && !(pair && t[0] == 4))
        || (t[1] != 0 && t[1] != 8 && t[1] != 16 && !(t[1] == 24 && !pair)) || t[2] < 0
        || (tile[3] != 0 && tile[3] != 1 && tile[3] != 2))
        return fail(c, CE_EINVAL,
                    "tile: stages 0, 2, 3 (or 4 paired); rows 0, 8, 16 (or 24 single); planes >= 0; cols 0, 1 or 2");
    if (vform(c)) {
        size_t nb = (size_t)fused_tma_blocks(c->L, t);
        if ((size_t)fused_blocks(c->L, t) > nb) nb = (size_t)fused_blocks(c->L, t);
        if (nb > c->npart) {
            double* p = (double*)dev_alloc(c, (size_t)CE_MAX_CASES * nb * sizeof(double));
            if (!p) return fail(c, CE_ENOMEM, "device allocation failed");
            c->partials = p;
            c->npart = nb;
        }
        if (use_tma(c) && !encode_tma_maps(*c->tma, c->L, c->state[0], c->state[1], c->K, sweep_rows(t), t[3]))
            return fail(c, CE_ECUDA, "tensor map encoding failed");
    }
    for (int q = 0; q < 4; ++q) c->opts.tile[q] = t[q];
    return CE_OK;
}

// ------------------------------------------------------------------ batches
namespace {

// per-check control of the batched solve (one block): reduce the residual
// partials of every active sample and load case in a fixed order, retire
// converged, diverged or exhausted samples, and keep the graph's WHILE loop
// running while any sample is active (first > 0: while any active sample's
// largest relative residual is above first, the end of the first phase).  A
// sample whose sweeps raised the device error flag (a copy wait that timed
// out, a bad block mapping) is retired with CE_ECUDA, and its residuals are
// not trusted.
__global__ void k_batch_control(cudaGraphConditionalHandle h, int nsamp, int nchk, const BatchEntry* ents,
                                int* ints, double* dbl, const double* part, int pstride, double first)
{
    int* active = ints;
    int* parity = ints + nsamp;
    int* iters = ints + 2 * nsamp;
    int* status = ints + 3 * nsamp;
    const double* res0 = dbl;
    double* rel = dbl + 6 * nsamp;
    const double tol = dbl[12 * nsamp], maxit = dbl[12 * nsamp + 1];
    __shared__ double sh[32];
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int s = 0; s < nsamp; ++s) {
        if (!active[s]) continue;
        if (*ents[s].a.err) {
            if (threadIdx.x == 0) {
                active[s] = 0;
                status[s] = CE_ECUDA;
            }
            __syncthreads();
            continue;
        }
        const int nb = ents[s].nbx * ents[s].nby * ents[s].nch;
        bool all_ok = true, bad = false;
        double worst = 0.0;
        for (int m = 0; m < CE_MAX_CASES; ++m) {
            double v = 0.0;
            const double* p = part + ((size_t)s * CE_MAX_CASES + m) * pstride;
            for (int b = threadIdx.x; b < nb; b += blockDim.x) v += p[b];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
                double r0 = res0[s * CE_MAX_CASES + m];
                rel[s * CE_MAX_CASES + m] = r0 > 0 ? sqrt(t) / r0 : 0.0;
            }
            __syncthreads();
            double rr = rel[s * CE_MAX_CASES + m];
            if (rr > worst) worst = rr;
            if (!(rr <= tol)) all_ok = false;
            if (!isfinite(rr) || rr > 1e10) bad = true;
        }
        if (threadIdx.x == 0) {
            iters[s] += nchk;
            parity[s] = (parity[s] + nchk) & 1;
            if (bad) { active[s] = 0; status[s] = CE_EDIVERGED; }
            else if (all_ok) { active[s] = 0; status[s] = CE_OK; }
            else if ((double)iters[s] >= maxit) { active[s] = 0; status[s] = CE_ENOTCONV; }
            else if (!(first > 0.0) || worst > first) any = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// The graph: for the single-column sweep a first phase (w in FP32 alone, no
// low part read or written: 48 instead of 60 B per voxel and case) while any
// active sample's residual is above BATCH_FIRST, then the double-word sweep
// until every sample is done.  The low parts are zero from the initial state
// and stay zero in the first phase, so the second phase starts from the
// double-word value of the FP32 w.
constexpr double BATCH_FIRST = 1e-3;

ce_status build_batch_graph(ce_ctx* c)
{
    const int n = (int)c->samples.size();
    CK(c, cudaGraphCreate(&c->graph, 0));
    const BatchEntry* ents = c->d_ents;
    int* active = c->d_int;
    int* parity = c->d_int + n;
    double* part = c->d_part;
    int nsamp = n, pstride = c->pstride;
    // one WHILE loop: n_check sweeps over all active samples in a chain (the
    // last one also writes residual partials), then the control kernel
    auto add_loop = [&](int mode, double first, cudaGraphNode_t* dep, cudaGraphNode_t* out) -> ce_status {
        cudaGraphConditionalHandle h;
        CK(c, cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        CK(c, cudaGraphAddNode(out, c->graph, dep, nullptr, dep ? 1 : 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t prev = nullptr;
        for (int k = 0; k < c->batch_nchk; ++k) {
            int smem = 0;
            const bool chk = k == c->batch_nchk - 1;
            const void* fn = c->opts.tile[3] == 2
                                 ? pair_batch_kernel(c->batch_ty, c->opts.tile[0] == 4 ? 4 : 3, chk, &smem)
                                 : batch_kernel(c->batch_ty, c->opts.tile[0] == 2 ? 2 : 3, chk, mode, &smem);
            if (!fn) return fail(c, CE_ECUDA, "cannot set the shared memory of the batched sweep");
            int kk = k;
            void* args[] = { (void*)&ents, (void*)&nsamp, (void*)&active, (void*)&parity, (void*)&kk, (void*)&part,
                             (void*)&pstride };
            cudaKernelNodeParams kp = {};
            kp.func = const_cast<void*>(fn);
            kp.gridDim = dim3((unsigned)c->total_blocks);
            kp.blockDim = dim3(32, (unsigned)c->batch_ty);
            kp.sharedMemBytes = (unsigned)smem;
            kp.kernelParams = args;
            cudaGraphNode_t nd;
            CK(c, cudaGraphAddKernelNode(&nd, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
            prev = nd;
        }
        int nchk = c->batch_nchk;
        int* ints = c->d_int;
        double* dbl = c->d_dbl;
        const double* cpart = c->d_part;
        void* args[] = { (void*)&h, (void*)&nsamp, (void*)&nchk, (void*)&ents, (void*)&ints, (void*)&dbl,
                         (void*)&cpart, (void*)&pstride, (void*)&first };
        cudaKernelNodeParams kp = {};
        kp.func = reinterpret_cast<void*>(k_batch_control);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(256);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t nd;
        CK(c, cudaGraphAddKernelNode(&nd, body, &prev, 1, &kp));
        return CE_OK;
    };
    cudaGraphNode_t first_loop = nullptr, second_loop = nullptr;
    ce_status st;
    // (the paired-column sweep keeps the double-word state throughout)
    if (c->opts.tile[3] != 2 && (st = add_loop(MODE_F32, BATCH_FIRST, nullptr, &first_loop)) != CE_OK) return st;
    if ((st = add_loop(MODE_DW, 0.0, first_loop ? &first_loop : nullptr, &second_loop)) != CE_OK) return st;
    CK(c, cudaGraphInstantiate(&c->gexec, c->graph, 0));
    return CE_OK;
}

}  // namespace

extern "C" ce_status ce_create_batch(int n, const ce_grid* g, const float* const* K, const float* const* G,
                                     int moduli_on_device, const ce_opts* opts, const ce_allocator* a,
                                     void* stream, ce_ctx** out)
{
    set_free_error("");
    if (!out) return free_fail(CE_EINVAL, "create_batch: NULL output pointer");
    *out = nullptr;
    if (n < 1 || n > 1024 || !g || !K || !G) return free_fail(CE_EINVAL, "create_batch: n outside 1..1024 or NULL");
    ce_ctx* c = new (std::nothrow) ce_ctx();
    if (!c) return free_fail(CE_ENOMEM, "create_batch: out of host memory");
    ce_default_opts(&c->opts);
    if (opts) c->opts = *opts;
    if (c->opts.prec != CE_PREC_FP32) { delete c; return free_fail(CE_ENOTIMPL, "create_batch: FP32 only"); }
    c->opts.kernel = CE_KERNEL_FUSED;
    if (a) { c->alloc = *a; c->own_alloc = false; }
    c->st = (cudaStream_t)stream;
    c->opts.tile[3] = c->opts.tile[3] == 2 ? 2 : 1;
    c->batch_ty = sweep_rows(c->opts.tile);
    c->batch_nchk = c->opts.n_check > 0 ? c->opts.n_check : 32;
    ce_opts so = c->opts;
    so.tile[1] = c->batch_ty;
    std::vector<BatchEntry> ents((size_t)n);
    int off = 0, pmax = 0;
    for (int s = 0; s < n; ++s) {
        ce_ctx* sc = nullptr;
        ce_status st = create_ctx(&g[s], K[s], G[s], moduli_on_device, &so, a, stream, &sc, nullptr, false);
        if (st != CE_OK) {
            ce_destroy(c);
            char msg[256];
            snprintf(msg, sizeof msg, "create_batch: sample %d: %s", s, free_last_error());
            return free_fail(st, msg);
        }
        c->samples.push_back(sc);
        BatchEntry& e = ents[s];
        e.a = *sc->tma;
        e.a.L = sc->L;
        e.a.ncase = CE_MAX_CASES;
        e.a.bc = sc->opts.bc;
        e.a.a = (float)(sc->theta / (1.0 + sc->theta));
        double unit[6] = { 0, 0, 0, 0, 0, 0 };
        for (int q = 0; q < CE_MAX_CASES; ++q) {
            e.a.buf[q] = 0;
            e.a.case_id[q] = q;
            unit[q] = 1.0;
            e.a.eb[q] = ebar_from_voigt<float>(unit);
            unit[q] = 0.0;
        }
        e.a.partials = nullptr;
        e.a.err = sc->derr;
        batch_geometry(sc->L, so.tile, &e.nbx, &e.nby, &e.nch, &e.zc);
        e.off = off;
        int nb = e.nbx * e.nby * e.nch;
        // the single-column batched sweep gives each load case of a tile its
        // own block; the paired-column one sweeps all cases in each block
        off += nb * (so.tile[3] == 2 ? 1 : CE_MAX_CASES);
        if (nb > pmax) pmax = nb;
    }
    c->total_blocks = off;
    c->pstride = pmax;
    c->d_ents = (BatchEntry*)dev_alloc(c, ents.size() * sizeof(BatchEntry));
    c->d_int = (int*)dev_alloc(c, 4 * (size_t)n * sizeof(int));
    c->d_dbl = (double*)dev_alloc(c, (12 * (size_t)n + 2) * sizeof(double));
    c->d_part = (double*)dev_alloc(c, (size_t)n * CE_MAX_CASES * pmax * sizeof(double));
    if (!c->d_ents || !c->d_int || !c->d_dbl || !c->d_part) {
        ce_destroy(c);
        return free_fail(CE_ENOMEM, "create_batch: device allocation failed");
    }
    if (cudaMemcpyAsync(c->d_ents, ents.data(), ents.size() * sizeof(BatchEntry), cudaMemcpyHostToDevice, c->st)
            != cudaSuccess
        || cudaMallocHost(&c->hres, (12 * (size_t)n + 2) * sizeof(double) + 4 * (size_t)n * sizeof(int)) != cudaSuccess
        || cudaStreamSynchronize(c->st) != cudaSuccess) {
        cudaGetLastError();
        ce_destroy(c);
        return free_fail(CE_ECUDA, "create_batch: copy of the sample descriptors failed");
    }
    *out = c;
    return CE_OK;
}

extern "C" ce_status ce_solve_batch(ce_ctx* c, double tol, int max_iter, int* iters)
{
    if (!c || c->samples.empty()) return CE_EINVAL;
    if (!(tol >= 0) || max_iter < 0) return fail(c, CE_EINVAL, "bad tol or max_iter");
    const int n = (int)c->samples.size();
    std::vector<int> hint(4 * (size_t)n, 0);
    std::vector<double> hdbl(12 * (size_t)n + 2, 0.0);
    // per sample: initial state and ||div T(0)|| of the six unit cases
    for (int s = 0; s < n; ++s) {
        ce_ctx* sc = c->samples[s];
        ce_solve_info inf;
        memset(&inf, 0, sizeof inf);
        for (int m = 0; m < 6; ++m)
            for (int t = 0; t < 6; ++t) sc->loads[m][t] = m == t ? 1.0 : 0.0;
        sc->n_cases = 6;
        sc->unit_loads = true;
        sc->have_avg = false;
        int all[CE_MAX_CASES] = { 0, 1, 2, 3, 4, 5 };
        ce_status st = run_cases<float>(sc, all, 6, tol, 0, false, true, &inf);
        if (st != CE_OK) return fail(c, st, "sample %d: %s", s, sc->err);
        bool any = false;
        for (int m = 0; m < 6; ++m) {
            hdbl[(size_t)s * 6 + m] = inf.res0[m];
            if (inf.res0[m] > 0) any = true;
        }
        hint[s] = (any && max_iter > 0) ? 1 : 0;                  // active
        hint[3 * (size_t)n + s] = any ? CE_ENOTCONV : CE_OK;
    }
    hdbl[12 * (size_t)n] = tol;
    hdbl[12 * (size_t)n + 1] = (double)max_iter;
    CK(c, cudaMemcpyAsync(c->d_int, hint.data(), hint.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->d_dbl, hdbl.data(), hdbl.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    if (!c->gexec) {
        ce_status st = build_batch_graph(c);
        if (st != CE_OK) {
            if (c->graph) cudaGraphDestroy(c->graph);
            c->graph = nullptr;
            return st;
        }
    }
    bool any_active = false;
    for (int s = 0; s < n; ++s) any_active = any_active || hint[s];
    if (any_active) CK(c, cudaGraphLaunch(c->gexec, c->st));
    CK(c, cudaMemcpyAsync(hint.data(), c->d_int, hint.size() * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaMemcpyAsync(hdbl.data(), c->d_dbl, hdbl.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    for (int s = 0; s < n; ++s)
        if (hint[3 * (size_t)n + s] == CE_ECUDA)
            return fail(c, CE_ECUDA, "sample %d: a TMA wait of the batched sweep timed out", s);
    ce_status worst = CE_OK;
    for (int s = 0; s < n; ++s) {
        ce_ctx* sc = c->samples[s];
        const int par = hint[(size_t)n + s];
        for (int m = 0; m < 6; ++m) sc->cur[m] = par;
        ce_status st = averages<float>(sc, 6);
        if (st != CE_OK) return fail(c, st, "sample %d averages: %s", s, sc->err);
        int ss = hint[3 * (size_t)n + s];
        if (ss == CE_EDIVERGED) worst = CE_EDIVERGED;
        else if (ss == CE_ENOTCONV && worst == CE_OK) worst = CE_ENOTCONV;
        if (iters) iters[s] = hint[2 * (size_t)n + s];
    }
    c->n_cases = 6;
    c->have_avg = true;
    return worst;
}

extern "C" ce_status ce_ceff_batch(const ce_ctx* c, double* C)
{
    if (!c || !C) return CE_EINVAL;
    if (c->samples.empty()) return CE_ESTATE;
    for (size_t s = 0; s < c->samples.size(); ++s) {
        ce_status st = ce_ceff(c->samples[s], C + 36 * s);
        if (st != CE_OK) return st;
    }
    return CE_OK;
}

// ------------------------------------------------------------ z-slabs
// One context per slab of a z-decomposed grid (the domain decomposition the
// paper plans for several GPUs, Sec. 5.3).  The caller drives the loop: sweep,
// pack the two boundary planes, move the messages to the neighbours (device
// copies or send/receive between ranks), unpack, and every n_check sweeps
// sum the slabs' squared residuals.  The arithmetic of every point is that
// of the whole-grid sweep, so the slabs' fields equal the whole grid's.
namespace {

bool slab_window(const ce_grid* g, int z0, int z1, int* c0, int* c1)
{
    if (!g || g->nx < 2 || g->ny < 2 || g->nz < 2) return false;
    if (z0 < 0 || z1 > g->nz + 1 || z1 - z0 < 1) return false;
    const int zoff = z0 > 0 ? z0 - 1 : 0;                 // ghost plane below
    const int ztop = z1 < g->nz ? z1 : g->nz;             // ghost plane above (or the top face)
    *c0 = zoff;
    *c1 = ztop < g->nz ? ztop + 1 : g->nz;                // the ghost plane's cells are read
    return *c1 - *c0 >= 2;
}

// the buffer holding each case's newest state: the next one while a split
// sweep has written its boundary planes and not yet its interior
HaloArgs halo_args(const ce_ctx* c)
{
    HaloArgs h;
    for (int m = 0; m < CE_MAX_CASES; ++m)
        h.base[m] = m < c->n_cases ? field<float>(c, c->slab_pend[m] ? 1 - c->cur[m] : c->cur[m], m, 0) : nullptr;
    return h;
}

}  // namespace

extern "C" ce_status ce_sweep_chunk(const ce_grid* g, const int tile[4], int n_cases, int n_sm, int* planes)
{
    set_free_error("");
    if (!g || !tile || !planes || g->nx < 2 || g->ny < 2 || g->nz < 2 || n_cases < 1 || n_cases > CE_MAX_CASES)
        return free_fail(CE_EINVAL, "sweep_chunk: bad grid, tile, case count or NULL output");
    Layout L{};
    L.nx = g->nx;
    L.ny = g->ny;
    L.nz = g->nz;
    L.pitch = ((g->nx + 1) + 31) / 32 * 32;
    L.plane = (long long)L.pitch * (g->ny + 1);
    L.fsize = L.plane * (g->nz + 1);
    L.kz0 = 0;
    L.kz1 = g->nz + 1;
    L.nzg = g->nz;
    const int t[4] = { tile[0], tile[1], tile[2], tile[3] == 2 ? 2 : 1 };
    *planes = fused_tma_chunk(L, t, n_cases, n_sm);
    return CE_OK;
}

extern "C" ce_status ce_slab_cells(const ce_grid* g, int z0, int z1, int* c0, int* c1)
{
    if (!c0 || !c1) return free_fail(CE_EINVAL, "slab_cells: NULL output");
    return slab_window(g, z0, z1, c0, c1) ? CE_OK
                                          : free_fail(CE_EINVAL, "slab_cells: planes outside 0..nz or window < 2 cells");
}

extern "C" ce_status ce_create_slab(const ce_grid* g, int z0, int z1, const float* K, const float* G,
                                    int moduli_on_device, const ce_opts* opts, const ce_allocator* a,
                                    void* stream, ce_ctx** out)
{
    int c0, c1;
    set_free_error("");
    if (!out) return free_fail(CE_EINVAL, "create_slab: NULL output pointer");
    *out = nullptr;
    if (!slab_window(g, z0, z1, &c0, &c1))
        return free_fail(CE_EINVAL, "create_slab: planes outside 0..nz or window < 2 cells");
    ce_grid lg = *g;
    lg.nz = c1 - c0;
    Window w{ c0, g->nz, z0 - c0, z1 - c0 };
    return create_ctx(&lg, K, G, moduli_on_device, opts, a, stream, out, &w, false);
}

extern "C" ce_status ce_slab_start(ce_ctx* c, const double* loads, int n_cases, double* b2)
{
    if (!c || !b2) return CE_EINVAL;
    if (!c->slab) return fail(c, CE_ESTATE, "not a slab context");
    if (n_cases < 1 || n_cases > CE_MAX_CASES) return fail(c, CE_EINVAL, "bad n_cases");
    if (!loads && n_cases != 6) return fail(c, CE_EINVAL, "loads == NULL needs n_cases == 6");
    if (!c->moduli_ok) return fail(c, CE_ESTATE, "the moduli were rejected");
    for (int m = 0; m < n_cases; ++m)
        for (int t = 0; t < 6; ++t) {
            double v = loads ? loads[m * 6 + t] : (m == t ? 1.0 : 0.0);
            if (!isfinite(v)) return fail(c, CE_EINVAL, "non-finite load");
            c->loads[m][t] = v;
        }
    c->n_cases = n_cases;
    c->have_avg = false;
    c->have_state = false;
    c->slab_nres = 0;
    c->slab_npend = 0;
    for (int m = 0; m < CE_MAX_CASES; ++m) c->slab_pend[m] = false;
    // the whole-grid initial state (run_cases): T(0) in buffer 1, u = r div
    // T(0) in buffer 0, w = 0; then ||div T(0)||^2 over the own faces
    CaseArgs<float> a[CE_MAX_CASES], b[CE_MAX_CASES], sc[CE_MAX_CASES];
    for (int m = 0; m < n_cases; ++m) {
        c->cur[m] = 0;
        a[m] = case_args<float>(c, 0, m);
        b[m] = case_args<float>(c, 1, m);
    }
    launch_init<float>(c->L, c->K, c->G, a, n_cases, c->opts.bc, c->st);
    CKL(c);
    launch_init<float>(c->L, c->K, c->G, b, n_cases, c->opts.bc, c->st);
    CKL(c);
    launch_uinit<float>(c->L, (const float*)c->rx, (const float*)c->ry, (const float*)c->rz, b, a, n_cases, c->st);
    CKL(c);
    for (int m = 0; m < n_cases; ++m)
        CK(c, cudaMemsetAsync((void*)a[m].f[F_WLO_XY], 0, 2 * (size_t)c->L.fsize * sizeof(float), c->st));
    for (int m = 0; m < n_cases; ++m) {
        a[m] = case_args<float>(c, 0, m);
        sc[m] = case_args<float>(c, 1, m);
        sc[m].eb = a[m].eb;
    }
    launch_residual<float>(c->L, c->K, c->G, a, sc, n_cases, c->opts.bc, 1, c->partials, c->nblk, c->dres, c->st);
    CKL(c);
    for (int m = 0; m < n_cases; ++m)
        CK(c, cudaMemsetAsync((void*)sc[m].f[F_UX], 0, 5 * (size_t)c->L.fsize * sizeof(float), c->st));
    CK(c, cudaMemcpyAsync(c->hres, c->dres, n_cases * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    for (int m = 0; m < n_cases; ++m) b2[m] = c->hres[m];
    c->have_state = true;
    return CE_OK;
}

extern "C" ce_status ce_slab_sweep(ce_ctx* c, const int* cases, int n, int n_sweeps, int check)
{
    if (!c) return CE_EINVAL;
    if (!c->slab || !c->have_state) return fail(c, CE_ESTATE, "ce_slab_start first");
    int all[CE_MAX_CASES];
    if (!cases) {
        n = c->n_cases;
        for (int m = 0; m < n; ++m) all[m] = m;
        cases = all;
    }
    if (n < 1 || n > c->n_cases || n_sweeps < 1) return fail(c, CE_EINVAL, "bad case list or sweep count");
    if (c->slab_npend) return fail(c, CE_ESTATE, "a split sweep is waiting for its part 2");
    for (int q = 0; q < n; ++q) {
        if (cases[q] < 0 || cases[q] >= c->n_cases) return fail(c, CE_EINVAL, "bad case index");
        for (int p = 0; p < q; ++p)
            if (cases[p] == cases[q]) return fail(c, CE_EINVAL, "repeated case index");
    }
    c->have_avg = false;
    int nb = 0;
    for (int s = 0; s < n_sweeps; ++s) {
        const bool chk = check && s == n_sweeps - 1;
        ce_status st = sweep<float>(c, cases, n, true, chk, &nb);
        if (st != CE_OK) return st;
    }
    c->slab_nres = 0;
    if (check) {
        launch_reduce(c->partials, nb, n, c->dres, c->st);
        CKL(c);
        c->slab_nres = n;
    }
    return CE_OK;
}

// One sweep in two parts, so that the halo exchange can overlap the
// interior: part 1 updates the own planes next to a neighbour (plane z0 with
// a neighbour below, z1 - 1 with one above); ce_slab_pack then packs them
// from the new state; part 2 updates the remaining own planes and completes
// the sweep.  Every own plane is updated once, from the old state, as in
// ce_slab_sweep, so the fields are those of an unsplit sweep.
extern "C" ce_status ce_slab_sweep_part(ce_ctx* c, const int* cases, int n, int part)
{
    if (!c) return CE_EINVAL;
    if (!c->slab || !c->have_state) return fail(c, CE_ESTATE, "ce_slab_start first");
    if (part != 1 && part != 2) return fail(c, CE_EINVAL, "part must be 1 (boundary planes) or 2 (interior)");
    int all[CE_MAX_CASES];
    if (!cases) {
        n = c->n_cases;
        for (int m = 0; m < n; ++m) all[m] = m;
        cases = all;
    }
    if (n < 1 || n > c->n_cases) return fail(c, CE_EINVAL, "bad case list");
    for (int q = 0; q < n; ++q) {
        if (cases[q] < 0 || cases[q] >= c->n_cases) return fail(c, CE_EINVAL, "bad case index");
        for (int p = 0; p < q; ++p)
            if (cases[p] == cases[q]) return fail(c, CE_EINVAL, "repeated case index");
    }
    const int kz0 = c->L.kz0, kz1 = c->L.kz1;
    const bool lower = kz0 >= 1, upper = kz1 <= c->L.nz;
    c->have_avg = false;
    c->slab_nres = 0;
    ce_status st;
    if (part == 1) {
        if (c->slab_npend) return fail(c, CE_ESTATE, "part 1 again before part 2");
        if (lower && (st = sweep<float>(c, cases, n, true, false, nullptr, MODE_DW, kz0, kz0 + 1, false)) != CE_OK)
            return st;
        if (upper && kz1 - 1 > (lower ? kz0 : kz0 - 1)
            && (st = sweep<float>(c, cases, n, true, false, nullptr, MODE_DW, kz1 - 1, kz1, false)) != CE_OK)
            return st;
        for (int q = 0; q < n; ++q) c->slab_pend[cases[q]] = true;
        c->slab_npend = n;
        return CE_OK;
    }
    if (c->slab_npend != n) return fail(c, CE_ESTATE, "part 2 needs the cases of part 1");
    for (int q = 0; q < n; ++q)
        if (!c->slab_pend[cases[q]]) return fail(c, CE_ESTATE, "part 2 needs the cases of part 1");
    const int a = kz0 + (lower ? 1 : 0), b = kz1 - (upper ? 1 : 0);
    if (b > a && (st = sweep<float>(c, cases, n, true, false, nullptr, MODE_DW, a, b, false)) != CE_OK) return st;
    for (int q = 0; q < n; ++q) {
        c->cur[cases[q]] ^= 1;
        c->slab_pend[cases[q]] = false;
    }
    c->slab_npend = 0;
    return CE_OK;
}

extern "C" ce_status ce_slab_residual(ce_ctx* c, double* r2)
{
    if (!c || !r2) return CE_EINVAL;
    if (!c->slab || c->slab_nres < 1) return fail(c, CE_ESTATE, "no checked sweep to read");
    CK(c, cudaMemcpyAsync(c->hres, c->dres, CE_MAX_CASES * 12 * sizeof(double) + sizeof(int),
                          cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (*(int*)(c->hres + CE_MAX_CASES * 12)) return fail(c, CE_ECUDA, "a TMA wait of the fused sweep timed out");
    for (int q = 0; q < c->slab_nres; ++q) r2[q] = c->hres[q];
    return CE_OK;
}

extern "C" ce_status ce_slab_halo_bytes(const ce_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return CE_EINVAL;
    if (!c->slab || !c->have_state) return fail(const_cast<ce_ctx*>(c), CE_ESTATE, "ce_slab_start first");
    *bytes = halo_bytes(c->L, c->n_cases);
    return CE_OK;
}

extern "C" ce_status ce_slab_pack(ce_ctx* c, int side, void* msg)
{
    if (!c || !msg || (side != 0 && side != 1)) return CE_EINVAL;
    if (!c->slab || !c->have_state) return fail(c, CE_ESTATE, "ce_slab_start first");
    if ((reinterpret_cast<uintptr_t>(msg) & 15) != 0) return fail(c, CE_EINVAL, "message not 16-byte aligned");
    const int plane = side == 0 ? c->L.kz0 : c->L.kz1 - 1;
    launch_halo(c->L, halo_args(c), c->n_cases, plane, msg, 0, c->st);
    CKL(c);
    return CE_OK;
}

extern "C" ce_status ce_slab_unpack(ce_ctx* c, int side, const void* msg)
{
    if (!c || !msg || (side != 0 && side != 1)) return CE_EINVAL;
    if (!c->slab || !c->have_state) return fail(c, CE_ESTATE, "ce_slab_start first");
    if ((reinterpret_cast<uintptr_t>(msg) & 15) != 0) return fail(c, CE_EINVAL, "message not 16-byte aligned");
    const int plane = side == 0 ? c->L.kz0 - 1 : c->L.kz1;
    if (plane < 0 || plane > c->L.nz) return fail(c, CE_EINVAL, "this side has no neighbour");
    launch_halo(c->L, halo_args(c), c->n_cases, plane, const_cast<void*>(msg), 1, c->st);
    CKL(c);
    return CE_OK;
}

extern "C" ce_status ce_slab_sums(ce_ctx* c, double* sums)
{
    if (!c || !sums) return CE_EINVAL;
    if (!c->slab || !c->have_state) return fail(c, CE_ESTATE, "ce_slab_start first");
    const int n = c->n_cases;
    CaseArgs<float> a[CE_MAX_CASES];
    for (int m = 0; m < n; ++m) a[m] = case_args<float>(c, c->cur[m], m);
    launch_average<float>(c->L, c->K, c->G, a, n, 1, c->opts.bc, c->partials, c->nblk, c->dres, c->st);
    CKL(c);
    CK(c, cudaMemcpyAsync(c->hres, c->dres, (size_t)n * 12 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    for (int q = 0; q < n * 12; ++q) sums[q] = c->hres[q];
    return CE_OK;
}
