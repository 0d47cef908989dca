// sw_api.cu -- the C ABI declared in include/sw_elliptic.h: grid handles,
// coefficient storage, workspace, argument checks and kernel launches.
#include <cstddef>
#include <string>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/sw_elliptic.h"
#include "sw_common.cuh"
#include "sw_internal.h"

using namespace sw;

static thread_local std::string g_err;

static sw_status fail(sw_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

sw_status sw::api_fail(sw_status st, const char *msg) { return fail(st, msg); }

static sw_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

struct sw_grid_s {
    int nx, ny, device, sms;
    double radius, dlam, dphi;
    size_t N;
    // coefficient storage (one allocation)
    void *cmem;
    double *ax, *cx, *bx, *ay, *cy, *by, *C, *diag, *lf, *invD, *zz, *gam, *ec, *rowmax, *eta;
    double *gam32, *ec32;          // per row, of the FP32 zonal factors
    bool f64_valid;                // the FP64 zonal factors match the coefficients and eta
    float *wax, *wcx, *wbx, *way, *wcy, *wby, *wC, *wdiag, *lf32, *invD32, *zz32;
    // the zonal factors transposed per row for the warp-per-row solver (rows
    // of a power of two of at least 128 points; null otherwise)
    double *lfT, *invDT, *zzT;
    float *lf32T, *invD32T, *zz32T;
    // split fluid thickness (Sec. 4.2, Eq. 14): Phi_hat and its derivative
    // parts, allocated by the first sw_split_refresh
    void *split_mem;
    float *shat, *sdx, *scx, *sdy, *scy;
    bool split_valid;
    bool has_coeffs;
    double eta_explicit;           // > 0 when chosen by sw_grid_set_eta
    // solver workspace
    void *ws;
    size_t ws_bytes;
    bool ws_owned;
    SolverBlock *blk;              // device: member state of this grid
    EnsDesc *desc;                 // device: launch descriptor when this grid leads a launch
    EnsDesc *h_desc;               // pinned host staging of desc
    MemberCtl *h_ctl;              // pinned host copies read after a solve
    void *h_mdev;                  // pinned staging of the member descriptor (recorded async solves)
    GlobalCtl *h_g;
    double *h_eta;
    // async solves outside a graph capture: a ring of pinned staging slots
    // (member descriptor + launch descriptor), each reused only after the
    // copies that read it have run (its event)
    unsigned char *h_ring;
    cudaEvent_t ring_ev[4];
    int ring_next;
    // the learned preconditioner's loop on the device (a CUDA graph with a
    // conditional node) and what its nodes hold
    cudaGraphExec_t lgraph;
    unsigned long long lkey[14];
    cudaStream_t lcap;             // a stream of its own to capture the loop on (not the legacy stream)
};

constexpr int RING = 4;

static size_t ring_slot_bytes() { return ((sizeof(SolverBlock::dev) + 255) & ~(size_t)255) + sizeof(EnsDesc); }

GridGeom sw::grid_geom(const sw_grid_s *g) { return GridGeom{g->nx, g->ny, g->sms > 0 ? g->sms : 1, g->radius}; }

GridView sw::grid_view(const sw_grid_s *g)
{
    return GridView{g->nx, g->ny, g->device, g->sms, g->wax, g->way, g->wdiag};
}

// threads of the block that works on one row: about four values per thread,
// at least nx/16 (the tridiagonal chunks live in registers, 16 values at most)
static int row_threads(int nx, int requested = 0)
{
    int t = requested > 0 ? requested : ((nx / 4 + 31) / 32) * 32;
    const int tmin = ((nx + 16 * 32 - 1) / (16 * 32)) * 32;
    if (t < tmin) t = tmin;
    if (t < 32) t = 32;
    if (t > MAX_THREADS) t = MAX_THREADS;
    return t;
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" void sw_solve_opts_default(sw_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->k = 4;
    o->tol = 1e-8;
    o->max_iters = 1000;
    o->min_iters = 0;
    o->pc = SW_PC_SI_RICHARDSON;
    o->n_richardson = 2;
    o->eta = 0.0;
    o->omega = 1.0;
    o->prec = SW_PREC_FP64;
    o->pole_band_rows = -1;
    o->ru_every = 0;
    o->fb_ratio = 0.5;
}

extern "C" const char *sw_last_error(void) { return g_err.c_str(); }

extern "C" sw_status sw_grid_create(int nx, int ny, double radius, sw_grid *out)
{
    if (!out) return fail(SW_ERR_INVALID_ARG, "sw_grid_create: out is NULL");
    *out = nullptr;
    if (nx < 4 || nx > MAX_NX || (nx & 1)) return fail(SW_ERR_INVALID_ARG, "sw_grid_create: nx must be even, 4..4096");
    if (ny < 2 || ny > 65536) return fail(SW_ERR_INVALID_ARG, "sw_grid_create: ny must be 2..65536");
    if (!(radius > 0.0) || !std::isfinite(radius)) return fail(SW_ERR_INVALID_ARG, "sw_grid_create: radius must be > 0");
    sw_grid g = new (std::nothrow) sw_grid_s();
    if (!g) return fail(SW_ERR_OOM, "sw_grid_create: host allocation failed");
    g->nx = nx; g->ny = ny; g->radius = radius;
    g->dlam = 2.0 * M_PI / nx; g->dphi = M_PI / ny;
    g->N = (size_t)nx * ny;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device);
    size_t N = g->N;
    const bool wt = warp_rows_ok(nx);
    size_t bytes = 11 * al(N * 8) + 5 * al((size_t)ny * 8) + al(8) + 11 * al(N * 4) + (wt ? 3 * (al(N * 8) + al(N * 4)) : 0);
    if (e == cudaSuccess) e = cudaMalloc(&g->cmem, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->blk, sizeof(SolverBlock));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->desc, sizeof(EnsDesc));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_desc, sizeof(EnsDesc));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_ctl, sizeof(MemberCtl) + sizeof(GlobalCtl) + 64);
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_mdev, sizeof(SolverBlock::dev));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_ring, RING * ring_slot_bytes());
    int nev = 0;
    for (; e == cudaSuccess && nev < RING; ++nev) e = cudaEventCreateWithFlags(&g->ring_ev[nev], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (g->cmem) cudaFree(g->cmem);
        if (g->blk) cudaFree(g->blk);
        if (g->desc) cudaFree(g->desc);
        if (g->h_desc) cudaFreeHost(g->h_desc);
        if (g->h_ctl) cudaFreeHost(g->h_ctl);
        if (g->h_mdev) cudaFreeHost(g->h_mdev);
        if (g->h_ring) cudaFreeHost(g->h_ring);
        for (int q = 0; q + 1 < nev; ++q) cudaEventDestroy(g->ring_ev[q]);
        delete g;
        return cuda_fail(e, "sw_grid_create");
    }
    g->h_g = (GlobalCtl *)((char *)g->h_ctl + sizeof(MemberCtl));
    g->h_eta = (double *)((char *)g->h_g + sizeof(GlobalCtl) + 16);
    char *p = (char *)g->cmem;
    double **d64[] = {&g->ax, &g->cx, &g->bx, &g->ay, &g->cy, &g->by, &g->C, &g->diag, &g->lf, &g->invD, &g->zz};
    for (auto q : d64) { *q = (double *)p; p += al(N * 8); }
    g->gam = (double *)p; p += al((size_t)ny * 8);
    g->ec = (double *)p; p += al((size_t)ny * 8);
    g->rowmax = (double *)p; p += al((size_t)ny * 8);
    g->gam32 = (double *)p; p += al((size_t)ny * 8);
    g->ec32 = (double *)p; p += al((size_t)ny * 8);
    g->eta = (double *)p; p += al(8);
    float **d32[] = {&g->wax, &g->wcx, &g->wbx, &g->way, &g->wcy, &g->wby, &g->wC, &g->wdiag, &g->lf32, &g->invD32, &g->zz32};
    for (auto q : d32) { *q = (float *)p; p += al(N * 4); }
    if (wt) {
        for (auto q : {&g->lfT, &g->invDT, &g->zzT}) { *q = (double *)p; p += al(N * 8); }
        for (auto q : {&g->lf32T, &g->invD32T, &g->zz32T}) { *q = (float *)p; p += al(N * 4); }
    }
    *out = g;
    return SW_OK;
}

extern "C" sw_status sw_grid_destroy(sw_grid g)
{
    if (!g) return fail(SW_ERR_INVALID_ARG, "sw_grid_destroy: NULL grid");
    cudaFree(g->cmem);
    if (g->split_mem) cudaFree(g->split_mem);
    cudaFree(g->blk);
    cudaFree(g->desc);
    cudaFreeHost(g->h_desc);
    if (g->ws_owned && g->ws) cudaFree(g->ws);
    cudaFreeHost(g->h_ctl);
    cudaFreeHost(g->h_mdev);
    cudaFreeHost(g->h_ring);
    for (int q = 0; q < RING; ++q) cudaEventDestroy(g->ring_ev[q]);
    if (g->lgraph) cudaGraphExecDestroy(g->lgraph);
    if (g->lcap) cudaStreamDestroy(g->lcap);
    delete g;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct WsLayout {
    size_t r, qa, qb, e, qa32, qb32, e32, qa_s, qb_s, e_s, Le, p, Lp, part, total;
};

static WsLayout ws_layout(const sw_grid_s *g, int prec, int k)
{
    WsLayout L{};
    size_t N = g->N, ny = g->ny, off = 0;
    bool mixed = prec != SW_PREC_FP64;
    size_t v = mixed ? 4 : 8, q = mixed ? 2 : 8;
    auto take = [&](size_t b) { size_t o = off; off += al(b); return o; };
    L.r = take(N * v);
    L.qa = take(N * q); L.qb = take(N * q); L.e = take(N * q);
    if (mixed) {
        L.qa32 = take(N * 4); L.qb32 = take(N * 4); L.e32 = take(N * 4);
        L.qa_s = take(ny * 4); L.qb_s = take(ny * 4); L.e_s = take(ny * 4);
    }
    L.Le = take(N * v);
    L.p = take(N * v * (k + 1));
    L.Lp = take(N * v * (k + 1));
    L.part = take(2 * ny * NSLOT * 8);
    L.total = off;
    return L;
}

static sw_status check_opts(const sw_solve_opts *o, bool solve)
{
    if (!o) return fail(SW_ERR_INVALID_ARG, "options are NULL");
    if (o->k < 1 || o->k > KMAX) return fail(SW_ERR_INVALID_ARG, "k must be 1..8");
    if (o->pc < 0 || o->pc > 4) return fail(SW_ERR_INVALID_ARG, "pc must be 0..4");
    if (o->pc == SW_PC_LEARNED) {
        if (!solve) return fail(SW_ERR_INVALID_ARG, "the learned preconditioner is applied by sw_model_apply");
        if (!o->model) return fail(SW_ERR_INVALID_ARG, "SW_PC_LEARNED needs opts.model");
        if (!(o->fb_ratio >= 0.0) || !std::isfinite(o->fb_ratio)) return fail(SW_ERR_INVALID_ARG, "fb_ratio must be >= 0");
    }
    if (o->pc >= 2 && (o->n_richardson < 1 || o->n_richardson > 16))
        return fail(SW_ERR_INVALID_ARG, "n_richardson must be 1..16");
    if (o->prec < 0 || o->prec > 2) return fail(SW_ERR_INVALID_ARG, "prec must be FP64, MIXED_FP16 or MIXED_BF16");
    if (solve) {
        if (o->max_iters < 1) return fail(SW_ERR_INVALID_ARG, "max_iters must be >= 1");
        if (!(o->tol >= 0.0) || !std::isfinite(o->tol)) return fail(SW_ERR_INVALID_ARG, "tol must be finite and >= 0");
        if (o->ru_every < 0) return fail(SW_ERR_INVALID_ARG, "ru_every must be >= 0");
    }
    if (o->pc == 2 && !(std::isfinite(o->omega))) return fail(SW_ERR_INVALID_ARG, "omega must be finite");
    if (o->threads_per_row < 0 || o->threads_per_row > MAX_THREADS || (o->threads_per_row & 31))
        return fail(SW_ERR_INVALID_ARG, "threads_per_row must be 0 or a multiple of 32 up to 256");
    if (!std::isfinite(o->eta)) return fail(SW_ERR_INVALID_ARG, "eta must be finite");
    if (o->row_mode < 0 || o->row_mode > 2) return fail(SW_ERR_INVALID_ARG, "row_mode must be 0, 1 or 2");
    if (o->split_r0 < 0 || o->split_r0 > 1) return fail(SW_ERR_INVALID_ARG, "split_r0 must be 0 or 1");
    return SW_OK;
}

extern "C" sw_status sw_grid_workspace_bytes(sw_grid g, const sw_solve_opts *o, size_t *bytes)
{
    if (!g || !bytes) return fail(SW_ERR_INVALID_ARG, "sw_grid_workspace_bytes: NULL argument");
    sw_solve_opts d;
    if (!o) { sw_solve_opts_default(&d); o = &d; }
    sw_status st = check_opts(o, false);
    if (st) return st;
    *bytes = ws_layout(g, o->prec, o->k).total;
    return SW_OK;
}

extern "C" sw_status sw_grid_attach_workspace(sw_grid g, void *dev_ptr, size_t bytes)
{
    if (!g) return fail(SW_ERR_INVALID_ARG, "sw_grid_attach_workspace: NULL grid");
    if (dev_ptr && ((uintptr_t)dev_ptr & 255)) return fail(SW_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (g->ws_owned && g->ws) cudaFree(g->ws);
    g->ws = dev_ptr;
    g->ws_bytes = dev_ptr ? bytes : 0;
    g->ws_owned = false;
    return SW_OK;
}

static sw_status ensure_ws(sw_grid g, int prec, int k)
{
    size_t need = ws_layout(g, prec, k).total;
    if (g->ws && g->ws_bytes >= need) return SW_OK;
    if (g->ws && !g->ws_owned)
        return fail(SW_ERR_INVALID_ARG, "attached workspace is smaller than sw_grid_workspace_bytes");
    if (g->ws) { cudaFree(g->ws); g->ws = nullptr; g->ws_bytes = 0; }
    CK(cudaMalloc(&g->ws, need));
    g->ws_bytes = need;
    g->ws_owned = true;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// coefficients
// ---------------------------------------------------------------------------
static FactorArgs factor_args(const sw_grid_s *g)
{
    FactorArgs f;
    f.nx = g->nx; f.ny = g->ny; f.eta_explicit = g->eta_explicit;
    f.ax = g->ax; f.C = g->C; f.rowmax = g->rowmax;
    f.lf = g->lf; f.invD = g->invD; f.zz = g->zz; f.gam = g->gam; f.ec = g->ec; f.eta_out = g->eta;
    f.lf32 = g->lf32; f.invD32 = g->invD32; f.zz32 = g->zz32; f.gam32 = g->gam32; f.ec32 = g->ec32;
    f.lfT = g->lfT; f.invDT = g->invDT; f.zzT = g->zzT;
    f.lf32T = g->lf32T; f.invD32T = g->invD32T; f.zz32T = g->zz32T;
    return f;
}

// new coefficients or eta: the FP32 zonal factors (mixed solvers) now; the
// FP64 ones when an FP64 solve or preconditioner needs them (ensure_f64)
static sw_status refactor(sw_grid g, cudaStream_t s)
{
    CK(launch_factor(factor_args(g), false, row_threads(g->nx), s));
    g->f64_valid = false;
    return SW_OK;
}

// the FP64 zonal factors, stream-ordered before the FP64 work that follows on
// s.  Inside a CUDA graph capture they are always recorded: a replay cannot
// know whether the coefficients changed since.
static sw_status ensure_f64(sw_grid g, cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap));
    const bool recorded = (cap != cudaStreamCaptureStatusNone);
    if (g->f64_valid && !recorded) return SW_OK;
    CK(launch_factor(factor_args(g), true, row_threads(g->nx), s));
    if (!recorded) g->f64_valid = true;
    return SW_OK;
}

extern "C" sw_status sw_elliptic_set_coeffs(sw_grid g, const double *A11, const double *A12, const double *A21,
                                            const double *A22, const double *B1, const double *B2, const double *C,
                                            void *stream)
{
    if (!g) return fail(SW_ERR_INVALID_ARG, "sw_elliptic_set_coeffs: NULL grid");
    if (!A11 || !A12 || !A21 || !A22 || !B1 || !B2 || !C)
        return fail(SW_ERR_INVALID_ARG, "sw_elliptic_set_coeffs: NULL coefficient pointer");
    cudaStream_t s = (cudaStream_t)stream;
    FaceArgs a;
    a.nx = g->nx; a.ny = g->ny; a.dlam = g->dlam; a.dphi = g->dphi;
    a.A11 = A11; a.A12 = A12; a.A21 = A21; a.A22 = A22; a.B1 = B1; a.B2 = B2; a.C = C;
    a.ax = g->ax; a.cx = g->cx; a.bx = g->bx; a.ay = g->ay; a.cy = g->cy; a.by = g->by; a.C64 = g->C; a.diag = g->diag;
    a.wax = g->wax; a.wcx = g->wcx; a.wbx = g->wbx; a.way = g->way; a.wcy = g->wcy; a.wby = g->wby; a.wC = g->wC;
    a.wdiag = g->wdiag; a.rowmax = g->rowmax;
    CK(launch_faces(a, row_threads(g->nx), s));
    sw_status st = refactor(g, s);
    if (st) return st;
    g->has_coeffs = true;
    return SW_OK;
}

extern "C" sw_status sw_grid_set_eta(sw_grid g, double eta, void *stream)
{
    if (!g) return fail(SW_ERR_INVALID_ARG, "sw_grid_set_eta: NULL grid");
    if (!std::isfinite(eta)) return fail(SW_ERR_INVALID_ARG, "sw_grid_set_eta: eta must be finite");
    if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "sw_grid_set_eta: coefficients not set");
    g->eta_explicit = eta > 0.0 ? eta : 0.0;
    return refactor(g, (cudaStream_t)stream);
}

extern "C" sw_status sw_grid_get_eta(sw_grid g, double *eta)
{
    if (!g || !eta) return fail(SW_ERR_INVALID_ARG, "sw_grid_get_eta: NULL argument");
    if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "sw_grid_get_eta: coefficients not set");
    CK(cudaMemcpy(eta, g->eta, sizeof(double), cudaMemcpyDeviceToHost));
    return SW_OK;
}

// ---------------------------------------------------------------------------
// operator and preconditioner
// ---------------------------------------------------------------------------
extern "C" sw_status sw_operator_apply(sw_grid g, int prec, const void *x, void *y, void *stream)
{
    if (!g || !x || !y) return fail(SW_ERR_INVALID_ARG, "sw_operator_apply: NULL argument");
    if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "sw_operator_apply: coefficients not set");
    cudaStream_t s = (cudaStream_t)stream;
    size_t eb = prec == SW_PREC_FP32 ? 4 : 8;
    const char *xb = (const char *)x, *yb = (const char *)y;
    if (xb < yb + g->N * eb && yb < xb + g->N * eb) return fail(SW_ERR_INVALID_ARG, "sw_operator_apply: x and y overlap");
    if (prec == SW_PREC_FP64) {
        OpArgs<double> a{g->nx, g->ny, g->ax, g->cx, g->bx, g->ay, g->cy, g->by, g->C};
        CK(launch_operator_f64(a, (const double *)x, (double *)y, row_threads(g->nx), s));
    } else if (prec == SW_PREC_FP32) {
        OpArgs<float> a{g->nx, g->ny, g->wax, g->wcx, g->wbx, g->way, g->wcy, g->wby, g->wC};
        CK(launch_operator_f32(a, (const float *)x, (float *)y, row_threads(g->nx), s));
    } else {
        return fail(SW_ERR_INVALID_ARG, "sw_operator_apply: prec must be SW_PREC_FP64 or SW_PREC_FP32");
    }
    return SW_OK;
}

static int pole_band(const sw_grid_s *g, const sw_solve_opts *o)
{
    if (o->prec == SW_PREC_FP64) return 0;
    if (o->pole_band_rows >= 0) return std::min(o->pole_band_rows, g->ny / 2);
    // a band of fixed angular width: 1 / 2 / 3 rows at ny = 64 / 128 / 256
    // (Sec. 4.3), round(3 ny / 256) rows in general
    int b = (3 * g->ny + 128) / 256;
    if (b < 1) b = 1;
    return std::min(b, g->ny / 2);
}

template <class Pol>
static void fill_member(sw_grid g, const sw_solve_opts *o, const double *R, double *phi, MemberDev<Pol> &M)
{
    typedef typename Pol::coef ct;
    typedef typename Pol::fac ft;
    typedef typename Pol::vec vt;
    typedef typename Pol::res rt;
    typedef typename Pol::q16 qt;
    std::memset(&M, 0, sizeof(M));
    WsLayout L = ws_layout(g, o->prec, o->k);
    char *w = (char *)g->ws;
    M.nx = g->nx; M.ny = g->ny; M.k = o->k; M.pc = o->pc;
    M.nstages = o->pc >= 2 ? o->n_richardson : 1;     // the learned option falls back to option 3
    M.fb_ratio = o->fb_ratio;
    M.min_iters = o->min_iters; M.max_iters = o->max_iters; M.ru_every = o->ru_every;
    M.band = pole_band(g, o);
    M.tol = o->tol; M.omega = o->omega; M.etap = g->eta;
    M.ax = g->ax; M.cx = g->cx; M.bx = g->bx; M.ay = g->ay; M.cy = g->cy; M.by = g->by; M.C = g->C;
    if constexpr (Pol::kMixed) {
        M.wax = (const ct *)g->wax; M.wcx = (const ct *)g->wcx; M.wbx = (const ct *)g->wbx;
        M.way = (const ct *)g->way; M.wcy = (const ct *)g->wcy; M.wby = (const ct *)g->wby;
        M.wC = (const ct *)g->wC; M.wdiag = (const ct *)g->wdiag;
        M.lf = (const ft *)g->lf32; M.invD = (const ft *)g->invD32; M.zz = (const ft *)g->zz32;
        M.lfT = (const ft *)g->lf32T; M.invDT = (const ft *)g->invD32T; M.zzT = (const ft *)g->zz32T;
    } else {
        M.wax = (const ct *)g->ax; M.wcx = (const ct *)g->cx; M.wbx = (const ct *)g->bx;
        M.way = (const ct *)g->ay; M.wcy = (const ct *)g->cy; M.wby = (const ct *)g->by;
        M.wC = (const ct *)g->C; M.wdiag = (const ct *)g->diag;
        M.lf = (const ft *)g->lf; M.invD = (const ft *)g->invD; M.zz = (const ft *)g->zz;
        M.lfT = (const ft *)g->lfT; M.invDT = (const ft *)g->invDT; M.zzT = (const ft *)g->zzT;
    }
    if constexpr (Pol::kMixed) { M.gam = g->gam32; M.ec = g->ec32; }
    else { M.gam = g->gam; M.ec = g->ec; }
    M.R = R; M.phi = phi;
    M.r = (rt *)(w + L.r);
    M.qa = (qt *)(w + L.qa); M.qb = (qt *)(w + L.qb); M.e = (qt *)(w + L.e);
    if constexpr (Pol::kMixed) {
        M.qa32 = (float *)(w + L.qa32); M.qb32 = (float *)(w + L.qb32); M.e32 = (float *)(w + L.e32);
        M.qa_s = (float *)(w + L.qa_s); M.qb_s = (float *)(w + L.qb_s); M.e_s = (float *)(w + L.e_s);
    }
    M.Le = (vt *)(w + L.Le); M.p = (vt *)(w + L.p); M.Lp = (vt *)(w + L.Lp);
    M.part = (double *)(w + L.part);
    M.hist = o->res_history;
    M.rowres = o->row_residual;
    M.split = (Pol::kMixed && o->split_r0) ? 1 : 0;
    M.shat = g->shat; M.sdx = g->sdx; M.scx = g->scx; M.sdy = g->sdy; M.scy = g->scy;
}

// the split initial residual needs a mixed precision, a refresh of this grid
// and rows of a multiple of 8 points
static sw_status check_split(const sw_grid_s *g, const sw_solve_opts *o)
{
    if (!o->split_r0) return SW_OK;
    if (o->prec == SW_PREC_FP64) return fail(SW_ERR_INVALID_ARG, "split_r0 is for the mixed precisions");
    if (!g->split_valid) return fail(SW_ERR_INVALID_ARG, "split_r0: call sw_split_refresh on the grid first");
    if (g->nx % 8) return fail(SW_ERR_INVALID_ARG, "split_r0: nx must be a multiple of 8");
    return SW_OK;
}

static sw_status upload_member(sw_grid g, const sw_solve_opts *o, const double *R, double *phi, cudaStream_t s,
                               void *Mdev_out_host)
{
    if (o->prec == SW_PREC_FP64) {
        sw_status st = ensure_f64(g, s);
        if (st) return st;
        MemberDev<PolFP64> M;
        fill_member<PolFP64>(g, o, R, phi, M);
        std::memcpy(Mdev_out_host, &M, sizeof(M));
    } else if (o->prec == SW_PREC_MIXED_FP16) {
        MemberDev<PolF16> M;
        fill_member<PolF16>(g, o, R, phi, M);
        std::memcpy(Mdev_out_host, &M, sizeof(M));
    } else {
        MemberDev<PolBF16> M;
        fill_member<PolBF16>(g, o, R, phi, M);
        std::memcpy(Mdev_out_host, &M, sizeof(M));
    }
    CK(cudaMemcpyAsync(g->blk->dev, Mdev_out_host, member_dev_bytes(o->prec), cudaMemcpyHostToDevice, s));
    return SW_OK;
}

extern "C" sw_status sw_precond_apply(sw_grid g, const sw_solve_opts *o, const void *r, void *q, void *stream)
{
    if (!g || !r || !q) return fail(SW_ERR_INVALID_ARG, "sw_precond_apply: NULL argument");
    if (o && o->pc == SW_PC_LEARNED) return fail(SW_ERR_INVALID_ARG, "sw_precond_apply: use sw_model_apply for SW_PC_LEARNED");
    if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "sw_precond_apply: coefficients not set");
    sw_status st = check_opts(o, false);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    size_t eb = o->prec == SW_PREC_FP64 ? 8 : 4;
    const char *rb = (const char *)r, *qb = (const char *)q;
    if (rb < qb + g->N * eb && qb < rb + g->N * eb) return fail(SW_ERR_INVALID_ARG, "sw_precond_apply: r and q overlap");
    if (o->eta > 0.0 && o->eta != g->eta_explicit) {
        g->eta_explicit = o->eta;
        if ((st = refactor(g, s))) return st;
    }
    if ((st = ensure_ws(g, o->prec, o->k))) return st;
    alignas(16) unsigned char hbuf[sizeof(SolverBlock::dev)];
    int nst = o->pc >= 2 ? o->n_richardson : 1;
    if (o->prec == SW_PREC_FP64) {
        if ((st = ensure_f64(g, s))) return st;
        MemberDev<PolFP64> M;
        fill_member<PolFP64>(g, o, nullptr, nullptr, M);
        M.r = (double *)r;                    // the stages read r from the member's r
        M.e = (double *)q;                    // FP64: the last stage writes q directly
        std::memcpy(hbuf, &M, sizeof(M));
    } else if (o->prec == SW_PREC_MIXED_FP16) {
        MemberDev<PolF16> M;
        fill_member<PolF16>(g, o, nullptr, nullptr, M);
        M.r = (float *)r;
        std::memcpy(hbuf, &M, sizeof(M));
    } else {
        MemberDev<PolBF16> M;
        fill_member<PolBF16>(g, o, nullptr, nullptr, M);
        M.r = (float *)r;
        std::memcpy(hbuf, &M, sizeof(M));
    }
    CK(cudaMemcpyAsync(g->blk->dev, hbuf, member_dev_bytes(o->prec), cudaMemcpyHostToDevice, s));
    CK(launch_precond(o->prec, g->blk->dev, g->nx, g->ny, nst, o->prec == SW_PREC_FP64 ? nullptr : q,
                      row_threads(g->nx, o->threads_per_row), s));
    // the host staging buffer must outlive the asynchronous copy
    CK(cudaStreamSynchronize(s));
    return SW_OK;
}

// ---------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------
// Launch shape of one persistent launch: every member owns a group of blocks
// and every block one latitude row when the co-resident blocks suffice, so
// the row's constant data and owner-only vectors stay in shared memory;
// otherwise the co-resident blocks are shared out in proportion to each
// member's expected work (points times nx: the iteration count grows about
// linearly with the resolution) and cycle over several rows each, with
// everything in global memory.
struct Plan {
    int grid = 0, cc = 0, cs = 0, threads = 0, minb = 1, warp = 0, stage = 0;
    size_t smem = 0;
    std::vector<int> nb;
};

static sw_status plan_launch(int n, const sw_grid *grids, const sw_solve_opts *o, int max_nx, Plan &P)
{
    const int sms = grids[0]->sms;
    P.threads = row_threads(max_nx, o->threads_per_row);
    P.nb.assign(n, 1);
    const int levels[3][2] = {{1, 1}, {1, 0}, {0, 0}};
    long rows_total = 0;
    for (int m = 0; m < n; ++m) rows_total += grids[m]->ny;
    // the learned preconditioner ends a launch before every application of
    // the network, so the owner-only vectors cannot live in shared memory
    bool warp_possible = o->pc != SW_PC_LEARNED;
    for (int m = 0; m < n; ++m) warp_possible = warp_possible && grids[m]->lfT;
    if (o->row_mode == 2 && !warp_possible)
        return fail(SW_ERR_INVALID_ARG, "row_mode 2 (one warp per row) needs grids with nx a power of two >= 128 "
                                        "and a preconditioner other than the learned one");
    for (int lv = (o->pc == SW_PC_LEARNED ? 1 : 0); lv < 3 && !P.grid && o->row_mode != 2; ++lv) {
        const size_t sm_l = gcr_smem_bytes(o->prec, max_nx, o->k, levels[lv][0], levels[lv][1]);
        int bps = 0;
        CK(gcr_occupancy(o->prec, o->k, 1, 0, P.threads, sm_l, &bps));
        if (bps > 0 && rows_total <= (long)bps * sms) {
            for (int m = 0; m < n; ++m) P.nb[m] = grids[m]->ny;
            P.grid = (int)rows_total; P.cc = levels[lv][0]; P.cs = levels[lv][1]; P.smem = sm_l;
        }
    }
    // the automatic choice takes one warp per row for the mixed precisions;
    // the FP64 solver, bound by FP64 instruction issue, measured no faster
    // with it (582 against 572 us per iteration at 2048 x 1024)
    const bool warp_auto = o->prec != SW_PREC_FP64;
    if (!P.grid && warp_possible && (o->row_mode == 2 || (o->row_mode == 0 && warp_auto))) {
        // more rows than resident blocks, rows of a power of two of at least
        // 128 points: one warp per row (every SM works on as many rows at once
        // as it holds warps), on every SM
        P.threads = MAX_THREADS;
        P.cc = P.cs = 0;
        // the rows' zonal factors staged in shared memory where they fit
        int bps = 0, bps2 = 0;
        P.stage = 1;
        P.smem = gcr_warp_smem_bytes(o->prec, max_nx, P.threads, 1);
        CK(gcr_occupancy(o->prec, o->k, 1, 1, P.threads, P.smem, &bps));
        if (bps < 1) {
            P.stage = 0;
            P.smem = gcr_warp_smem_bytes(o->prec, max_nx, P.threads, 0);
            CK(gcr_occupancy(o->prec, o->k, 1, 1, P.threads, P.smem, &bps));
        }
        CK(gcr_occupancy(o->prec, o->k, 2, 1, P.threads, P.smem, &bps2));
        const int warps = P.threads / 32;
        long need = 0;                                          // blocks that give every row its own warp
        for (int m = 0; m < n; ++m) need += (grids[m]->ny + warps - 1) / warps;
        // the register budget of one block per SM unless that leaves rows
        // without a warp and two blocks fit
        P.minb = 1;
        if ((long)bps * sms < need && bps2 > bps) { bps = bps2; P.minb = 2; }
        if (bps >= 1 && n <= bps * sms) {
            if (n == 1) {
                // the same number of blocks on every SM, as few as give every
                // row a warp, and no more blocks than rows (the block partial
                // sums are kept per row slot)
                const int per_sm = std::min(bps, std::max(1, (int)((need + sms - 1) / sms)));
                P.grid = std::min(per_sm * sms, grids[0]->ny);
                P.nb[0] = P.grid;
            } else {
                // members share the resident blocks in proportion to their work
                // (rows per warp x row length x iterations, which grow with nx),
                // each at most the blocks that give all of its rows a warp
                const int cap = bps * sms;
                int used = n;
                while (used < cap) {
                    int best = -1;
                    double bw = 0.0;
                    for (int m = 0; m < n; ++m) {
                        const int mcap = std::min(grids[m]->ny, (grids[m]->ny + warps - 1) / warps);
                        if (P.nb[m] >= mcap) continue;
                        const double wgt = (double)grids[m]->ny * grids[m]->nx * grids[m]->nx / P.nb[m];
                        if (wgt > bw) { bw = wgt; best = m; }
                    }
                    if (best < 0) break;
                    ++P.nb[best];
                    ++used;
                }
                P.grid = used;
            }
            P.warp = 1;
            // every member with rows of 1024 or 2048 points (and GCR k <= 4,
            // mixed precision, one block per SM): the kernel specialised for
            // that row length, with one zonal-solve variant compiled in
            const int m0 = grids[0]->nx / 32;
            bool one_len = P.minb == 1 && o->k <= 4 && o->prec != SW_PREC_FP64 && (m0 == 32 || m0 == 64);
            for (int m = 1; m < n && one_len; ++m) one_len = grids[m]->nx == grids[0]->nx;
            if (one_len) {
                int bs = 0;
                CK(gcr_occupancy(o->prec, o->k, 1, m0, P.threads, P.smem, &bs));
                if (bs >= bps) P.warp = m0;
            }
        } else if (o->row_mode == 2) {
            return fail(SW_ERR_INVALID_ARG, "row_mode 2: the warp-per-row kernel does not fit this device");
        } else {
            P.threads = row_threads(max_nx, o->threads_per_row);
            P.minb = 1;
        }
    }
    if (!P.grid) {
        // blocks own several rows: take the register budget that fits more
        // resident blocks
        P.smem = gcr_smem_bytes(o->prec, max_nx, o->k, 0, 0);
        P.cc = P.cs = 0;
        int bps = 0, bps2 = 0;
        CK(gcr_occupancy(o->prec, o->k, 1, 0, P.threads, P.smem, &bps));
        CK(gcr_occupancy(o->prec, o->k, 2, 0, P.threads, P.smem, &bps2));
        if (bps2 > bps) { bps = bps2; P.minb = 2; }
        if (bps < 1) return fail(SW_ERR_INVALID_ARG, "grid rows too long for the solver kernel");
        const int cap = bps * sms;
        if (n > cap) return fail(SW_ERR_INVALID_ARG, "too many members for one launch on this device");
        int used = n;
        while (used < cap) {
            int best = -1;
            double bw = 0.0;
            for (int m = 0; m < n; ++m) {
                if (P.nb[m] >= grids[m]->ny) continue;
                const double wgt = (double)grids[m]->ny * grids[m]->nx * grids[m]->nx / P.nb[m];
                if (wgt > bw) { bw = wgt; best = m; }
            }
            if (best < 0) break;
            ++P.nb[best];
            ++used;
        }
        P.grid = used;
    }
    return SW_OK;
}

static void fill_desc(EnsDesc &D, int n, const sw_grid *grids, const Plan &P, sw_solve_stats *stats = nullptr)
{
    D.n = n;
    D.stats = stats;
    D.grid = P.grid;
    D.cache_const = P.cc;
    D.cache_state = P.cs;
    D.warp_rows = P.warp != 0;
    D.warp_stage = P.stage;
    D.cta_begin[0] = 0;
    for (int m = 0; m < n; ++m) {
        D.cta_begin[m + 1] = D.cta_begin[m] + P.nb[m];
        D.blk[m] = grids[m]->blk;
    }
}

static sw_status check_members(int n, const sw_grid *grids, const sw_solve_opts *o, const double *const *R,
                               double *const *phi, int &max_nx)
{
    if (n < 1 || n > MAX_MEMBERS) return fail(SW_ERR_INVALID_ARG, "number of members must be 1..480");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    max_nx = 0;
    for (int m = 0; m < n; ++m) {
        sw_grid g = grids[m];
        if (!g) return fail(SW_ERR_INVALID_ARG, "NULL grid in the member list");
        if (!R[m] || !phi[m]) return fail(SW_ERR_INVALID_ARG, "NULL R or phi");
        if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "coefficients not set for a member grid");
        if (g->device != dev) return fail(SW_ERR_INVALID_ARG, "member grid belongs to another device");
        for (int q = 0; q < m; ++q)
            if (grids[q] == g) return fail(SW_ERR_INVALID_ARG, "the member grids must be distinct");
        if (n > 1 && (o->res_history || o->row_residual))
            return fail(SW_ERR_INVALID_ARG, "res_history / row_residual are for single solves");
        if (sw_status sst = check_split(g, o)) return sst;
        max_nx = std::max(max_nx, g->nx);
    }
    return SW_OK;
}

// one member: its descriptor and the launch descriptor go to the device as
// kernel parameters of k_init_one (no host staging, no copies; a graph capture
// records them by value)
static sw_status solve_one_async(sw_grid g, const sw_solve_opts *o, const double *R, double *phi,
                                 sw_solve_stats *stats_dev, int max_nx, cudaStream_t s)
{
    sw_status st;
    if (o->eta > 0.0 && o->eta != g->eta_explicit) {
        g->eta_explicit = o->eta;
        if ((st = refactor(g, s))) return st;
    }
    if ((st = ensure_ws(g, o->prec, o->k))) return st;
    if (o->prec == SW_PREC_FP64 && (st = ensure_f64(g, s))) return st;
    InitOneArgs a;
    std::memset(&a, 0, sizeof(a));
    if (o->prec == SW_PREC_FP64) {
        MemberDev<PolFP64> M;
        fill_member<PolFP64>(g, o, R, phi, M);
        std::memcpy(a.mdev, &M, sizeof(M));
    } else if (o->prec == SW_PREC_MIXED_FP16) {
        MemberDev<PolF16> M;
        fill_member<PolF16>(g, o, R, phi, M);
        std::memcpy(a.mdev, &M, sizeof(M));
    } else {
        MemberDev<PolBF16> M;
        fill_member<PolBF16>(g, o, R, phi, M);
        std::memcpy(a.mdev, &M, sizeof(M));
    }
    if (o->res_history) CK(launch_fill(o->res_history, (size_t)o->max_iters + 1, NAN, s));
    Plan P;
    if ((st = plan_launch(1, &g, o, max_nx, P))) return st;
    a.blk = g->blk;
    a.desc = g->desc;
    a.stats = stats_dev;
    a.grid = P.grid;
    a.nb0 = P.nb[0];
    a.cache_const = P.cc;
    a.cache_state = P.cs;
    a.warp_rows = P.warp != 0;
    a.warp_stage = P.stage;
    CK(launch_init_one(a, s));
    CK(launch_gcr(o->prec, o->k, P.minb, P.warp, g->desc, P.grid, max_nx, P.threads, P.smem, s));
    return SW_OK;
}

static sw_status finish_members(int n, const sw_grid *grids, sw_solve_stats *stats, cudaStream_t s,
                                bool learned = false);
static sw_status build_learned_loop(sw_grid g, const sw_solve_opts *o, const Plan &P, int max_nx, const void *r,
                                    float *ef, cudaStream_t s, cudaGraphExec_t *out);

static sw_status solve_members(int n, const sw_grid *grids, const sw_solve_opts *o, const double *const *R,
                               double *const *phi, sw_solve_stats *stats, cudaStream_t s)
{
    sw_status st = check_opts(o, true);
    if (st) return st;
    if (n < 1 || n > MAX_MEMBERS) return fail(SW_ERR_INVALID_ARG, "number of members must be 1..480");
    if (o->pc == SW_PC_LEARNED) {
        if (n != 1) return fail(SW_ERR_INVALID_ARG, "SW_PC_LEARNED solves one grid per call");
        if ((st = model_check_grid(grids[0]))) return st;
    }
    int dev = -1;
    CK(cudaGetDevice(&dev));
    int max_nx = 0;
    for (int m = 0; m < n; ++m) {
        sw_grid g = grids[m];
        if (!g) return fail(SW_ERR_INVALID_ARG, "NULL grid in the member list");
        if (!R[m] || !phi[m]) return fail(SW_ERR_INVALID_ARG, "NULL R or phi");
        if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "coefficients not set for a member grid");
        if (g->device != dev) return fail(SW_ERR_INVALID_ARG, "member grid belongs to another device");
        for (int q = 0; q < m; ++q)
            if (grids[q] == g) return fail(SW_ERR_INVALID_ARG, "the member grids must be distinct");
        if (n > 1 && (o->res_history || o->row_residual))
            return fail(SW_ERR_INVALID_ARG, "res_history / row_residual are for single solves");
        if (sw_status sst = check_split(g, o)) return sst;
        max_nx = std::max(max_nx, g->nx);
    }
    if (n == 1 && o->pc != SW_PC_LEARNED) {
        // one member: descriptors as kernel parameters, stats read back below
        if ((st = solve_one_async(grids[0], o, R[0], phi[0], nullptr, max_nx, s))) return st;
        return finish_members(n, grids, stats, s);
    }
    static thread_local std::vector<unsigned char> staging;
    staging.resize((size_t)n * sizeof(SolverBlock::dev));
    for (int m = 0; m < n; ++m) {
        sw_grid g = grids[m];
        if (o->eta > 0.0 && o->eta != g->eta_explicit) {
            g->eta_explicit = o->eta;
            if ((st = refactor(g, s))) return st;
        }
        if ((st = ensure_ws(g, o->prec, o->k))) return st;
        if ((st = upload_member(g, o, R[m], phi[m], s, staging.data() + (size_t)m * sizeof(SolverBlock::dev)))) return st;
        MemberCtl c;
        std::memset(&c, 0, sizeof(c));
        c.phase = PH_TRUE;
        c.init = 1;
        c.nu = -1;
        *g->h_ctl = c;
        CK(cudaMemcpyAsync(&g->blk->ctl, g->h_ctl, sizeof(MemberCtl), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(&g->blk->g, 0, sizeof(GlobalCtl), s));
    }
    if (o->res_history) CK(launch_fill(o->res_history, (size_t)o->max_iters + 1, NAN, s));

    Plan P;
    if ((st = plan_launch(n, grids, o, max_nx, P))) return st;
    const int threads = P.threads, grid = P.grid, cc = P.cc, cs = P.cs;
    const size_t smem = P.smem;
    const std::vector<int> &nb = P.nb;
    (void)cc; (void)cs; (void)nb;
    sw_grid lead = grids[0];
    EnsDesc &D = *lead->h_desc;
    fill_desc(D, n, grids, P);
    CK(cudaMemcpyAsync(lead->desc, &D, sizeof(EnsDesc), cudaMemcpyHostToDevice, s));
    CK(launch_gcr(o->prec, o->k, P.minb, P.warp, lead->desc, grid, max_nx, threads, smem, s));
    if (o->pc == SW_PC_LEARNED) {
        // flexible GCR: a launch ends where the next direction is the
        // network's; the network runs on r, its output becomes e, and the
        // solver resumes with L(e)
        sw_grid g = grids[0];
        float *ef = model_scratch(o->model, g->ny, g->nx);
        if (!ef) return fail(SW_ERR_OOM, "learned preconditioner: buffers");
        const void *r = (const char *)g->ws + ws_layout(g, o->prec, o->k).r;
        // the turns run on the device, without a host round trip per turn:
        // a graph whose conditional node repeats [network, e, resumed
        // solve] while the member's state asks for a network turn
        const unsigned long long key[14] = {
            (unsigned long long)(uintptr_t)o->model, model_gen(o->model),
            (unsigned long long)(uintptr_t)g->ws, (unsigned long long)(uintptr_t)ef, (unsigned long long)o->prec,
            (unsigned long long)o->k, (unsigned long long)P.minb, (unsigned long long)P.warp,
            (unsigned long long)grid, (unsigned long long)threads, (unsigned long long)smem,
            (unsigned long long)max_nx, (unsigned long long)o->max_iters,
            (unsigned long long)row_threads(g->nx, o->threads_per_row)};
        if (std::memcmp(key, g->lkey, sizeof(key)) != 0) {
            // (built once per configuration; one that cannot be built is not tried again)
            if (g->lgraph) { cudaGraphExecDestroy(g->lgraph); g->lgraph = nullptr; }
            if (build_learned_loop(g, o, P, max_nx, r, ef, s, &g->lgraph) != SW_OK) g->lgraph = nullptr;
            std::memcpy(g->lkey, key, sizeof(key));
        }
        if (g->lgraph) {
            // (the graph's state test counts the turns in the member's block)
            CK(cudaGraphLaunch(g->lgraph, s));
            return finish_members(n, grids, stats, s, true);
        }
        // (a graph that could not be built: the same turns driven by the host)
        int turns = 0;
        for (int guard = 0; guard <= o->max_iters + 2; ++guard) {
            CK(cudaMemcpyAsync(g->h_ctl, &g->blk->ctl, sizeof(MemberCtl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (g->h_ctl->phase != PH_EXT) break;
            ++turns;
            if ((st = model_precondition(o->model, g, r, o->prec == SW_PREC_FP64, ef, s))) return st;
            CK(launch_store_e(o->prec, g->blk->dev, ef, g->nx, g->ny, row_threads(g->nx, o->threads_per_row), s));
            CK(cudaMemsetAsync(&g->blk->g, 0, sizeof(GlobalCtl), s));
            CK(launch_gcr(o->prec, o->k, P.minb, P.warp, lead->desc, grid, max_nx, threads, smem, s));
        }
        CK(cudaMemcpyAsync(&g->blk->lturns, &turns, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return finish_members(n, grids, stats, s, true);
    }
    return finish_members(n, grids, stats, s);
}

// the device-side loop of the learned preconditioner: its condition is set
// by this kernel, which lets the body run while the member's state asks for a
// network turn (at most limit turns; reset starts the count)
__global__ void k_learned_cond(cudaGraphConditionalHandle h, SolverBlock *b, int limit, int reset)
{
    if (reset) b->lturns = 0;
    const bool go = b->ctl.phase == PH_EXT && b->lturns < limit;
    if (go) b->lturns += 1;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Build the graph of the learned turns of one grid's solve: a first test of
// the member's state, then a while node whose body runs the network on r,
// stores its output as e, clears the barrier state, resumes the solver and
// tests again.  The body is captured from the stream; nothing runs here.
static sw_status build_learned_loop(sw_grid g, const sw_solve_opts *o, const Plan &P, int max_nx, const void *r,
                                    float *ef, cudaStream_t s, cudaGraphExec_t *out)
{
    *out = nullptr;
    // one application of the network outside the capture, so that the
    // launchers' one-time queries (occupancy) are made (its output, in the
    // scratch e, is overwritten by the loop's first turn)
    if (model_precondition(o->model, g, r, o->prec == SW_PREC_FP64, ef, s) != SW_OK) return SW_ERR_CUDA;
    // the body is captured on a stream of the grid's own (a capture cannot
    // run on the legacy default stream); the graph is launched on s
    if (!g->lcap && cudaStreamCreateWithFlags(&g->lcap, cudaStreamNonBlocking) != cudaSuccess) {
        g->lcap = nullptr;
        return SW_ERR_CUDA;
    }
    const cudaStream_t cs = g->lcap;
    cudaGraph_t graph = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return SW_ERR_CUDA;
    sw_status st = SW_ERR_CUDA;
    cudaGraphConditionalHandle h;
    SolverBlock *b = g->blk;
    int limit = o->max_iters + 2, reset = 1;
    cudaGraphNode_t first = nullptr, loop = nullptr;
    void *args[] = {(void *)&h, (void *)&b, (void *)&limit, (void *)&reset};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_learned_cond;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphConditionalHandleCreate(&h, graph, 0, 0) == cudaSuccess &&
        cudaGraphAddKernelNode(&first, graph, nullptr, 0, &kp) == cudaSuccess) {
        cp.conditional.handle = h;
        if (cudaGraphAddNode(&loop, graph, &first, nullptr, 1, &cp) == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                bool ok = model_precondition(o->model, g, r, o->prec == SW_PREC_FP64, ef, cs) == SW_OK;
                ok = ok && launch_store_e(o->prec, g->blk->dev, ef, g->nx, g->ny, row_threads(g->nx, o->threads_per_row),
                                          cs) == cudaSuccess;
                ok = ok && cudaMemsetAsync(&g->blk->g, 0, sizeof(GlobalCtl), cs) == cudaSuccess;
                ok = ok && launch_gcr(o->prec, o->k, P.minb, P.warp, g->desc, P.grid, max_nx, P.threads, P.smem, cs) ==
                           cudaSuccess;
                if (ok) {
                    k_learned_cond<<<1, 1, 0, cs>>>(h, b, limit, 0);
                    ok = cudaGetLastError() == cudaSuccess;
                }
                cudaGraph_t captured = nullptr;
                const bool ended = cudaStreamEndCapture(cs, &captured) == cudaSuccess;
                if (ok && ended && cudaGraphInstantiate(out, graph, 0) == cudaSuccess) st = SW_OK;
            }
        }
    }
    cudaGraphDestroy(graph);
    if (st != SW_OK) {
        *out = nullptr;
        cudaGetLastError();         // the failed capture leaves no error behind: the host loop runs instead
    }
    return st;
}

// wait for a synchronous solve and fill the host stats from each member's
// final state (learned: also the network turns the member's block counted)
static sw_status finish_members(int n, const sw_grid *grids, sw_solve_stats *stats, cudaStream_t s, bool learned)
{
    // the control words, the barrier state and the turn count lie together
    constexpr size_t ctl_bytes = offsetof(SolverBlock, lturns) + sizeof(int) - offsetof(SolverBlock, ctl);
    static_assert(offsetof(SolverBlock, g) - offsetof(SolverBlock, ctl) == sizeof(MemberCtl) &&
                      ctl_bytes <= sizeof(MemberCtl) + sizeof(GlobalCtl) + 64,
                  "the pinned control copy holds ctl, g and lturns in their device order");
    for (int m = 0; m < n; ++m) {
        sw_grid g = grids[m];
        CK(cudaMemcpyAsync(g->h_ctl, &g->blk->ctl, ctl_bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(g->h_eta, g->eta, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    sw_status first = SW_OK;
    bool any_timeout = false;
    for (int m = 0; m < n; ++m) {
        sw_grid g = grids[m];
        const MemberCtl &c = *g->h_ctl;
        const bool timeout = g->h_g->abort != 0;
        any_timeout |= timeout;
        int mst = timeout ? SW_ERR_TIMEOUT : (c.phase == PH_DONE ? c.status : SW_ERR_INTERNAL);
        if (stats) {
            sw_solve_stats &S = stats[m];
            std::memset(&S, 0, sizeof(S));
            S.iterations = c.it;
            S.fallbacks = c.fallbacks;
            S.status = mst;
            S.converged = (mst == SW_OK);
            S.r0_norm = c.r0;
            S.R_norm = c.nR;
            S.true_rel_residual = c.nR > 0 ? c.rn_true / c.nR : 0.0;
            S.recursive_rel_residual = c.nR > 0 ? std::sqrt(c.rn2_rec) / c.nR : 0.0;
            S.eta = *g->h_eta;
            S.network_turns =
                learned ? *(const int *)((const char *)g->h_ctl + offsetof(SolverBlock, lturns) - offsetof(SolverBlock, ctl))
                        : 0;
        }
        if (mst != SW_OK && first == SW_OK) first = (sw_status)mst;
    }
    if (any_timeout) return fail(SW_ERR_TIMEOUT, "a device-side barrier wait ran out");
    if (first == SW_ERR_NOT_CONVERGED) g_err = "max_iters reached before the tolerance";
    else if (first == SW_ERR_BREAKDOWN) g_err = "GCR breakdown: <L p, L p> not positive";
    else if (first == SW_ERR_NONFINITE) g_err = "non-finite residual norm";
    else if (first == SW_ERR_INTERNAL) g_err = "solver ended in an unexpected state";
    return first;
}

extern "C" sw_status sw_gcr_solve(sw_grid g, const sw_solve_opts *o, const double *R, double *phi,
                                  sw_solve_stats *stats, void *stream)
{
    if (!g || !R || !phi) return fail(SW_ERR_INVALID_ARG, "sw_gcr_solve: NULL argument");
    const double *Rs[1] = {R};
    double *Ps[1] = {phi};
    return solve_members(1, &g, o, Rs, Ps, stats, (cudaStream_t)stream);
}

extern "C" sw_status sw_ensemble_solve(int n, const sw_grid *grids, const sw_solve_opts *o, const double *const *R,
                                       double *const *phi, sw_solve_stats *stats, void *stream)
{
    if (!grids || !R || !phi) return fail(SW_ERR_INVALID_ARG, "sw_ensemble_solve: NULL argument");
    return solve_members(n, grids, o, R, phi, stats, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// the solve of one grid with its work vectors in the fixed scratch: the same
// kernel and launch shape as sw_gcr_solve, with no allocation
// ---------------------------------------------------------------------------
template <class Pol>
static void fill_member_noalloc(const sw_grid_s *g, void *scratch, const sw_solve_opts *o, const double *R,
                                double *phi, void *out)
{
    sw_grid_s view = *g;          // a copy of the handle that points at the scratch
    view.ws = scratch;
    MemberDev<Pol> M;
    fill_member<Pol>(&view, o, R, phi, M);
    std::memcpy(out, &M, sizeof(M));
}

extern "C" sw_status sw_gcr_solve_noalloc(sw_grid g, const sw_solve_opts *o, const double *R, double *phi,
                                          sw_solve_stats *stats, void *stream)
{
    if (!g || !R || !phi) return fail(SW_ERR_INVALID_ARG, "sw_gcr_solve_noalloc: NULL argument");
    sw_status st = check_opts(o, true);
    if (st) return st;
    if (o->pc == SW_PC_LEARNED)
        return fail(SW_ERR_INVALID_ARG, "sw_gcr_solve_noalloc: the learned preconditioner needs its own buffers");
    if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "sw_gcr_solve_noalloc: coefficients not set");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (g->device != dev) return fail(SW_ERR_INVALID_ARG, "sw_gcr_solve_noalloc: the grid belongs to another device");
    if ((st = check_split(g, o))) return st;
    const size_t need = ws_layout(g, o->prec, o->k).total;
    if (need > SW_NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "sw_gcr_solve_noalloc: this grid and these options need %zu bytes of scratch, more than the "
                      "fixed %u (use sw_gcr_solve)", need, (unsigned)SW_NOALLOC_SCRATCH_BYTES);
        return fail(SW_ERR_INVALID_ARG, msg);
    }
    void *scratch = nullptr;
    size_t cap = 0;
    CK(noalloc_scratch(&scratch, &cap));
    cudaStream_t s = (cudaStream_t)stream;
    if (o->eta > 0.0 && o->eta != g->eta_explicit) {
        g->eta_explicit = o->eta;
        if ((st = refactor(g, s))) return st;
    }
    alignas(16) unsigned char hbuf[sizeof(SolverBlock::dev)];
    if (o->prec == SW_PREC_FP64 && (st = ensure_f64(g, s))) return st;
    if (o->prec == SW_PREC_FP64) fill_member_noalloc<PolFP64>(g, scratch, o, R, phi, hbuf);
    else if (o->prec == SW_PREC_MIXED_FP16) fill_member_noalloc<PolF16>(g, scratch, o, R, phi, hbuf);
    else fill_member_noalloc<PolBF16>(g, scratch, o, R, phi, hbuf);
    CK(cudaMemcpyAsync(g->blk->dev, hbuf, member_dev_bytes(o->prec), cudaMemcpyHostToDevice, s));
    MemberCtl c;
    std::memset(&c, 0, sizeof(c));
    c.phase = PH_TRUE;
    c.init = 1;
    c.nu = -1;
    *g->h_ctl = c;
    CK(cudaMemcpyAsync(&g->blk->ctl, g->h_ctl, sizeof(MemberCtl), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(&g->blk->g, 0, sizeof(GlobalCtl), s));
    if (o->res_history) CK(launch_fill(o->res_history, (size_t)o->max_iters + 1, NAN, s));

    // the launch shape of sw_gcr_solve for this grid and these options
    Plan P;
    if ((st = plan_launch(1, &g, o, g->nx, P))) return st;
    fill_desc(*g->h_desc, 1, &g, P);
    CK(cudaMemcpyAsync(g->desc, g->h_desc, sizeof(EnsDesc), cudaMemcpyHostToDevice, s));
    CK(launch_gcr(o->prec, o->k, P.minb, P.warp, g->desc, P.grid, g->nx, P.threads, P.smem, s));
    CK(cudaMemcpyAsync(g->h_ctl, &g->blk->ctl, sizeof(MemberCtl) + sizeof(GlobalCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g->h_eta, g->eta, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    const MemberCtl &r = *g->h_ctl;
    const bool timeout = g->h_g->abort != 0;
    const int mst = timeout ? SW_ERR_TIMEOUT : (r.phase == PH_DONE ? r.status : SW_ERR_INTERNAL);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->iterations = r.it;
        stats->status = mst;
        stats->converged = (mst == SW_OK);
        stats->r0_norm = r.r0;
        stats->R_norm = r.nR;
        stats->true_rel_residual = r.nR > 0 ? r.rn_true / r.nR : 0.0;
        stats->recursive_rel_residual = r.nR > 0 ? std::sqrt(r.rn2_rec) / r.nR : 0.0;
        stats->eta = *g->h_eta;
    }
    switch (mst) {
    case SW_OK: return SW_OK;
    case SW_ERR_TIMEOUT: return fail(SW_ERR_TIMEOUT, "a device-side barrier wait ran out");
    case SW_ERR_NOT_CONVERGED: return fail(SW_ERR_NOT_CONVERGED, "max_iters reached before the tolerance");
    case SW_ERR_BREAKDOWN: return fail(SW_ERR_BREAKDOWN, "GCR breakdown: <L p, L p> not positive");
    case SW_ERR_NONFINITE: return fail(SW_ERR_NONFINITE, "non-finite residual norm");
    default: return fail(SW_ERR_INTERNAL, "solver ended in an unexpected state");
    }
}

// ---------------------------------------------------------------------------
// ensemble solve without host synchronisation
// ---------------------------------------------------------------------------
extern "C" sw_status sw_ensemble_solve_async(int n, const sw_grid *grids, const sw_solve_opts *o,
                                             const double *const *R, double *const *phi,
                                             sw_solve_stats *stats_dev, void *stream)
{
    if (!grids || !R || !phi) return fail(SW_ERR_INVALID_ARG, "sw_ensemble_solve_async: NULL argument");
    sw_status st = check_opts(o, true);
    if (st) return st;
    if (o->pc == SW_PC_LEARNED)
        return fail(SW_ERR_INVALID_ARG, "sw_ensemble_solve_async: the learned preconditioner needs the host");
    int max_nx = 0;
    if ((st = check_members(n, grids, o, R, phi, max_nx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 1) return solve_one_async(grids[0], o, R[0], phi[0], stats_dev, max_nx, s);
    // host staging: a recorded call uses each grid's dedicated slot, which a
    // graph replay reads; otherwise the next ring slot, once the copies of
    // its previous use have run
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap));
    const bool recorded = (cap != cudaStreamCaptureStatusNone);
    auto mdev_slot = [&](sw_grid g) -> void * {
        return recorded ? g->h_mdev : (void *)(g->h_ring + (size_t)g->ring_next * ring_slot_bytes());
    };
    for (int m = 0; m < n; ++m) {
        sw_grid g = grids[m];
        if (o->eta > 0.0 && o->eta != g->eta_explicit) {
            g->eta_explicit = o->eta;
            if ((st = refactor(g, s))) return st;
        }
        if ((st = ensure_ws(g, o->prec, o->k))) return st;
        if (o->prec == SW_PREC_FP64 && (st = ensure_f64(g, s))) return st;
        if (!recorded) CK(cudaEventSynchronize(g->ring_ev[g->ring_next]));
        void *hm = mdev_slot(g);
        if (o->prec == SW_PREC_FP64) {
            MemberDev<PolFP64> M;
            fill_member<PolFP64>(g, o, R[m], phi[m], M);
            std::memcpy(hm, &M, sizeof(M));
        } else if (o->prec == SW_PREC_MIXED_FP16) {
            MemberDev<PolF16> M;
            fill_member<PolF16>(g, o, R[m], phi[m], M);
            std::memcpy(hm, &M, sizeof(M));
        } else {
            MemberDev<PolBF16> M;
            fill_member<PolBF16>(g, o, R[m], phi[m], M);
            std::memcpy(hm, &M, sizeof(M));
        }
        CK(cudaMemcpyAsync(g->blk->dev, hm, member_dev_bytes(o->prec), cudaMemcpyHostToDevice, s));
    }
    if (o->res_history) CK(launch_fill(o->res_history, (size_t)o->max_iters + 1, NAN, s));
    Plan P;
    if ((st = plan_launch(n, grids, o, max_nx, P))) return st;
    sw_grid lead = grids[0];
    EnsDesc *hd = recorded ? lead->h_desc
                           : (EnsDesc *)((unsigned char *)mdev_slot(lead) +
                                         ((sizeof(SolverBlock::dev) + 255) & ~(size_t)255));
    fill_desc(*hd, n, grids, P, stats_dev);
    CK(cudaMemcpyAsync(lead->desc, hd, sizeof(EnsDesc), cudaMemcpyHostToDevice, s));
    if (!recorded) {
        for (int m = 0; m < n; ++m) {
            sw_grid g = grids[m];
            CK(cudaEventRecord(g->ring_ev[g->ring_next], s));
            g->ring_next = (g->ring_next + 1) % RING;
        }
    }
    CK(launch_init_members(lead->desc, n, s));
    CK(launch_gcr(o->prec, o->k, P.minb, P.warp, lead->desc, P.grid, max_nx, P.threads, P.smem, s));
    return SW_OK;
}

// ---------------------------------------------------------------------------
// split fluid thickness (Sec. 4.2, Eq. 14)
// ---------------------------------------------------------------------------
extern "C" sw_status sw_split_refresh(sw_grid g, const double *phi, void *stream)
{
    if (!g || !phi) return fail(SW_ERR_INVALID_ARG, "sw_split_refresh: NULL argument");
    if (g->nx % 8) return fail(SW_ERR_INVALID_ARG, "sw_split_refresh: nx must be a multiple of 8");
    if (!g->split_mem) {
        const size_t b = al(g->N * 4);
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, 5 * b);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(SW_ERR_OOM, "sw_split_refresh: device allocation failed"); }
        g->split_mem = p;
        char *c = (char *)p;
        g->shat = (float *)c; g->sdx = (float *)(c + b); g->scx = (float *)(c + 2 * b);
        g->sdy = (float *)(c + 3 * b); g->scy = (float *)(c + 4 * b);
    }
    SplitRefreshArgs a{g->nx, g->ny, phi, g->shat, g->sdx, g->scx, g->sdy, g->scy};
    CK(launch_split_refresh(a, (cudaStream_t)stream));
    g->split_valid = true;
    return SW_OK;
}

extern "C" sw_status sw_split_residual(sw_grid g, const double *phi, const double *R, float *r, void *stream)
{
    if (!g || !phi || !R || !r) return fail(SW_ERR_INVALID_ARG, "sw_split_residual: NULL argument");
    if (!g->has_coeffs) return fail(SW_ERR_INVALID_ARG, "sw_split_residual: coefficients not set");
    if (!g->split_valid) return fail(SW_ERR_INVALID_ARG, "sw_split_residual: call sw_split_refresh first");
    if (((uintptr_t)phi & 15) || ((uintptr_t)R & 15) || ((uintptr_t)r & 15))
        return fail(SW_ERR_INVALID_ARG, "sw_split_residual: phi, R and r must be 16-byte aligned");
    SplitResidualArgs a{g->nx, g->ny, phi, R, r, g->wax, g->wcx, g->wbx, g->way, g->wcy, g->wby, g->wC,
                        g->shat, g->sdx, g->scx, g->sdy, g->scy};
    CK(launch_split_residual(a, (cudaStream_t)stream));
    return SW_OK;
}

extern "C" sw_status sw_debug_barrier(int extra_arrivals, double wait_limit_s)
{
    if (extra_arrivals < 0 || !(wait_limit_s >= 0.0) || wait_limit_s > 60.0)
        return fail(SW_ERR_INVALID_ARG, "sw_debug_barrier: extra_arrivals >= 0, 0 <= wait_limit_s <= 60");
    const unsigned long long ns = wait_limit_s > 0.0 ? (unsigned long long)(wait_limit_s * 1e9) : 2000000000ull;
    CK(set_barrier_debug((unsigned long long)extra_arrivals, ns));
    return SW_OK;
}
