// sw_solver.cu -- the standalone operator and preconditioner kernels behind
// sw_operator_apply and sw_precond_apply, the member initialisation kernels,
// and the host-side launchers of the persistent GCR kernel, whose
// instantiations live in sw_gcr_*.cu.
#include "sw_gcr.cuh"
#include "sw_internal.h"

namespace sw {

// ---------------------------------------------------------------------------
// standalone kernels: one block per row
// ---------------------------------------------------------------------------
template <class T, class CT>
__global__ void __launch_bounds__(MAX_THREADS) k_operator(OpArgs<CT> a, const T *x, T *y)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    T *s3 = (T *)dsm;
    const int nx = a.nx, ny = a.ny, j = blockIdx.x;
    const size_t row = (size_t)j * nx, rs = j > 0 ? row - nx : row;
    const RowCoef<CT> c = {a.ax + row, a.cx + row, a.bx + row, a.ay + row, a.cy + row, a.by + row,
                           a.ay + rs, a.cy + rs, a.by + rs, a.C + row};
    for (int r = 0; r < 3; ++r) {
        int src, sh;
        ghost_row(j - 1 + r, nx, ny, src, sh);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            int ii = i + sh;
            if (ii >= nx) ii -= nx;
            s3[r * nx + i] = x[(size_t)src * nx + ii];
        }
    }
    __syncthreads();
    stencil_row<T, CT>(s3, s3 + nx, s3 + 2 * nx, nx, j, ny, c, true, y + row, false);
}

// Standalone operator for rows of a multiple of 8 points: a thread computes 4
// consecutive points from vector loads, all issued before the arithmetic (one
// round trip): the three rows of x with a point of halo on each side (the
// rows beyond a pole are the pole row shifted by half a circle, which keeps
// 4-point alignment when nx/2 is a multiple of 4) and the face coefficients.
// Each zonal face flux is formed once and used by both of its points (the
// same expression as in stencil_row, so the result is the same).
template <class T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 q = __ldg((const float4 *)p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = __ldg((const double2 *)p), q1 = __ldg((const double2 *)p + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

template <class T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        ((double2 *)p)[0] = make_double2(v[0], v[1]);
        ((double2 *)p)[1] = make_double2(v[2], v[3]);
    }
}

// values k = 0..5 at longitudes i0 - 1 + k of a row shifted by sh (periodic)
template <class T>
__device__ __forceinline__ void ld6(const T *rowp, int i0, int sh, int nx, T (&v)[6])
{
    int a = i0 + sh;
    if (a >= nx) a -= nx;
    T m[4];
    ld4(rowp + a, m);
    v[1] = m[0]; v[2] = m[1]; v[3] = m[2]; v[4] = m[3];
    v[0] = __ldg(rowp + (a == 0 ? nx - 1 : a - 1));
    v[5] = __ldg(rowp + (a + 4 == nx ? 0 : a + 4));
}

template <class T, class CT>
__global__ void __launch_bounds__(128) k_operator4(OpArgs<CT> a, const T *__restrict__ x, T *__restrict__ y)
{
    const int nx = a.nx, ny = a.ny, j = blockIdx.y;
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= nx) return;
    const size_t row = (size_t)j * nx, rs = j > 0 ? row - nx : row;
    const bool has_n = j < ny - 1, has_s = j > 0;
    int srcS, shS, srcN, shN;
    ghost_row(j - 1, nx, ny, srcS, shS);
    ghost_row(j + 1, nx, ny, srcN, shN);
    T xc[6], xn[6], xs[6];
    ld6(x + row, i0, 0, nx, xc);
    ld6(x + (size_t)srcN * nx, i0, shN, nx, xn);
    ld6(x + (size_t)srcS * nx, i0, shS, nx, xs);
    // zonal faces i0 - 1 .. i0 + 3 (index 0 = face i0 - 1/2)
    const int iw = i0 == 0 ? nx - 1 : i0 - 1;
    CT ax[5], cx[5], bx[5], q[4];
    ax[0] = __ldg(a.ax + row + iw); cx[0] = __ldg(a.cx + row + iw); bx[0] = __ldg(a.bx + row + iw);
    ld4(a.ax + row + i0, q); for (int k = 0; k < 4; ++k) ax[k + 1] = q[k];
    ld4(a.cx + row + i0, q); for (int k = 0; k < 4; ++k) cx[k + 1] = q[k];
    ld4(a.bx + row + i0, q); for (int k = 0; k < 4; ++k) bx[k + 1] = q[k];
    CT ay[4] = {}, cy[4] = {}, by[4] = {}, ays[4] = {}, cys[4] = {}, bys[4] = {}, cc[4];
    if (has_n) { ld4(a.ay + row + i0, ay); ld4(a.cy + row + i0, cy); ld4(a.by + row + i0, by); }
    if (has_s) { ld4(a.ay + rs + i0, ays); ld4(a.cy + rs + i0, cys); ld4(a.by + rs + i0, bys); }
    ld4(a.C + row + i0, cc);
    // zonal fluxes: face m (m = 0..4) lies between points m - 1 and m of the
    // 6-point windows (window index k = longitude i0 - 1 + k)
    T F[5];
#pragma unroll
    for (int m = 0; m < 5; ++m)
        F[m] = (T)cx[m] * (xn[m] + xn[m + 1] - xs[m] - xs[m + 1]) + (T)bx[m] * (xc[m] + xc[m + 1]) +
               (T)ax[m] * (xc[m + 1] - xc[m]);
    T out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int k = u + 1;                      // window index of the point
        T v = F[u + 1] - F[u];
        if (has_n) v += (T)ay[u] * (xn[k] - xc[k]) + (T)cy[u] * (xc[k + 1] + xn[k + 1] - xc[k - 1] - xn[k - 1]) +
                        (T)by[u] * (xc[k] + xn[k]);
        if (has_s) v -= (T)ays[u] * (xc[k] - xs[k]) + (T)cys[u] * (xs[k + 1] + xc[k + 1] - xs[k - 1] - xc[k - 1]) +
                        (T)bys[u] * (xs[k] + xc[k]);
        out[u] = v - (T)cc[u] * xc[k];
    }
    st4(y + row + i0, out);
}

// one preconditioner stage of every row (stage 0 from the residual r)
template <class Pol>
__global__ void __launch_bounds__(MAX_THREADS) k_precond(const MemberDev<Pol> *Mp, int mu)
{
    typedef typename Pol::comp comp;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ MemberDev<Pol> s_M;
    copy_in(&s_M, Mp);
    __syncthreads();
    const MemberDev<Pol> &M = s_M;
    const int j = blockIdx.x;
    RowView<Pol> v;
    view_const_global(M, j, v);
    view_state_global(M, j, v);
    const comp eta = (comp)(*M.etap);
    if (mu == 0) {
        comp *sb = (comp *)(dsm + sb_offset<Pol>(M.nx));
        for (int i = threadIdx.x; i < M.nx; i += blockDim.x) sb[pidx(i)] = stage0_input(M, v, eta, (comp)v.r[i], i);
        stage0_finish(M, v, j, dsm);
    } else {
        precond_stage<Pol>(M, v, eta, mu, j, dsm);
    }
}

// e of the member from an FP32 field (the network's direction), stored like
// the last preconditioner stage: FP64, or 16-bit with the row scale (FP32 on
// the pole-band rows)
template <class Pol>
__global__ void __launch_bounds__(MAX_THREADS) k_store_e(const MemberDev<Pol> *Mp, const float *ef)
{
    typedef typename Pol::comp comp;
    extern __shared__ __align__(16) unsigned char dsm[];
    const MemberDev<Pol> &M = *Mp;
    const int j = blockIdx.x, nx = M.nx;
    comp *sb = (comp *)(dsm + sb_offset<Pol>(nx));
    float *scratch = (float *)(dsm + red_offset<Pol>(nx));
    for (int i = threadIdx.x; i < nx; i += blockDim.x) sb[pidx(i)] = (comp)ef[(size_t)j * nx + i];
    __syncthreads();
    q_store_row(M, M.e, M.e32, M.e_s, j, sb, (comp *)nullptr, scratch);
}

// dequantise the preconditioner output e into q (mixed policies)
template <class Pol>
__global__ void k_unpack_e(const MemberDev<Pol> *Mp, float *q)
{
    const MemberDev<Pol> &M = *Mp;
    const int j = blockIdx.x;
    const float sc = q_scale(M, M.e_s, j);
    for (int i = threadIdx.x; i < M.nx; i += blockDim.x) q[(size_t)j * M.nx + i] = (float)q_load(M, M.e, M.e32, sc, j, i);
}

// ---------------------------------------------------------------------------
// split fluid thickness (Sec. 4.2, Eq. 14): refresh and standalone residual
// ---------------------------------------------------------------------------
// Phi_hat = fp32(Phi) of row j and the derivative parts of its face fluxes,
// computed in FP64 from the FP32 values and rounded to FP32 (sw_split.cuh)
__global__ void __launch_bounds__(MAX_THREADS) k_split_refresh(SplitRefreshArgs a)
{
    const int nx = a.nx, ny = a.ny, j = blockIdx.x;
    auto H = [&](int ii, int jj) -> double {
        if (jj < 0) { jj = 0; ii += nx / 2; }
        else if (jj >= ny) { jj = ny - 1; ii += nx / 2; }
        ii %= nx;
        if (ii < 0) ii += nx;
        return (double)(float)a.phi[(size_t)jj * nx + ii];
    };
    const size_t row = (size_t)j * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        a.hat[row + i] = (float)a.phi[row + i];
        a.dx[row + i] = (float)(H(i + 1, j) - H(i, j));
        a.cx[row + i] = (float)((H(i, j + 1) + H(i + 1, j + 1)) - (H(i, j - 1) + H(i + 1, j - 1)));
        a.dy[row + i] = j < ny - 1 ? (float)(H(i, j + 1) - H(i, j)) : 0.f;
        a.cy[row + i] = j < ny - 1 ? (float)((H(i + 1, j) + H(i + 1, j + 1)) - (H(i - 1, j) + H(i - 1, j + 1))) : 0.f;
    }
}

// r = L(Phi) - R with L by Eq. 14 in FP32 (the difference with R in FP64)
__global__ void __launch_bounds__(128) k_split_residual(SplitResidualArgs a)
{
    const SplitOp op = {a.nx, a.ny, a.phi, a.wax, a.wcx, a.wbx, a.way, a.wcy, a.wby, a.wC};
    const SplitState S = {a.hat, a.dx, a.cx, a.dy, a.cy};
    const int j = blockIdx.y;
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= a.nx) return;
    float L[4];
    split_quad(op, S, j, i0, L);
    const size_t at = (size_t)j * a.nx + i0;
    double Rv[4];
    ldg4(a.R + at, Rv);
    float r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = (float)((double)L[u] - Rv[u]);
    stv4(a.r + at, r);
}

cudaError_t launch_split_refresh(const SplitRefreshArgs &a, cudaStream_t s)
{
    k_split_refresh<<<a.ny, MAX_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_split_residual(const SplitResidualArgs &a, cudaStream_t s)
{
    k_split_residual<<<dim3((a.nx / 4 + 127) / 128, a.ny), 128, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_fill(double *p, size_t n, double v)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------------------------
// host-side launchers (declared in sw_internal.h)
// ---------------------------------------------------------------------------
template <class Pol>
static size_t smem_t(int max_nx, int k, int cache_const, int cache_state)
{
    return work_bytes<Pol>(max_nx) + (cache_const ? const_bytes<Pol>(max_nx) : 0) +
           (cache_state ? state_bytes<Pol>(max_nx, k) : 0);
}

template <class Pol>
static size_t warp_smem_t(int nx, int threads, bool stage)
{
    return (size_t)(threads / 32) * warp_slot_bytes<Pol>(nx, stage) + al16(RED_WORDS * sizeof(double));
}

size_t gcr_warp_smem_bytes(int prec, int nx, int threads, int stage)
{
    if (!warp_rows_ok(nx)) return 0;
    return prec == 0 ? warp_smem_t<PolFP64>(nx, threads, stage) : warp_smem_t<PolF16>(nx, threads, stage);
}

size_t gcr_smem_bytes(int prec, int max_nx, int k, int cache_const, int cache_state)
{
    switch (prec) {
    case 0: return smem_t<PolFP64>(max_nx, k, cache_const, cache_state);
    case 1: return smem_t<PolF16>(max_nx, k, cache_const, cache_state);
    default: return smem_t<PolBF16>(max_nx, k, cache_const, cache_state);
    }
}

// the instantiation of k_gcr for a precision, a GCR k, the register budget and
// the row mode (warp 0: block per row; 1: warp per row; m > 1: warp per row,
// specialised for rows of 32 m points)
static const void *gcr_kernel(int prec, int k, int minb, int warp)
{
    if (warp > 1) {
        if (k > 4 || minb != 1) return nullptr;
        return prec == 1 ? gcr_kernel_s16(warp) : (prec == 2 ? gcr_kernel_sbf16(warp) : nullptr);
    }
    switch (prec) {
    case 0: return warp ? gcr_kernel_w64(k, minb) : gcr_kernel_f64(k, minb);
    case 1: return warp ? gcr_kernel_w16(k, minb) : gcr_kernel_f16(k, minb);
    case 2: return warp ? gcr_kernel_wbf16(k, minb) : gcr_kernel_bf16(k, minb);
    default: return nullptr;
    }
}

cudaError_t raise_smem_limit(const void *f, size_t smem)
{
    struct Lim { const void *f; int dev; size_t smem; };
    static Lim lim[256];
    static int n = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int q = 0;
    while (q < n && !(lim[q].f == f && lim[q].dev == dev)) ++q;
    if (q < n && lim[q].smem >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (q < n) lim[q].smem = smem;
    else if (n < 256) lim[n++] = Lim{f, dev, smem};
    return cudaSuccess;
}

cudaError_t gcr_occupancy(int prec, int k, int minb, int warp, int threads, size_t smem, int *blocks_per_sm)
{
    const void *f = gcr_kernel(prec, k, minb, warp);
    if (!f) return cudaErrorInvalidValue;
    if (smem > 227 * 1024 - 8192) { *blocks_per_sm = 0; return cudaSuccess; }
    cudaError_t e = raise_smem_limit(f, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

cudaError_t launch_gcr(int prec, int k, int minb, int warp, const EnsDesc *Ddev, int grid, int max_nx, int threads,
                       size_t smem, cudaStream_t s)
{
    const void *f = gcr_kernel(prec, k, minb, warp);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit(f, smem);
    if (e != cudaSuccess) return e;
    const EnsDesc *d = Ddev;
    int mx = max_nx;
    void *args[] = {(void *)&d, (void *)&mx};
    return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

template <class T>
static bool op4_ok(const OpArgs<T> &a, const T *x, const T *y)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    return a.nx % 8 == 0 && a.ny <= 65535 && al(x) && al(y) && al(a.ax) && al(a.cx) && al(a.bx) && al(a.ay) &&
           al(a.cy) && al(a.by) && al(a.C);
}

cudaError_t launch_operator_f64(const OpArgs<double> &a, const double *x, double *y, int threads, cudaStream_t s)
{
    if (op4_ok(a, x, y)) {
        k_operator4<double, double><<<dim3((a.nx / 4 + 127) / 128, a.ny), 128, 0, s>>>(a, x, y);
        return cudaGetLastError();
    }
    size_t smem = 3 * (size_t)a.nx * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_operator<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_operator<double, double><<<a.ny, threads, smem, s>>>(a, x, y);
    return cudaGetLastError();
}

cudaError_t launch_operator_f32(const OpArgs<float> &a, const float *x, float *y, int threads, cudaStream_t s)
{
    if (op4_ok(a, x, y)) {
        k_operator4<float, float><<<dim3((a.nx / 4 + 127) / 128, a.ny), 128, 0, s>>>(a, x, y);
        return cudaGetLastError();
    }
    size_t smem = 3 * (size_t)a.nx * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_operator<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_operator<float, float><<<a.ny, threads, smem, s>>>(a, x, y);
    return cudaGetLastError();
}

template <class Pol>
static cudaError_t launch_precond_t(const void *Mdev, int nx, int ny, int nstages, float *qout, int threads,
                                    cudaStream_t s)
{
    const MemberDev<Pol> *M = (const MemberDev<Pol> *)Mdev;
    size_t smem = work_bytes<Pol>(nx);
    cudaError_t e = cudaFuncSetAttribute(k_precond<Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int mu = 0; mu < nstages; ++mu) k_precond<Pol><<<ny, threads, smem, s>>>(M, mu);
    if (qout) k_unpack_e<Pol><<<ny, 128, 0, s>>>(M, qout);
    return cudaGetLastError();
}

cudaError_t launch_precond(int prec, const void *Mdev, int nx, int ny, int nstages, void *qout, int threads,
                           cudaStream_t s)
{
    switch (prec) {
    case 0: return launch_precond_t<PolFP64>(Mdev, nx, ny, nstages, nullptr, threads, s);
    case 1: return launch_precond_t<PolF16>(Mdev, nx, ny, nstages, (float *)qout, threads, s);
    case 2: return launch_precond_t<PolBF16>(Mdev, nx, ny, nstages, (float *)qout, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class Pol>
static cudaError_t store_e_t(const void *Mdev, const float *ef, int nx, int ny, int threads, cudaStream_t s)
{
    const size_t smem = work_bytes<Pol>(nx);
    cudaError_t e = cudaFuncSetAttribute(k_store_e<Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_store_e<Pol><<<ny, threads, smem, s>>>((const MemberDev<Pol> *)Mdev, ef);
    return cudaGetLastError();
}

cudaError_t launch_store_e(int prec, const void *Mdev, const float *ef, int nx, int ny, int threads, cudaStream_t s)
{
    switch (prec) {
    case 0: return store_e_t<PolFP64>(Mdev, ef, nx, ny, threads, s);
    case 1: return store_e_t<PolF16>(Mdev, ef, nx, ny, threads, s);
    case 2: return store_e_t<PolBF16>(Mdev, ef, nx, ny, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_init_members(const EnsDesc *D)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= D->n) return;
    SolverBlock *B = D->blk[m];
    MemberCtl c = {};
    c.phase = PH_TRUE;
    c.init = 1;
    c.nu = -1;
    B->ctl = c;
    B->g.count = 0;
    B->g.abort = 0;
    B->g.where = 0;
}

cudaError_t launch_init_members(const EnsDesc *Ddev, int n, cudaStream_t s)
{
    k_init_members<<<(n + 127) / 128, 128, 0, s>>>(Ddev);
    return cudaGetLastError();
}

__global__ void k_init_one(const __grid_constant__ InitOneArgs a)
{
    static_assert(sizeof(SolverBlock::dev) % 4 == 0, "member descriptor copied as 32-bit words");
    constexpr int W = (int)(sizeof(SolverBlock::dev) / 4);
    const unsigned *src = reinterpret_cast<const unsigned *>(a.mdev);
    unsigned *dst = reinterpret_cast<unsigned *>(a.blk->dev);
    for (int k = threadIdx.x; k < W; k += blockDim.x) dst[k] = src[k];
    if (threadIdx.x == 0) {
        EnsDesc *D = a.desc;
        D->n = 1;
        D->grid = a.grid;
        D->cache_const = a.cache_const;
        D->cache_state = a.cache_state;
        D->warp_rows = a.warp_rows;
        D->warp_stage = a.warp_stage;
        D->stats = a.stats;
        D->cta_begin[0] = 0;
        D->cta_begin[1] = a.nb0;
        D->blk[0] = a.blk;
        MemberCtl c = {};
        c.phase = PH_TRUE;
        c.init = 1;
        c.nu = -1;
        a.blk->ctl = c;
        a.blk->g.count = 0;
        a.blk->g.abort = 0;
        a.blk->g.where = 0;
    }
}

cudaError_t launch_init_one(const InitOneArgs &a, cudaStream_t s)
{
    k_init_one<<<1, 128, 0, s>>>(a);
    return cudaGetLastError();
}


#ifdef SW_PHASE_TRACE
SW_GCR_TRACE_FN(solver)
// configure the device timeline (traced builds only): buffer of 2*cap words,
// in every translation unit that records one
extern "C" void sw_trace_configure(unsigned long long *buf, int cap, int block)
{
    gcr_trace_solver(buf, cap, block);
    gcr_trace_f64(buf, cap, block); gcr_trace_f16(buf, cap, block); gcr_trace_bf16(buf, cap, block);
    gcr_trace_w64(buf, cap, block); gcr_trace_w16(buf, cap, block); gcr_trace_wbf16(buf, cap, block);
    gcr_trace_s16(buf, cap, block); gcr_trace_sbf16(buf, cap, block);
}
#endif

// the barrier test hook of every instantiation of the GCR kernel
cudaError_t set_barrier_debug(unsigned long long extra, unsigned long long limit_ns)
{
    cudaError_t (*const set[])(unsigned long long, unsigned long long) = {
        gcr_debug_f64, gcr_debug_f16, gcr_debug_bf16, gcr_debug_w64, gcr_debug_w16, gcr_debug_wbf16,
        gcr_debug_s16, gcr_debug_sbf16};
    for (auto f : set) {
        cudaError_t e = f(extra, limit_ns);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fill(double *p, size_t n, double v, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_fill<<<blocks, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

size_t member_dev_bytes(int prec)
{
    return prec == 0 ? sizeof(MemberDev<PolFP64>) : sizeof(MemberDev<PolF16>);
}

} // namespace sw
