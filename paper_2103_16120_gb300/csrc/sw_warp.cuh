// sw_warp.cuh -- the row work of the solver with one warp per latitude row.
//
// For grids whose rows outnumber the resident thread blocks, one block per
// row leaves each SM with only one or two rows in flight, and every row phase
// is a chain of dependent memory round trips (neighbour rows, coefficients,
// zonal factors, store).  Here every warp of a block owns its own rows, so an
// SM works on as many rows at once as it holds warps, and each row's loads
// are issued as 16-byte vector loads over 4 consecutive points per lane.
//
// Layouts.  A lane works on 4 consecutive points per pass, 128 points per
// warp pass (rows of a power of two of at least 128 points).  The zonal solve
// of Eq. 13 gives each lane a chunk of m = nx/32 consecutive points: the
// warp's row buffer holds point i at (i % m) * 33 + i / m, so both the chunk
// walk of the solve and the coalesced passes are free of shared-memory bank
// conflicts, and the zonal factors are stored transposed in global memory
// (point i at (i % m) * 32 + i / m of its row) so that the chunk walk reads
// them coalesced.  The arithmetic of each point is the one of the block
// path (sw_rows.cuh, sw_solver.cu): the same expressions in the same order.
#pragma once

#include <type_traits>

#include "sw_rows.cuh"

namespace sw {

// elements of one warp's row buffer
__host__ __device__ inline int wbuf_len(int nx) { return (nx >> 5) * 33; }

struct WRow {
    int nx, m, lm;      // points per row, per lane chunk, log2 of the chunk
};

__device__ __forceinline__ WRow wrow(int nx)
{
    const int m = nx >> 5;
    return WRow{nx, m, __ffs(m) - 1};
}

// buffer position of the first of 4 consecutive points i0 .. i0 + 3 (i0 a
// multiple of 4); the others follow at strides of 33
__device__ __forceinline__ int tpos4(const WRow &w, int i0) { return (i0 & (w.m - 1)) * 33 + (i0 >> w.lm); }
__device__ __forceinline__ int tpos(const WRow &w, int i) { return (i & (w.m - 1)) * 33 + (i >> w.lm); }

// ---------------------------------------------------------------------------
// loads
// ---------------------------------------------------------------------------
// 6 consecutive values at longitudes a - 1 .. a + 4 (periodic) of a row of a
// field written by other blocks during the launch (L2-coherent loads)
__device__ __forceinline__ void cg6(const double *rowp, int a, int nx, double (&v)[6])
{
    const double2 q0 = __ldcg((const double2 *)(rowp + a)), q1 = __ldcg((const double2 *)(rowp + a) + 1);
    v[1] = q0.x; v[2] = q0.y; v[3] = q1.x; v[4] = q1.y;
    v[0] = __ldcg(rowp + (a == 0 ? nx - 1 : a - 1));
    v[5] = __ldcg(rowp + (a + 4 == nx ? 0 : a + 4));
}

__device__ __forceinline__ void cg6(const float *rowp, int a, int nx, float (&v)[6])
{
    const float4 q = __ldcg((const float4 *)(rowp + a));
    v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
    v[0] = __ldcg(rowp + (a == 0 ? nx - 1 : a - 1));
    v[5] = __ldcg(rowp + (a + 4 == nx ? 0 : a + 4));
}

// 16-bit values times the row scale (the dequantisation of stage3_q)
template <class H>
__device__ __forceinline__ void cg6h(const H *rowp, int a, int nx, float sc, float (&v)[6])
{
    const uint2 q = __ldcg((const uint2 *)(rowp + a));
    H h[4];
    memcpy(h, &q, sizeof(q));
    v[1] = q_to_f(h[0]) * sc; v[2] = q_to_f(h[1]) * sc; v[3] = q_to_f(h[2]) * sc; v[4] = q_to_f(h[3]) * sc;
    v[0] = q_to_f(__ldcg(rowp + (a == 0 ? nx - 1 : a - 1))) * sc;
    v[5] = q_to_f(__ldcg(rowp + (a + 4 == nx ? 0 : a + 4))) * sc;
}

// one source row of a preconditioner field as the stencil sees it
template <class Pol>
struct QRow {
    const typename Pol::q16 *h;     // 16-bit (or FP64) row
    const float *f;                 // FP32 row (pole band, mixed policies)
    float sc;                       // row scale of the 16-bit storage
    int sh;                         // shift of a row beyond a pole
    bool band;
};

template <class Pol>
__device__ __forceinline__ QRow<Pol> qrow(const MemberDev<Pol> &M, const typename Pol::q16 *h, const float *f32,
                                          const float *sc, int jj)
{
    int src, sh;
    ghost_row(jj, M.nx, M.ny, src, sh);
    QRow<Pol> q;
    const size_t off = (size_t)src * M.nx;
    q.h = h + off;
    q.f = Pol::kMixed ? f32 + off : nullptr;
    q.band = in_band(M, src);
    q.sc = q_scale(M, sc, src);
    q.sh = sh;
    return q;
}

template <class Pol>
__device__ __forceinline__ void q6(const QRow<Pol> &q, int i0, int nx, typename Pol::comp (&v)[6])
{
    int a = i0 + q.sh;
    if (a >= nx) a -= nx;
    if constexpr (!Pol::kMixed) cg6(q.h, a, nx, v);
    else if (q.band) cg6(q.f, a, nx, v);
    else cg6h(q.h, a, nx, q.sc, v);
}

// q6 for a row inside the grid, unshifted and outside the FP32 pole band
template <class Pol>
__device__ __forceinline__ void q6i(const QRow<Pol> &q, int i0, int nx, typename Pol::comp (&v)[6])
{
    if constexpr (!Pol::kMixed) cg6(q.h, i0, nx, v);
    else cg6h(q.h, i0, nx, q.sc, v);
}

// a row whose three source rows are all plain (q6i applies): the stencil
// passes of the generic warp kernels take a loop with these conditions fixed
// at compile time, whose loads are then free of per-row branches (the
// kernels specialised for one row length keep the single loop: their larger
// code measured slower with two)
template <class Pol>
__device__ __forceinline__ bool rows_plain(const QRow<Pol> &s, const QRow<Pol> &x, const QRow<Pol> &n, bool has_n,
                                           bool has_s)
{
    return has_n && has_s && !s.band && !x.band && !n.band && s.sh == 0 && n.sh == 0;
}

// 4 values i0 .. i0 + 3 of the row's own preconditioner output (q_load)
template <class Pol>
__device__ __forceinline__ void q4own(const QRow<Pol> &q, int i0, typename Pol::comp (&v)[4])
{
    if constexpr (!Pol::kMixed) {
        const double2 a = __ldcg((const double2 *)(q.h + i0)), b = __ldcg((const double2 *)(q.h + i0) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else if (q.band) {
        const float4 a = __ldcg((const float4 *)(q.f + i0));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const uint2 a = __ldcg((const uint2 *)(q.h + i0));
        typename Pol::q16 h[4];
        memcpy(h, &a, sizeof(a));
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = q_to_f(h[u]) * q.sc;
    }
}

// face coefficients of points i0 .. i0 + 3 (read-only during the launch)
template <class CT>
struct Coef4 {
    CT ax[5], cx[5], bx[5], ay[4], cy[4], by[4], ays[4], cys[4], bys[4], cc[4];
};

template <class CT>
__device__ __forceinline__ void ldg4(const CT *p, CT (&v)[4])
{
    if constexpr (sizeof(CT) == 4) {
        const float4 q = __ldg((const float4 *)p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = __ldg((const double2 *)p), q1 = __ldg((const double2 *)p + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

template <class CT>
__device__ __forceinline__ void coef4(const RowCoef<CT> &c, int i0, int nx, bool full, bool has_n, bool has_s,
                                      Coef4<CT> &k)
{
    const int iw = i0 == 0 ? nx - 1 : i0 - 1;
    CT q[4];
    k.cx[0] = __ldg(c.cx + iw); k.bx[0] = __ldg(c.bx + iw);
    ldg4(c.cx + i0, q); for (int u = 0; u < 4; ++u) k.cx[u + 1] = q[u];
    ldg4(c.bx + i0, q); for (int u = 0; u < 4; ++u) k.bx[u + 1] = q[u];
    if (full) {
        k.ax[0] = __ldg(c.ax + iw);
        ldg4(c.ax + i0, q); for (int u = 0; u < 4; ++u) k.ax[u + 1] = q[u];
        ldg4(c.C + i0, k.cc);
    } else {
#pragma unroll
        for (int u = 0; u < 5; ++u) k.ax[u] = CT(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) k.cc[u] = CT(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) { k.ay[u] = k.cy[u] = k.by[u] = k.ays[u] = k.cys[u] = k.bys[u] = CT(0); }
    if (has_n) { ldg4(c.ay + i0, k.ay); ldg4(c.cy + i0, k.cy); ldg4(c.by + i0, k.by); }
    if (has_s) { ldg4(c.ays + i0, k.ays); ldg4(c.cys + i0, k.cys); ldg4(c.bys + i0, k.bys); }
}

// the stencil of Eq. 10 (or P^M when the zonal a11 and C terms are zero) at
// points i0 .. i0 + 3 from 6-point windows of the rows j (xc), j + 1 (xn) and
// j - 1 (xs): the expressions of stencil_row4
template <class T, class CT>
__device__ __forceinline__ void apply4(const Coef4<CT> &k, const T (&xc)[6], const T (&xn)[6], const T (&xs)[6],
                                       bool has_n, bool has_s, T (&y)[4])
{
    T F[5];
#pragma unroll
    for (int m = 0; m < 5; ++m)
        F[m] = (T)k.cx[m] * (xn[m] + xn[m + 1] - xs[m] - xs[m + 1]) + (T)k.bx[m] * (xc[m] + xc[m + 1]) +
               (T)k.ax[m] * (xc[m + 1] - xc[m]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int q = u + 1;
        T v = F[u + 1] - F[u];
        if (has_n) v += (T)k.ay[u] * (xn[q] - xc[q]) + (T)k.cy[u] * (xc[q + 1] + xn[q + 1] - xc[q - 1] - xn[q - 1]) +
                        (T)k.by[u] * (xc[q] + xn[q]);
        if (has_s) v -= (T)k.ays[u] * (xc[q] - xs[q]) + (T)k.cys[u] * (xs[q + 1] + xc[q + 1] - xs[q - 1] - xc[q - 1]) +
                        (T)k.bys[u] * (xs[q] + xc[q]);
        y[u] = v - (T)k.cc[u] * xc[q];
    }
}

// ---------------------------------------------------------------------------
// staging of a row's zonal factors into shared memory
// ---------------------------------------------------------------------------
// The serial chunk walks of the zonal solve read the row's multipliers and
// inverse pivots several times.  One lane of the warp copies both transposed
// rows into the warp's shared memory with two bulk asynchronous copies
// (cp.async.bulk, completion counted on the warp's mbarrier) when the row's
// phase begins, so that the copy overlaps the stencil or update pass and the
// walks then read shared memory.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long wtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// longest wait for a staging copy: a copy of two rows takes microseconds
constexpr unsigned long long STAGE_WAIT_NS = 200000000ull;

template <class F>
struct WFac {
    F *lf, *iD;            // the row's transposed lf and invD in shared memory (null: read from global)
    unsigned bar;          // shared address of the warp's mbarrier
    unsigned parity;       // phase parity of the next wait
    int *abort;            // the member's abort flag, set when a wait runs out
    int pre;               // row whose lf and invD copies were started ahead (else -1)
};

// lane 0 starts the copy of one or two rows (src1 optional) into the warp's
// buffers dst0, dst1
template <class F>
__device__ __forceinline__ void wfac_copy(const WFac<F> &f, F *dst0, const F *src0, F *dst1, const F *src1, int nx)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        const unsigned bytes = (unsigned)(nx * sizeof(F));
        // the warp's earlier reads of the buffers come before the async writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(f.bar), "r"(src1 ? 2 * bytes : bytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(dst0)), "l"(src0), "r"(bytes), "r"(f.bar) : "memory");
        if (src1)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(dst1)), "l"(src1), "r"(bytes), "r"(f.bar) : "memory");
    }
}

// the multipliers and inverse pivots of row j, when its phase begins (unless
// they were started ahead, across the member barrier: wfac_ahead)
template <class F>
__device__ __forceinline__ void wfac_issue(WFac<F> &f, int j, const F *lfT, const F *iDT, int nx)
{
    if (!f.lf) return;
    if (f.pre == j) { f.pre = -1; return; }
    wfac_copy(f, f.lf, lfT, f.iD, iDT, nx);
}

// start the copies of row j's factors for the next phase now, so that they
// overlap the member barrier (the buffers are free at the end of a phase's
// rows; the factors are read-only)
template <class F>
__device__ __forceinline__ void wfac_ahead(WFac<F> &f, int j, const F *lfT, const F *iDT, int nx)
{
    if (!f.lf || f.pre >= 0) return;
    wfac_copy(f, f.lf, lfT, f.iD, iDT, nx);
    f.pre = j;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity)
{
    unsigned long long t0 = 0;
    for (unsigned n = 0;; ++n) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((n & 63) == 0) {
            const unsigned long long t = wtimer();
            if (n == 0) t0 = t;
            else if (t - t0 > STAGE_WAIT_NS) return false;
        }
    }
}

// every lane waits for the staged rows; a wait that runs out sets the abort
// flag (the solve then ends with SW_ERR_TIMEOUT) and waits once more, again
// bounded, for the copies in flight
template <class F>
__device__ __forceinline__ void wfac_wait(WFac<F> &f)
{
    if (!f.lf) return;
    if (!mbar_wait_bounded(f.bar, f.parity)) {
        if ((threadIdx.x & 31) == 0) atomicExch(f.abort, 1);
        mbar_wait_bounded(f.bar, f.parity);
    }
    f.parity ^= 1u;
}

// ---------------------------------------------------------------------------
// the cyclic zonal solve of Eq. 13 by one warp
// ---------------------------------------------------------------------------
// exclusive scan over the lanes of affine maps x -> a x + b, in lane order
// (REV: reversed lane order); on return (a, b) composes the maps of the
// earlier lanes (identity for the first)
template <class T, bool REV>
__device__ __forceinline__ void warp_affine_excl(T &a, T &b)
{
    const int lane = threadIdx.x & 31;
    T ia = a, ib = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T oa = REV ? __shfl_down_sync(0xffffffffu, ia, d) : __shfl_up_sync(0xffffffffu, ia, d);
        const T ob = REV ? __shfl_down_sync(0xffffffffu, ib, d) : __shfl_up_sync(0xffffffffu, ib, d);
        const bool ok = REV ? (lane + d < 32) : (lane >= d);
        if (ok) { ib = ia * ob + ib; ia = ia * oa; }
    }
    T ea = REV ? __shfl_down_sync(0xffffffffu, ia, 1) : __shfl_up_sync(0xffffffffu, ia, 1);
    T eb = REV ? __shfl_down_sync(0xffffffffu, ib, 1) : __shfl_up_sync(0xffffffffu, ib, 1);
    if (REV ? lane == 31 : lane == 0) { ea = T(1); eb = T(0); }
    a = ea;
    b = eb;
}

// Solve the row's cyclic system T x = b in place in the warp's buffer: the
// LDL^T factors of the non-cyclic part (multipliers lf with lf_0 = 0, inverse
// pivots invD) and the Sherman-Morrison vector zz, as in trisolve_rm, but
// transposed (point t of lane l at t * 32 + l, in shared memory when staged)
// and with each lane walking its chunk of m points serially between two warp
// scans.
template <class T, class F>
__device__ __forceinline__ float wtrisolve(T *wb, const WRow w, const F *lfT, const F *invDT, const F *__restrict__ zzT,
                                       T gam, T ec, WFac<F> &f)
{
    const int lane = threadIdx.x & 31, m = w.m;
    T *col = wb + lane;
    const F *lc = lfT + lane, *dc = invDT + lane;
    // forward elimination u_i = b_i - l_i u_{i-1}
    T a = T(1), b = T(0);
#pragma unroll 8
    for (int t = 0; t < m; ++t) {
        const T l = (T)lc[t * 32];
        b = col[t * 33] - l * b;
        a = -l * a;
    }
    SW_TRACE(221);
    warp_affine_excl<T, false>(a, b);
    T u = b;
#pragma unroll 8
    for (int t = 0; t < m; ++t) {
        const T l = (T)lc[t * 32];
        u = col[t * 33] - l * u;
        col[t * 33] = u * (T)dc[t * 32];
    }
    SW_TRACE(222);
    // staged rows: the Sherman-Morrison vector goes into the inverse pivots'
    // buffer, which the walks no longer read, while the backward walks run
    const F *zc = zzT + lane;
    if (f.lf) {
        wfac_copy(f, f.iD, zzT, (F *)nullptr, (const F *)nullptr, w.nx);
        zc = f.iD + lane;
    }
    // back substitution y_i = v_i - l_{i+1} y_{i+1}
    const T lfirst = (T)lc[0];
    const T lsh = __shfl_down_sync(0xffffffffu, lfirst, 1);
    const T lnext = lane < 31 ? lsh : T(0);
    a = T(1); b = T(0);
#pragma unroll 8
    for (int t = m - 1; t >= 0; --t) {
        const T ln = t + 1 < m ? (T)lc[(t + 1) * 32] : lnext;
        b = col[t * 33] - ln * b;
        a = -ln * a;
    }
    warp_affine_excl<T, true>(a, b);
    T y = b, ylast = T(0);
#pragma unroll 8
    for (int t = m - 1; t >= 0; --t) {
        const T ln = t + 1 < m ? (T)lc[(t + 1) * 32] : lnext;
        y = col[t * 33] - ln * y;
        col[t * 33] = y;
        if (t == m - 1) ylast = y;
    }
    SW_TRACE(223);
    // Sherman-Morrison correction with y_0 (lane 0, t = 0) and y_{n-1}
    // (lane 31, t = m - 1)
    const T y0 = __shfl_sync(0xffffffffu, y, 0);
    const T yn = __shfl_sync(0xffffffffu, ylast, 31);
    const T s = gam * y0 + ec * yn;
    wfac_wait(f);
#pragma unroll 16
    for (int t = 0; t < m; ++t) col[t * 33] -= (T)zc[t * 32] * s;
    return -1.f;
}

// The same solve with the lane's chunk of MM points and its multipliers held
// in registers: the chunk, the multipliers, the inverse pivots and the
// Sherman-Morrison vector are each read from shared memory once, and the
// four walks run on registers.  Every value is computed by the same
// expressions in the same order as in wtrisolve.  Returns the largest
// magnitude of the lane's results (FP32 rows; -1 for FP64) for the row
// scale of the 16-bit store.
template <class T, class F, int MM>
__device__ __forceinline__ float wtrisolve_r(T *wb, const WRow w, const F *lfT, const F *invDT,
                                            const F *__restrict__ zzT, T gam, T ec, WFac<F> &f)
{
    const int lane = threadIdx.x & 31;
    T *col = wb + lane;
    const F *lc = lfT + lane, *dc = invDT + lane;
    T x[MM], l[MM];
#pragma unroll
    for (int t = 0; t < MM; ++t) {
        x[t] = col[t * 33];
        l[t] = (T)lc[t * 32];
    }
    // forward elimination u_i = b_i - l_i u_{i-1}
    T a = T(1), b = T(0);
#pragma unroll
    for (int t = 0; t < MM; ++t) {
        b = x[t] - l[t] * b;
        a = -l[t] * a;
    }
    SW_TRACE(221);
    warp_affine_excl<T, false>(a, b);
    T u = b;
#pragma unroll
    for (int t = 0; t < MM; ++t) {
        u = x[t] - l[t] * u;
        x[t] = u * (T)dc[t * 32];
    }
    SW_TRACE(222);
    const F *zc = zzT + lane;
    if (f.lf) {
        wfac_copy(f, f.iD, zzT, (F *)nullptr, (const F *)nullptr, w.nx);
        zc = f.iD + lane;
    }
    // back substitution y_i = v_i - l_{i+1} y_{i+1}
    const T lsh = __shfl_down_sync(0xffffffffu, l[0], 1);
    const T lnext = lane < 31 ? lsh : T(0);
    a = T(1); b = T(0);
#pragma unroll
    for (int t = MM - 1; t >= 0; --t) {
        const T ln = t + 1 < MM ? l[t + 1] : lnext;
        b = x[t] - ln * b;
        a = -ln * a;
    }
    warp_affine_excl<T, true>(a, b);
    T y = b;
#pragma unroll
    for (int t = MM - 1; t >= 0; --t) {
        const T ln = t + 1 < MM ? l[t + 1] : lnext;
        y = x[t] - ln * y;
        x[t] = y;
    }
    SW_TRACE(223);
    const T y0 = __shfl_sync(0xffffffffu, x[0], 0);
    const T yn = __shfl_sync(0xffffffffu, x[MM - 1], 31);
    const T s = gam * y0 + ec * yn;
    wfac_wait(f);
    float mx = 0.f;
#pragma unroll
    for (int t = 0; t < MM; ++t) {
        const T r = x[t] - (T)zc[t * 32] * s;
        col[t * 33] = r;
        if constexpr (sizeof(T) == 4) mx = fmaxf(mx, fabsf(r));
    }
    return sizeof(T) == 4 ? mx : -1.f;
}

// store row j of a preconditioner field from the warp's buffer (q_store_row:
// FP64; FP32 on the pole band; else 16-bit with a power-of-two row scale so
// that the stored magnitudes are at most 1), with 16-byte stores.  lmax is
// the lane's largest magnitude when the zonal solve left it (else negative:
// it is taken from the buffer here); it is the same maximum over the same
// values either way.
template <class Pol>
__device__ void wq_store_row(const MemberDev<Pol> &M, typename Pol::q16 *h, float *f32, float *sc, int j,
                             const typename Pol::comp *wb, const WRow w, float lmax)
{
    typedef typename Pol::q16 qt;
    const int lane = threadIdx.x & 31, nx = w.nx;
    const size_t row = (size_t)j * nx;
    if constexpr (!Pol::kMixed) {
        for (int i = 2 * lane; i < nx; i += 64)
            *(double2 *)(h + row + i) = make_double2(wb[tpos(w, i)], wb[tpos(w, i + 1)]);
    } else {
        if (in_band(M, j)) {
            for (int i = 4 * lane; i < nx; i += 128) {
                const int p = tpos4(w, i);
                *(float4 *)(f32 + row + i) = make_float4(wb[p], wb[p + 33], wb[p + 66], wb[p + 99]);
            }
        } else {
            float mx = lmax;
            if (mx < 0.f) {
                mx = 0.f;
                for (int t = 0; t < w.m; ++t) mx = fmaxf(mx, fabsf(wb[t * 33 + lane]));
            }
            mx = warp_max(mx);
            float s = 1.f;
            if (mx > 0.f && mx <= 3.0e38f) { int e; frexpf(mx, &e); s = ldexpf(1.f, e); }
            else if (!(mx <= 3.0e38f)) s = mx;       // NaN / Inf: propagate
            const float inv = 1.f / s;                // exact: s is a power of two
            if (w.m >= 8) {
                // 8 consecutive points per lane (their chunk positions are
                // consecutive: i is a multiple of 8 and m of 8)
                for (int i = 8 * lane; i < nx; i += 256) {
                    const int p = tpos(w, i);
                    qt q[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) q[u] = f_to_q<qt>(wb[p + 33 * u] * inv);
                    uint4 v;
                    memcpy(&v, q, sizeof(v));
                    *(uint4 *)(h + row + i) = v;
                }
            } else {
                for (int i = 4 * lane; i < nx; i += 128) {
                    const int p = tpos4(w, i);
                    qt q[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) q[u] = f_to_q<qt>(wb[p + 33 * u] * inv);
                    uint2 v;
                    memcpy(&v, q, sizeof(v));
                    *(uint2 *)(h + row + i) = v;
                }
            }
            if (lane == 0) sc[j] = s;
        }
    }
}

// the zonal solve of row j (its factors staged by wfac_issue, or read from
// global memory)
template <class Pol, int SEL>
__device__ __forceinline__ float wsolve_row(const MemberDev<Pol> &M, const RowView<Pol> &v, int j,
                                           typename Pol::comp *wb, const WRow w, WFac<typename Pol::fac> &f)
{
    typedef typename Pol::comp comp;
    typedef typename Pol::fac F;
    const size_t row = (size_t)j * M.nx;
    wfac_wait(f);
    SW_TRACE(220);
    const F *lf = f.lf ? (const F *)f.lf : M.lfT + row;
    const F *iD = f.lf ? (const F *)f.iD : M.invDT + row;
    const comp gam = (comp)v.gam, ec = (comp)v.ec;
    // SEL > 0: the kernel is specialised for rows whose chunk is SEL points
    // (its only register variant); SEL < 0: chunks of up to -SEL FP32 points
    // (-SEL / 4 FP64 points) in registers.  Other rows take the walks over
    // shared memory.
    if constexpr (SEL > 0) {
        if (w.m == SEL) return wtrisolve_r<comp, F, SEL>(wb, w, lf, iD, M.zzT + row, gam, ec, f);
        return wtrisolve<comp, F>(wb, w, lf, iD, M.zzT + row, gam, ec, f);
    }
    constexpr int rmax = SEL > 0 ? 0 : (sizeof(comp) == 4 ? -SEL : -SEL / 4);
    switch (w.m) {
    case 4: if constexpr (rmax >= 4) return wtrisolve_r<comp, F, 4>(wb, w, lf, iD, M.zzT + row, gam, ec, f); break;
    case 8: if constexpr (rmax >= 8) return wtrisolve_r<comp, F, 8>(wb, w, lf, iD, M.zzT + row, gam, ec, f); break;
    case 16: if constexpr (rmax >= 16) return wtrisolve_r<comp, F, 16>(wb, w, lf, iD, M.zzT + row, gam, ec, f); break;
    case 32: if constexpr (rmax >= 32) return wtrisolve_r<comp, F, 32>(wb, w, lf, iD, M.zzT + row, gam, ec, f); break;
    case 64: if constexpr (rmax >= 64) return wtrisolve_r<comp, F, 64>(wb, w, lf, iD, M.zzT + row, gam, ec, f); break;
    default: break;
    }
    return wtrisolve<comp, F>(wb, w, lf, iD, M.zzT + row, gam, ec, f);
}

// the zonal solve (option 3) and the store of the first preconditioner stage
// of row j, whose input the warp's buffer holds (stage0_finish)
template <class Pol, int SEL>
__device__ void wstage0_finish(const MemberDev<Pol> &M, const RowView<Pol> &v, int j, typename Pol::comp *wb,
                               const WRow w, WFac<typename Pol::fac> &f, bool staged)
{
    __syncwarp();
    SW_TRACE(211);
    float lmax = -1.f;
    if (M.pc >= 3) lmax = wsolve_row<Pol, SEL>(M, v, j, wb, w, f);
    else if (staged) wfac_wait(f);           // options 0-2: the copies still complete
    __syncwarp();
    SW_TRACE(212);
    if (M.nstages == 1) wq_store_row(M, M.e, M.e32, M.e_s, j, wb, w, lmax);
    else wq_store_row(M, M.qa, M.qa32, M.qa_s, j, wb, w, lmax);
    __syncwarp();
    SW_TRACE(213);
}

// the warp's passes over a row, 4 consecutive points per lane and pass: all
// loads of a pass are issued before its arithmetic
template <class Q, class LD, class CP>
__device__ __forceinline__ void quads(int nx, LD load, CP compute)
{
    const int lane = threadIdx.x & 31;
    for (int i0 = 4 * lane; i0 < nx; i0 += 128) {
        Q a;
        load(i0, a);
        compute(i0, a);
    }
}

// ---------------------------------------------------------------------------
// phases on one row j (one warp); the thread adds its share of the phase's
// inner products to part (phase_true, phase_ub, precond_stage, phase_le)
// ---------------------------------------------------------------------------
template <class Pol, int NP, int SEL>
__device__ void wphase_true(const MemberDev<Pol> &M, const RowView<Pol> &v, typename Pol::comp eta, int j,
                            typename Pol::comp *wb, const WRow w, WFac<typename Pol::fac> &f,
                            typename Acc<Pol>::type (&part)[NP])
{
    typedef typename Pol::comp comp;
    const int nx = M.nx, ny = M.ny, lane = threadIdx.x & 31;
    const size_t row = (size_t)j * nx, rs = j > 0 ? row - nx : row;
    const bool staged = f.lf && M.pc >= 3;
    if (staged) wfac_issue(f, j, M.lfT + row, M.invDT + row, nx);
    const RowCoef<double> c = {M.ax + row, M.cx + row, M.bx + row, M.ay + row, M.cy + row, M.by + row,
                               M.ay + rs, M.cy + rs, M.by + rs, M.C + row};
    int srcS, shS, srcN, shN;
    ghost_row(j - 1, nx, ny, srcS, shS);
    ghost_row(j + 1, nx, ny, srcN, shN);
    const double *pX = M.phi + row, *pN = M.phi + (size_t)srcN * nx, *pS = M.phi + (size_t)srcS * nx;
    const bool has_n = j < ny - 1, has_s = j > 0;
    double rr = 0.0, RR = 0.0;
    for (int i0 = 4 * lane; i0 < nx; i0 += 128) {
        double xc[6], xn[6], xs[6];
        cg6(pX, i0, nx, xc);
        int a = i0 + shN; if (a >= nx) a -= nx;
        cg6(pN, a, nx, xn);
        a = i0 + shS; if (a >= nx) a -= nx;
        cg6(pS, a, nx, xs);
        Coef4<double> k;
        coef4(c, i0, nx, true, has_n, has_s, k);
        double Rv[4];
        ldg4(M.R + row + i0, Rv);
        double lphi[4];
        apply4(k, xc, xn, xs, has_n, has_s, lphi);
        const int p0 = tpos4(w, i0);
        typename Pol::res r4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double rv = lphi[u] - Rv[u];
            r4[u] = (typename Pol::res)rv;
            rr += rv * rv;
            RR += Rv[u] * Rv[u];
            wb[p0 + 33 * u] = stage0_input(M, v, eta, (comp)r4[u], i0 + u);
        }
        stv4(v.r + i0, r4);
    }
    part[0] += (typename Acc<Pol>::type)rr;
    part[1] += (typename Acc<Pol>::type)RR;
    wstage0_finish<Pol, SEL>(M, v, j, wb, w, f, staged);
}

// streaming store (evict-first) of 4 values: the update's p, L p and Phi,
// which no phase reads again before the next update (measured 0.5 % faster at
// 2048 x 1024 than plain stores)
template <class T>
__device__ __forceinline__ void stv4cs(T *p, const T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        __stcs((float4 *)p, make_float4(v[0], v[1], v[2], v[3]));
    } else {
        __stcs((double2 *)p, make_double2(v[0], v[1]));
        __stcs((double2 *)p + 1, make_double2(v[2], v[3]));
    }
}

template <class Pol, int KM>
struct UbQuad {
    typename Pol::comp ev[4];
    typename Pol::vec le4[4], pv4[KM][4], lp4[KM][4];
    typename Pol::res r4[4];
    double ph4[4];
};

template <class Pol, int KM, int SEL>
__device__ void wphase_ub(const MemberDev<Pol> &M, const MemberCtl &c, const RowView<Pol> &v,
                          typename Pol::comp eta, int j, typename Pol::comp *wb, const WRow w,
                          WFac<typename Pol::fac> &f, typename Acc<Pol>::type (&part)[2 + 2 * KM])
{
    typedef typename Pol::comp comp;
    typedef typename Pol::vec vec;
    typedef typename Acc<Pol>::type acc_t;
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    const bool staged = f.lf && M.pc >= 3;
    if (staged) wfac_issue(f, j, M.lfT + row, M.invDT + row, nx);
    const int nd = c.nu + 1;                      // directions before the new one
    vec *pn = v.pb + (size_t)phys_slot(c, M.k, nd) * v.vstride;
    vec *Lpn = v.Lpb + (size_t)phys_slot(c, M.k, nd) * v.vstride;
    const vec *pl[KM], *Lpl[KM];
    comp al[KM];
#pragma unroll
    for (int l = 0; l < KM; ++l) {
        const size_t off = (size_t)phys_slot(c, M.k, l < nd ? l : 0) * v.vstride;
        pl[l] = v.pb + off;
        Lpl[l] = v.Lpb + off;
        al[l] = l < nd ? (comp)c.alpha[l] : (comp)0;
    }
    const QRow<Pol> eq = qrow(M, M.e, M.e32, M.e_s, j);
    const double beta = c.beta;
    const comp beta_c = (comp)beta;
    double *ph = M.phi + row;
    auto load = [&](int i0, UbQuad<Pol, KM> &d) {
        q4own(eq, i0, d.ev);
        ldv4(v.Le + i0, d.le4);
        ldv4(v.r + i0, d.r4);
        ldv4(ph + i0, d.ph4);
#pragma unroll
        for (int l = 0; l < KM; ++l) {
            if (l < nd) {
                ldv4(pl[l] + i0, d.pv4[l]);
                ldv4(Lpl[l] + i0, d.lp4[l]);
            }
        }
    };
    auto compute = [&](int i0, UbQuad<Pol, KM> &d) {
        vec ps4[4], ls4[4];
        typename Pol::res rs4[4];
        double phn[4];
        const int p0 = tpos4(w, i0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            comp pv = d.ev[u], lw = (comp)d.le4[u];
#pragma unroll
            for (int l = 0; l < KM; ++l) {
                if (l < nd) {
                    pv += al[l] * (comp)d.pv4[l][u];
                    lw += al[l] * (comp)d.lp4[l][u];
                }
            }
            ps4[u] = (vec)pv;
            ls4[u] = (vec)lw;
            phn[u] = d.ph4[u] + beta * (double)ps4[u];
            if constexpr (Pol::kMixed) rs4[u] = (typename Pol::res)((comp)d.r4[u] + beta_c * ls4[u]);
            else rs4[u] = (comp)d.r4[u] + beta * ls4[u];
            const acc_t ra = (acc_t)rs4[u], la = (acc_t)ls4[u];
            part[0] += ra * ra;
            part[1] += la * la;
#pragma unroll
            for (int l = 0; l < KM; ++l)
                if (l < nd) part[2 + l] += la * (acc_t)d.lp4[l][u];
            wb[p0 + 33 * u] = stage0_input(M, v, eta, (comp)rs4[u], i0 + u);
        }
        stv4cs(pn + i0, ps4);
        stv4cs(Lpn + i0, ls4);
        stv4cs(ph + i0, phn);
        stv4(v.r + i0, rs4);
    };
    quads<UbQuad<Pol, KM>>(nx, load, compute);
    wstage0_finish<Pol, SEL>(M, v, j, wb, w, f, staged);
}

template <class Pol>
struct StQuad {
    typename Pol::comp xc[6], xn[6], xs[6], rv[4], dg[4];
    Coef4<typename Pol::coef> k;
};

// Richardson stage mu >= 1 (precond_stage): reads q_mu on rows j - 1 .. j + 1,
// writes q_{mu+1} (the last stage writes e)
template <class Pol, int SEL>
__device__ void wprecond_stage(const MemberDev<Pol> &M, const RowView<Pol> &v, typename Pol::comp eta, int mu,
                               int j, typename Pol::comp *wb, const WRow w, WFac<typename Pol::fac> &f)
{
    typedef typename Pol::comp comp;
    typedef typename Pol::coef CT;
    const int nx = M.nx, ny = M.ny;
    const size_t row = (size_t)j * nx;
    const bool opt3 = (M.pc >= 3), has_n = j < ny - 1, has_s = j > 0;
    const bool staged = f.lf && opt3;
    if (staged) wfac_issue(f, j, M.lfT + row, M.invDT + row, nx);
    const bool last = (mu == M.nstages - 1);
    const typename Pol::q16 *ih = (mu & 1) ? M.qa : M.qb;
    const float *if32 = (mu & 1) ? M.qa32 : M.qb32;
    const float *is = (mu & 1) ? M.qa_s : M.qb_s;
    typename Pol::q16 *oh = last ? M.e : ((mu & 1) ? M.qb : M.qa);
    float *of32 = last ? M.e32 : ((mu & 1) ? M.qb32 : M.qa32);
    float *os = last ? M.e_s : ((mu & 1) ? M.qb_s : M.qa_s);
    const QRow<Pol> qS = qrow(M, ih, if32, is, j - 1), qX = qrow(M, ih, if32, is, j), qN = qrow(M, ih, if32, is, j + 1);
    const RowCoef<CT> c = coef_of(v);
    // PL: option 3 on a plain row (rows_plain), conditions fixed at compile time
    auto pass = [&](auto plain_t) {
        constexpr bool PL = decltype(plain_t)::value;
        const bool o3 = PL || opt3, hn = PL || has_n, hs = PL || has_s;
        auto load = [&](int i0, StQuad<Pol> &d) {
            if constexpr (PL) {
                q6i(qX, i0, nx, d.xc);
                q6i(qN, i0, nx, d.xn);
                q6i(qS, i0, nx, d.xs);
            } else {
                q6(qX, i0, nx, d.xc);
                q6(qN, i0, nx, d.xn);
                q6(qS, i0, nx, d.xs);
            }
            coef4(c, i0, nx, !o3, hn, hs, d.k);
            ldv4(v.r + i0, d.rv);
#pragma unroll
            for (int u = 0; u < 4; ++u) d.dg[u] = comp(1);
            if (!o3) {
                CT d4[4];
                ldg4(v.diag + i0, d4);
#pragma unroll
                for (int u = 0; u < 4; ++u) d.dg[u] = (comp)d4[u];
            }
        };
        auto compute = [&](int i0, StQuad<Pol> &d) {
            comp y[4];
            apply4(d.k, d.xc, d.xn, d.xs, hn, hs, y);
            const int p0 = tpos4(w, i0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const comp xv = d.xc[u + 1];
                wb[p0 + 33 * u] = o3 ? xv + eta * (y[u] - d.rv[u]) : xv + (comp)M.omega * (d.rv[u] - y[u]) / d.dg[u];
            }
        };
        quads<StQuad<Pol>>(nx, load, compute);
    };
    if constexpr (SEL < 0) {
        if (opt3 && rows_plain(qS, qX, qN, has_n, has_s)) pass(std::true_type{});
        else pass(std::false_type{});
    } else {
        pass(std::false_type{});
    }
    __syncwarp();
    SW_TRACE(311);
    float lmax = -1.f;
    if (opt3) lmax = wsolve_row<Pol, SEL>(M, v, j, wb, w, f);
    __syncwarp();
    SW_TRACE(312);
    wq_store_row(M, oh, of32, os, j, wb, w, lmax);
    __syncwarp();
    SW_TRACE(313);
}

template <class Pol, int KM>
struct LeQuad {
    typename Pol::comp xc[6], xn[6], xs[6];
    Coef4<typename Pol::coef> k;
    typename Pol::res r4[4];
    typename Pol::vec lp4[KM][4];
};

// L(e) of row j into the row's L e and the inner products <Le,Le>, <r,Le>,
// <Le,Lp_l>, <r,Lp_l> (phase_le)
template <class Pol, int KM, int SEL>
__device__ void wphase_le(const MemberDev<Pol> &M, const MemberCtl &c, const RowView<Pol> &v, int j, const WRow w,
                          typename Acc<Pol>::type (&part)[2 + 2 * KM])
{
    typedef typename Pol::comp comp;
    typedef typename Pol::vec vec;
    typedef typename Pol::coef CT;
    typedef typename Acc<Pol>::type acc_t;
    const int nx = M.nx, ny = M.ny;
    const int nd = c.nu + 1;
    const QRow<Pol> qS = qrow(M, M.e, M.e32, M.e_s, j - 1), qX = qrow(M, M.e, M.e32, M.e_s, j),
                    qN = qrow(M, M.e, M.e32, M.e_s, j + 1);
    const bool has_n = j < ny - 1, has_s = j > 0;
    const RowCoef<CT> cf = coef_of(v);
    const vec *Lpl[KM];
#pragma unroll
    for (int l = 0; l < KM; ++l) Lpl[l] = v.Lpb + (size_t)phys_slot(c, M.k, l < nd ? l : 0) * v.vstride;
    // PL: a plain row (rows_plain), conditions fixed at compile time
    auto pass = [&](auto plain_t) {
        constexpr bool PL = decltype(plain_t)::value;
        const bool hn = PL || has_n, hs = PL || has_s;
        auto load = [&](int i0, LeQuad<Pol, KM> &d) {
            if constexpr (PL) {
                q6i(qX, i0, nx, d.xc);
                q6i(qN, i0, nx, d.xn);
                q6i(qS, i0, nx, d.xs);
            } else {
                q6(qX, i0, nx, d.xc);
                q6(qN, i0, nx, d.xn);
                q6(qS, i0, nx, d.xs);
            }
            coef4(cf, i0, nx, true, hn, hs, d.k);
            ldv4(v.r + i0, d.r4);
#pragma unroll
            for (int l = 0; l < KM; ++l)
                if (l < nd) ldv4(Lpl[l] + i0, d.lp4[l]);
        };
        auto compute = [&](int i0, LeQuad<Pol, KM> &d) {
            comp y[4];
            apply4(d.k, d.xc, d.xn, d.xs, hn, hs, y);
            vec le4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) le4[u] = (vec)y[u];
            stv4(v.Le + i0, le4);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const acc_t la = (acc_t)le4[u], rv = (acc_t)d.r4[u];
                part[0] += la * la;
                part[1] += rv * la;
#pragma unroll
                for (int l = 0; l < KM; ++l) {
                    if (l < nd) {
                        part[2 + l] += la * (acc_t)d.lp4[l][u];
                        part[2 + KM + l] += rv * (acc_t)d.lp4[l][u];
                    }
                }
            }
        };
        quads<LeQuad<Pol, KM>>(nx, load, compute);
    };
    if constexpr (SEL < 0) {
        if (rows_plain(qS, qX, qN, has_n, has_s)) pass(std::true_type{});
        else pass(std::false_type{});
    } else {
        pass(std::false_type{});
    }
    SW_TRACE(111);
}

// the first stage of option 3 from the stored r (phase_prec0)
template <class Pol, int SEL>
__device__ void wphase_prec0(const MemberDev<Pol> &M, const RowView<Pol> &v, typename Pol::comp eta, int j,
                             typename Pol::comp *wb, const WRow w, WFac<typename Pol::fac> &f)
{
    typedef typename Pol::comp comp;
    const int lane = threadIdx.x & 31;
    const bool staged = f.lf && M.pc >= 3;
    if (staged) wfac_issue(f, j, M.lfT + (size_t)j * M.nx, M.invDT + (size_t)j * M.nx, M.nx);
    for (int i0 = 4 * lane; i0 < M.nx; i0 += 128) {
        typename Pol::res r4[4];
        ldv4(v.r + i0, r4);
        const int p0 = tpos4(w, i0);
#pragma unroll
        for (int u = 0; u < 4; ++u) wb[p0 + 33 * u] = stage0_input(M, v, eta, (comp)r4[u], i0 + u);
    }
    wstage0_finish<Pol, SEL>(M, v, j, wb, w, f, staged);
}

// shared memory of one warp in the warp-per-row mode: its row buffer, then
// (when staged) the row's transposed lf and invD and the mbarrier
template <class Pol>
__host__ __device__ inline size_t warp_slot_bytes(int nx, bool stage)
{
    const size_t wbuf = al16((size_t)wbuf_len(nx) * sizeof(typename Pol::comp));
    const size_t fac = stage ? al16(2 * (size_t)nx * sizeof(typename Pol::fac)) + 16 : 0;
    return (wbuf + fac + 127) & ~(size_t)127;
}

} // namespace sw
