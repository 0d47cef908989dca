// sw_block.cuh -- block-level building blocks of the solver.  One thread
// block works on one latitude row at a time: reductions and scans within a
// row use warp shuffles plus one exchange through shared memory.
#pragma once

#include "sw_common.cuh"

namespace sw {

// Optional device timeline for performance work: built only with
// -DSW_PHASE_TRACE, thread 0 of one chosen block appends (globaltimer, tag)
// pairs to a caller buffer at the SW_TRACE points.  It changes no results.
#ifdef SW_PHASE_TRACE
__device__ __forceinline__ unsigned long long trace_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
static __device__ unsigned long long *g_trace_buf = nullptr;
static __device__ int g_trace_n = 0, g_trace_cap = 0, g_trace_blk = 0;
#define SW_TRACE(tag)                                                                      \
    do {                                                                                  \
        if (::sw::g_trace_buf && blockIdx.x == ::sw::g_trace_blk && threadIdx.x == 0 &&   \
            ::sw::g_trace_n < ::sw::g_trace_cap) {                                        \
            const int q_ = ::sw::g_trace_n++;                                             \
            ::sw::g_trace_buf[2 * q_] = ::sw::trace_clock();                              \
            ::sw::g_trace_buf[2 * q_ + 1] = (unsigned long long)(tag);                    \
        }                                                                                 \
    } while (0)
#else
#define SW_TRACE(tag) ((void)0)
#endif

// Row buffers used by the chunked tridiagonal scans are stored with one pad
// word per 32 values, which keeps the per-thread chunk accesses of a warp on
// distinct shared-memory banks.
__host__ __device__ __forceinline__ int pidx(int i) { return i + (i >> 5); }
__host__ __device__ inline int padded_len(int n) { return n + (n >> 5) + 1; }

__device__ __forceinline__ float warp_max(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Sum over the warp of 32 values per lane at once (transposed butterfly):
// five exchange levels, each halving the values a lane keeps; lane l ends
// with the total of value l.  The pairing, hence the rounding, is fixed.
template <class T>
__device__ __forceinline__ T warp_sum32(T (&v)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, cnt = 32; o > 0; o >>= 1, cnt >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < cnt / 2; ++k) {
            T send = hi ? v[k] : v[k + cnt / 2];
            T keep = hi ? v[k + cnt / 2] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// Block sum of NV <= 32 values per thread; tot[q] (shared memory) receives
// total q in FP64.  scratch: 32 doubles per warp.  Fixed order: a warp
// butterfly in T, then the warps in index order in FP64.
template <int NV, class T>
__device__ __forceinline__ void block_sum_many(const T (&x)[NV], double *tot, double *scratch)
{
    static_assert(NV <= 32, "");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = q < NV ? x[q] : T(0);
    const T s = warp_sum32(v);
    scratch[w * 32 + lane] = (double)s;
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0;
        for (int ww = 0; ww < nw; ++ww) t += scratch[ww * 32 + threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
}

// Double-float arithmetic (a value as an unevaluated sum hi + lo of two
// floats; Knuth's error-free TwoSum): about 44 significant bits on the FP32
// pipe.  On this GPU an FP64 instruction costs about 64 cycles per warp
// against about 5 for FP32, so the mixed policies keep their block and member
// sums in this form and convert to FP64 once per total.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b)
{
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);
    e += a.lo + b.lo;
    const float hi = s + e;
    return dfloat{hi, e - (hi - s)};
}

// Block sum of NV <= 32 FP32 values per thread into double-float totals
// tot[q] (shared memory): a warp butterfly in FP32, then the warps in index
// order in double-float.  scratch: 32 floats per warp.
template <int NV>
__device__ __forceinline__ void block_sum_many_df(const float (&x)[NV], dfloat *tot, float *scratch)
{
    static_assert(NV <= 32, "");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = q < NV ? x[q] : 0.f;
    scratch[w * 32 + lane] = warp_sum32(v);
    __syncthreads();
    if (threadIdx.x < NV) {
        dfloat t{0.f, 0.f};
        for (int ww = 0; ww < nw; ++ww) t = df_add(t, dfloat{scratch[ww * 32 + threadIdx.x], 0.f});
        tot[threadIdx.x] = t;
    }
    __syncthreads();
}

// Exclusive block scan of affine maps x -> a x + b in thread order (REV:
// reversed thread order).  On return (a, b) composes the maps of the earlier
// threads.  sm: 2 values per warp.
template <class T, bool REV>
__device__ __forceinline__ void block_affine_excl(T &a, T &b, T *sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T ia = a, ib = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T oa = REV ? __shfl_down_sync(0xffffffffu, ia, d) : __shfl_up_sync(0xffffffffu, ia, d);
        T ob = REV ? __shfl_down_sync(0xffffffffu, ib, d) : __shfl_up_sync(0xffffffffu, ib, d);
        bool ok = REV ? (lane + d < 32) : (lane >= d);
        if (ok) { ib = ia * ob + ib; ia = ia * oa; }
    }
    T ea = REV ? __shfl_down_sync(0xffffffffu, ia, 1) : __shfl_up_sync(0xffffffffu, ia, 1);
    T eb = REV ? __shfl_down_sync(0xffffffffu, ib, 1) : __shfl_up_sync(0xffffffffu, ib, 1);
    if (REV ? lane == 31 : lane == 0) { ea = T(1); eb = T(0); }
    if (nw > 1) {
        if (REV ? lane == 0 : lane == 31) { sm[2 * w] = ia; sm[2 * w + 1] = ib; }
        __syncthreads();
        T pa = T(1), pb = T(0);
        if (!REV) {
            for (int ww = 0; ww < w; ++ww) { T ga = sm[2 * ww], gb = sm[2 * ww + 1]; pb = ga * pb + gb; pa = ga * pa; }
        } else {
            for (int ww = nw - 1; ww > w; --ww) { T ga = sm[2 * ww], gb = sm[2 * ww + 1]; pb = ga * pb + gb; pa = ga * pa; }
        }
        __syncthreads();
        a = ea * pa;
        b = ea * pb + eb;
    } else {
        a = ea;
        b = eb;
    }
}

// Cyclic zonal solve T x = b of one row by one block, in place on the padded
// row buffer sb (length n).  T' = L D L^T with multipliers lf (lf[0] = 0) and
// inverse pivots invD; with zz = z / (gam + w.z) the Sherman-Morrison step is
// x = y - zz (gam y_0 + ec y_{n-1}) (no correction when zz is null).  FP: the
// factor rows are padded too.  Every thread owns a contiguous chunk of at most
// RM values held in registers (n <= RM * blockDim.x), so all loads are issued
// before the recurrences run; trisolve_block picks the smallest RM that fits.
constexpr int TRI_RM = 16;

template <int RM, class T, class F, bool FP>
__device__ __noinline__ void trisolve_rm(T *sb, int n, const F *lf, const F *invD, const F *zz, T gam, T ec, T *sm)
{
    const int m = (n + blockDim.x - 1) / blockDim.x;
    const int c0 = min((int)threadIdx.x * m, n), c1 = min(c0 + m, n);
    T x[RM], l[RM], d[RM], z[RM];
#pragma unroll
    for (int t = 0; t < RM; ++t) {
        const int i = min(c0 + t, n - 1);
        const int fi = FP ? pidx(i) : i;
        x[t] = sb[pidx(i)];
        l[t] = (T)lf[fi];
        d[t] = (T)invD[fi];
        z[t] = zz ? (T)zz[fi] : T(0);
    }
    const T lnext = (c1 < n && c1 > c0) ? (T)lf[FP ? pidx(c1) : c1] : T(0);
    // forward elimination u_i = b_i - l_i u_{i-1}
    T a = T(1), b = T(0);
#pragma unroll
    for (int t = 0; t < RM; ++t)
        if (c0 + t < c1) { b = x[t] - l[t] * b; a = -l[t] * a; }
    block_affine_excl<T, false>(a, b, sm);
    T u = b;
#pragma unroll
    for (int t = 0; t < RM; ++t)
        if (c0 + t < c1) { u = x[t] - l[t] * u; x[t] = u * d[t]; }
    // back substitution y_i = v_i - l_{i+1} y_{i+1}
    a = T(1); b = T(0);
#pragma unroll
    for (int t = RM - 1; t >= 0; --t) {
        if (c0 + t < c1) {
            const T ln = (c0 + t + 1 < c1) ? l[t + 1 < RM ? t + 1 : RM - 1] : lnext;
            b = x[t] - ln * b; a = -ln * a;
        }
    }
    block_affine_excl<T, true>(a, b, sm);
    T y = b;
#pragma unroll
    for (int t = RM - 1; t >= 0; --t) {
        if (c0 + t < c1) {
            const T ln = (c0 + t + 1 < c1) ? l[t + 1 < RM ? t + 1 : RM - 1] : lnext;
            y = x[t] - ln * y; x[t] = y;
        }
    }
    // Sherman-Morrison correction with y_0 and y_{n-1}
#pragma unroll
    for (int t = 0; t < RM; ++t)
        if (c0 + t < c1 && (c0 + t == 0 || c0 + t == n - 1)) sb[pidx(c0 + t)] = x[t];
    __syncthreads();
    const T s = zz ? gam * sb[pidx(0)] + ec * sb[pidx(n - 1)] : T(0);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < RM; ++t)
        if (c0 + t < c1) sb[pidx(c0 + t)] = x[t] - z[t] * s;
    __syncthreads();
}

template <class T, class F, bool FP>
__device__ __forceinline__ void trisolve_block(T *sb, int n, const F *lf, const F *invD, const F *zz, T gam, T ec,
                                               T *sm)
{
    const int m = (n + blockDim.x - 1) / blockDim.x;
    if (m <= 2) trisolve_rm<2, T, F, FP>(sb, n, lf, invD, zz, gam, ec, sm);
    else if (m <= 4) trisolve_rm<4, T, F, FP>(sb, n, lf, invD, zz, gam, ec, sm);
    else if (m <= 8) trisolve_rm<8, T, F, FP>(sb, n, lf, invD, zz, gam, ec, sm);
    else trisolve_rm<16, T, F, FP>(sb, n, lf, invD, zz, gam, ec, sm);
}

// ---------------------------------------------------------------------------
// row copies global -> shared for data written by other blocks during the
// launch: cp.async.cg (16-byte pieces, cached at L2 only) when both ends are
// 16-byte aligned, else coherent 32-bit loads; finish with row_copy_wait
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool al16ptr(const void *p) { return ((uintptr_t)p & 15) == 0; }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void row_copy_issue(void *dst, const void *src, int nbytes)
{
    if (al16ptr(dst) && al16ptr(src) && (nbytes & 15) == 0) {
        for (int off = threadIdx.x * 16; off < nbytes; off += blockDim.x * 16)
            cp_async16((char *)dst + off, (const char *)src + off);
    } else {
        const unsigned *s = (const unsigned *)src;
        unsigned *d = (unsigned *)dst;
        const int nwd = nbytes >> 2, T = blockDim.x;
        for (int b0 = threadIdx.x; b0 < nwd; b0 += T * 8) {
            unsigned v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (b0 + T * u < nwd) ? __ldcg(s + b0 + T * u) : 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (b0 + T * u < nwd) d[b0 + T * u] = v[u];
        }
    }
}

__device__ __forceinline__ void row_copy_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}

// release / acquire operations on the barrier counter
__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

} // namespace sw
