// sw_common.cuh -- shared device-side definitions of the GB300 elliptic solver:
// precision policies, the per-member solver state, bounded grid barrier,
// deterministic block reductions and block-wide scans of affine maps.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/sw_elliptic.h"

namespace sw {

constexpr int KMAX = 8;             // largest GCR k
// row partial sums kept per row and phase (two buffers by phase parity):
//   PH_TRUE: ||r||^2, ||R||^2
//   PH_LE:   <Le,Le>, <r,Le>, <Le,Lp_l> (l < nd), <r,Lp_l> (l < nd)
//   PH_UB:   ||r||^2, <Lp_new,Lp_new>, <Lp_new,Lp_m> (m < nd)
constexpr int NSLOT = 2 + 2 * KMAX;
constexpr int S_A = 0, S_B = 1, S_C0 = 2, S_T0 = 2 + KMAX;
constexpr int MAX_MEMBERS = 480;    // members of one ensemble launch
constexpr int MAX_NX = 4096;
constexpr int MAX_THREADS = 256;    // block size of the row kernels

// phase kinds of the GCR state machine (see sw_solver.cu)
enum Phase : int { PH_TRUE = 0, PH_UB = 1, PH_PREC = 2, PH_LE = 3, PH_ZERO = 5, PH_DONE = 6,
                   PH_EXT = 7,    // learned preconditioner: the launch ends, the host applies the network
                   PH_PREC0 = 8   // first stage of option 3 from r (a learned iteration falling back)
};
constexpr int PC_LEARNED = 4;

// status codes (mirror sw_status)
enum : int { ST_OK = 0, ST_INVALID = 1, ST_CUDA = 2, ST_OOM = 3, ST_NOT_CONVERGED = 4,
             ST_BREAKDOWN = 5, ST_NONFINITE = 6, ST_TIMEOUT = 7, ST_INTERNAL = 8 };

// ---------------------------------------------------------------------------
// precision policies
//   comp : arithmetic type of the operator / preconditioner / vector updates
//   coef : stored face coefficients used by that arithmetic
//   fac  : stored factors of the zonal tridiagonal operators
//   vec  : p, L p, L e
//   res  : recursive residual r
//   q16  : storage of the preconditioner's intermediate q and output e
//          (double for FP64; half / bf16 with one FP32 scale per row otherwise)
// Phi, the true residual, R and every inner product are FP64 in all policies.
// ---------------------------------------------------------------------------
struct PolFP64 {
    typedef double comp; typedef double coef; typedef double fac;
    typedef double vec;  typedef double res;  typedef double q16;
    static constexpr bool kMixed = false;
};
struct PolF16 {
    typedef float comp; typedef float coef; typedef float fac;
    typedef float vec;  typedef float res;  typedef __half q16;
    static constexpr bool kMixed = true;
};
struct PolBF16 {
    typedef float comp; typedef float coef; typedef float fac;
    typedef float vec;  typedef float res;  typedef __nv_bfloat16 q16;
    static constexpr bool kMixed = true;
};

// accumulation type of each thread's inner-product partials and of the warp
// sums: FP64 for the FP64 policy, FP32 for the mixed policies (at most 32
// threads' partials of a few products each).  The mixed policies add the
// warps and the blocks in double-float (sw_block.cuh) and convert each total
// to FP64 once; the FP64 policy adds in FP64.  The GCR scalars are FP64 for
// every policy.
template <class Pol> struct Acc { typedef double type; };
template <> struct Acc<PolF16> { typedef float type; };
template <> struct Acc<PolBF16> { typedef float type; };

__device__ __forceinline__ float q_to_f(__half h) { return __half2float(h); }
__device__ __forceinline__ float q_to_f(__nv_bfloat16 h) { return __bfloat162float(h); }
__device__ __forceinline__ double q_to_f(double h) { return h; }
template <class H> __device__ __forceinline__ H f_to_q(float x);
template <> __device__ __forceinline__ __half f_to_q<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 f_to_q<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// L2-coherent load for data written by other blocks during the same launch
template <class T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// grid-level data of one member (one elliptic problem) -- immutable during a launch
// ---------------------------------------------------------------------------
template <class Pol>
struct MemberDev {
    typedef typename Pol::coef coef_t;
    typedef typename Pol::fac fac_t;
    typedef typename Pol::vec vec_t;
    typedef typename Pol::res res_t;
    typedef typename Pol::q16 q_t;

    int nx, ny;
    int k, pc, nstages, min_iters, max_iters, ru_every, band;
    double tol, omega;
    double fb_ratio;                // learned preconditioner: fallback threshold
    const double *etap;             // device: eta of the factorised zonal operators
    // FP64 face coefficients (true residual): face x (i+1/2, j): ax = a11/dlam^2,
    // cx = a12/(4 dlam dphi), bx = b1/(2 dlam); face y (i, j+1/2): ay = a22/dphi^2,
    // cy = a21/(4 dlam dphi), by = b2/(2 dphi); C
    const double *ax, *cx, *bx, *ay, *cy, *by, *C;
    // the same in the policy's coefficient type, and diag(L) (options 1, 2)
    const coef_t *wax, *wcx, *wbx, *way, *wcy, *wby, *wC, *wdiag;
    // zonal factors of T = I - eta (P^Z - P^H): multipliers, inverse pivots,
    // Sherman-Morrison vector; per row gamma and the wrap coupling
    const fac_t *lf, *invD, *zz;
    // the same factors transposed per row for the warp-per-row path: point i
    // of a row at (i % m) * 32 + i / m, m = nx / 32 (null when not stored)
    const fac_t *lfT, *invDT, *zzT;
    const double *gam, *ec;
    // solve fields
    const double *R;
    double *phi;
    res_t *r;
    q_t *qa, *qb, *e;               // intermediates and preconditioner output
    float *qa32, *qb32, *e32;       // FP32 storage of the pole-band rows (mixed)
    float *qa_s, *qb_s, *e_s;       // per-row scales of the 16-bit storage
    vec_t *Le, *p, *Lp;             // p, Lp: (k+1) slots of nx*ny
    double *part;                   // [2][NSLOT][ny] block partial sums (phase parity)
    double *hist;                   // optional residual history
    double *rowres;                 // optional per-row final residual
    // split fluid thickness (Sec. 4.2, Eq. 14): the initial residual in FP32
    // from Phi_hat and its stored derivative parts (mixed policies)
    int split, pad_split_;
    const float *shat, *sdx, *scx, *sdy, *scy;
};

// per-member GCR state.  Every block of the member keeps an identical copy in
// shared memory and advances it with the same deterministic reductions; the
// global copy holds the initial state (from the host) and the final one.
struct MemberCtl {
    int phase, stage, it, nu, base, init, status, pad_;
    int fb_now, fallbacks;          // learned preconditioner: this iteration fell back; count
    int net_turn, pad2_;            // learned preconditioner: the next direction is the network's
    double beta, nR, r0, rn_true;
    double rn2_rec;                 // ||r||^2 of the recursive residual
    double rn2_cur;                 // ||r||^2 of the residual the next direction works on
    double g3;                      // share of ||r||^2 the last option-3 direction removed
    double tolr, tolr2;             // exit threshold on ||r|| and its square (set with ||R||)
    double alpha[KMAX + 1];
    double G[KMAX + 1][KMAX + 1];   // Gram matrix <L p_l, L p_m> of the cycle (logical)
    double Ginv[KMAX + 1];          // 1 / G[l][l], formed once per direction
};

struct GlobalCtl {
    unsigned long long count;       // member barrier arrivals (monotonic)
    int abort;                      // set on a device-side error (timeout)
    int where;                      // diagnostic: step of the abort
};

// one member's device block (one per grid)
struct alignas(256) SolverBlock {
    unsigned char dev[sizeof(MemberDev<PolFP64>) > sizeof(MemberDev<PolF16>)
                      ? sizeof(MemberDev<PolFP64>) : sizeof(MemberDev<PolF16>)];
    MemberCtl ctl;
    GlobalCtl g;
    int lturns;                     // network turns of the device-side learned loop
};

// a one-member launch: the member and launch descriptors travel as kernel
// parameters of k_init_one instead of host-to-device copies
struct InitOneArgs {
    alignas(16) unsigned char mdev[sizeof(SolverBlock::dev)];
    SolverBlock *blk;
    struct EnsDesc *desc;
    sw_solve_stats *stats;
    int grid, nb0, cache_const, cache_state, warp_rows, warp_stage;
};

// members of one persistent launch and their block ranges
struct EnsDesc {
    int n, grid;
    int cache_const, cache_state;   // row constants / owner-only vectors in shared memory
    int warp_rows;                  // one warp per latitude row (sw_warp.cuh) instead of one block
    int warp_stage;                 // warp mode: rows' zonal factors staged in shared memory
    sw_solve_stats *stats;          // device, n entries, or null: each member's stats at the end
    int cta_begin[MAX_MEMBERS + 1];
    SolverBlock *blk[MAX_MEMBERS];
};

// rows one warp can own in the warp-per-row solver (sw_warp.cuh): a power of
// two of 128 .. MAX_NX points
__host__ __device__ inline bool warp_rows_ok(int nx) { return nx >= 128 && nx <= MAX_NX && (nx & (nx - 1)) == 0; }

// physical slot of the cycle's logical direction l (restarts rotate the base)
__device__ __forceinline__ int phys_slot(const MemberCtl &c, int k, int l) { return (c.base + l) % (k + 1); }

// ---------------------------------------------------------------------------
// block-level helpers (blockDim.x a multiple of 32, <= MAX_THREADS)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int nwarps() { return blockDim.x >> 5; }

// deterministic sum of ns values per thread over the block; result valid in
// every thread. red: nwarps*ns doubles of shared memory.
__device__ __forceinline__ void block_sum(double *v, int ns, double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = 0; s < ns; ++s) {
        double x = v[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w * ns + s] = x;
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
        double x = 0.0;
        for (int ww = 0; ww < nwarps(); ++ww) x += red[ww * ns + s];
        v[s] = x;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(float x, float *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) red[w] = x;
    __syncthreads();
    float m = 0.f;
    for (int ww = 0; ww < nwarps(); ++ww) m = fmaxf(m, red[ww]);
    __syncthreads();
    return m;
}

// Exclusive block scan of affine maps x -> a x + b in processing order.
// Forward: thread order; reverse: reversed thread order.  On return (a, b) is
// the composition of the maps of all threads before this one (identity for
// the first).  sm: 2*nwarps values of T in shared memory.
template <class T, bool REV>
__device__ __forceinline__ void scan_affine_excl(T &a, T &b, T *sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = nwarps();
    T ia = a, ib = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T oa = REV ? __shfl_down_sync(0xffffffffu, ia, d) : __shfl_up_sync(0xffffffffu, ia, d);
        T ob = REV ? __shfl_down_sync(0xffffffffu, ib, d) : __shfl_up_sync(0xffffffffu, ib, d);
        bool ok = REV ? (lane + d < 32) : (lane >= d);
        if (ok) { ib = ia * ob + ib; ia = ia * oa; }   // mine after the earlier ones
    }
    T ea = REV ? __shfl_down_sync(0xffffffffu, ia, 1) : __shfl_up_sync(0xffffffffu, ia, 1);
    T eb = REV ? __shfl_down_sync(0xffffffffu, ib, 1) : __shfl_up_sync(0xffffffffu, ib, 1);
    if (REV ? lane == 31 : lane == 0) { ea = T(1); eb = T(0); }
    if (REV ? lane == 0 : lane == 31) { sm[2 * w] = ia; sm[2 * w + 1] = ib; }
    __syncthreads();
    T pa = T(1), pb = T(0);        // composition of the warps before mine
    if (!REV) {
        for (int ww = 0; ww < w; ++ww) { T ga = sm[2 * ww], gb = sm[2 * ww + 1]; pb = ga * pb + gb; pa = ga * pa; }
    } else {
        for (int ww = nw - 1; ww > w; --ww) { T ga = sm[2 * ww], gb = sm[2 * ww + 1]; pb = ga * pb + gb; pa = ga * pa; }
    }
    a = ea * pa;
    b = ea * pb + eb;
    __syncthreads();
}

// chunk of a row owned by this thread in the tridiagonal scans
__device__ __forceinline__ void row_chunk(int n, int &c0, int &c1)
{
    int m = (n + blockDim.x - 1) / blockDim.x;
    c0 = min((int)threadIdx.x * m, n);
    c1 = min(c0 + m, n);
}

// Solve the cyclic zonal system T x = b of one row in place (sb: the row in
// shared memory, length n).  T' = L D L^T with multipliers lf (lf[0] = 0) and
// inverse pivots invD; Sherman-Morrison with the precomputed zz = z / (gam +
// w.z) gives x = y - zz (gam y_0 + ec y_{n-1}).  sm: scan scratch.
template <class T, class F>
__device__ void trisolve_row(T *sb, int n, const F *lf, const F *invD, const F *zz,
                             T gam, T ec, T *sm)
{
    int c0, c1;
    row_chunk(n, c0, c1);
    // forward elimination u_i = b_i - l_i u_{i-1}
    T a = T(1), b = T(0);
    for (int i = c0; i < c1; ++i) { T l = (T)lf[i]; b = sb[i] - l * b; a = -l * a; }
    scan_affine_excl<T, false>(a, b, sm);
    T u = b;
    for (int i = c0; i < c1; ++i) { u = sb[i] - (T)lf[i] * u; sb[i] = u * (T)invD[i]; }
    // back substitution y_i = v_i - l_{i+1} y_{i+1}
    a = T(1); b = T(0);
    for (int i = c1 - 1; i >= c0; --i) { T l = i + 1 < n ? (T)lf[i + 1] : T(0); b = sb[i] - l * b; a = -l * a; }
    scan_affine_excl<T, true>(a, b, sm);
    T y = b;
    for (int i = c1 - 1; i >= c0; --i) { T l = i + 1 < n ? (T)lf[i + 1] : T(0); y = sb[i] - l * y; sb[i] = y; }
    __syncthreads();
    if (zz) {
        T s = gam * sb[0] + ec * sb[n - 1];
        __syncthreads();
        for (int i = c0; i < c1; ++i) sb[i] -= (T)zz[i] * s;
        __syncthreads();
    }
}

} // namespace sw
