// sw_solver.cu -- preconditioned GCR(k) (Sec. 2.3) as one persistent,
// cooperative kernel per solve or ensemble of solves, plus the standalone
// operator and preconditioner kernels behind sw_operator_apply and
// sw_precond_apply.
//
// The GCR iteration is a state machine per member.  Every step of the
// persistent kernel runs one phase for every active member, one latitude row
// per block at a time; after a member's last row of the phase, the block that
// finished it (found with an arrival counter) reduces the member's row
// partial sums in a fixed order and advances its state.  A bounded grid
// barrier separates the steps.  Phases (the text's step numbers in brackets):
//   PH_TRUE  r = L(Phi) - R in FP64 [step 1 / residual check], ||r||^2, first
//            preconditioner stage
//   PH_BETA  Phi += beta p_nu, r += beta L p_nu [step 2], ||r||^2, first
//            preconditioner stage of the new r [step 3]
//   PH_PREC  Richardson stage mu >= 1 (needs neighbour rows) [step 3]
//   PH_LE    L(e) and <L e, L p_l> [step 3]; at a (re)start p_0 = e
//   PH_UPD   p_{nu+1}, L p_{nu+1}, <L p, L p>, <r, L p> [step 4]
//   PH_ZERO  Phi = 0 for a zero right-hand side
#include "sw_rows.cuh"
#include "sw_internal.h"

namespace sw {

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // longest barrier wait (2 s)

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned vload(const unsigned *p) { return *(const volatile unsigned *)p; }
__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }

// Bounded grid barrier (all blocks co-resident: cooperative launch).
// Returns false if the wait ran out or another block gave up.
__device__ bool grid_barrier(GlobalCtl *G, int step)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen0 = vload(&G->gen);
        __threadfence();
        unsigned old = atomicAdd(&G->count, 1u);
        if (old == gridDim.x - 1) {
            atomicExch(&G->count, 0u);
            __threadfence();
            atomicAdd(&G->gen, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            while (vload(&G->gen) == gen0) {
                if (vload(&G->abort)) { ok = 0; break; }
                if (gtimer() - t0 > WAIT_LIMIT_NS) {
                    if (atomicExch(&G->abort, 1) == 0) G->where = step;
                    ok = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        if (vload(&G->abort)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class Pol>
__device__ __forceinline__ const MemberDev<Pol> *mdev(SolverBlock *b) { return (const MemberDev<Pol> *)b->dev; }

__device__ __forceinline__ int phys_slot(const MemberCtl &c, int k, int l) { return (c.base + l) % (k + 1); }

// copy a struct from global memory into shared memory, L2-coherent
template <class T>
__device__ __forceinline__ void copy_in(T *dst, const T *src)
{
    static_assert(sizeof(T) % 4 == 0, "");
    const int *s = (const int *)src;
    int *d = (int *)dst;
    for (int k = threadIdx.x; k < (int)(sizeof(T) / 4); k += blockDim.x) d[k] = ldcg(s + k);
}

// ---------------------------------------------------------------------------
// phases on one row j of member M (state snapshot c)
// ---------------------------------------------------------------------------
template <class Pol>
__device__ void phase_true(const MemberDev<Pol> &M, const MemberCtl &c, double eta, int j, RowSmem<Pol> &sm)
{
    typedef typename Pol::comp comp;
    const int nx = M.nx, ny = M.ny;
    const size_t row = (size_t)j * nx;
    const double *phi = M.phi;
    stage3<double>(sm.s3d, nx, ny, j, [&](int jj, int ii) { return ldcg(phi + (size_t)jj * nx + ii); });
    const double *S = sm.s3d, *X = sm.s3d + nx, *N = sm.s3d + 2 * nx;
    double acc[2] = {0.0, 0.0};
    // the staged rows alias sb's neighbour region only for the FP64 policy's
    // s3c, which is not used here; sb is a separate region
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        double Rv = M.R[row + i];
        double rv = stencil<double, double>(S, X, N, i, nx, j, ny, M.ax, M.cx, M.bx, M.ay, M.cy, M.by, M.C, true) - Rv;
        typename Pol::res rs = (typename Pol::res)rv;
        M.r[row + i] = rs;
        acc[0] += rv * rv;
        acc[1] += Rv * Rv;
        sm.sb[i] = stage0_input(M, eta, (comp)rs, row + i);
    }
    block_sum(acc, 2, sm.red);
    if (threadIdx.x == 0) {
        M.part[(size_t)j * NSLOT + S_RR] = acc[0];
        M.part[(size_t)j * NSLOT + S_R2] = acc[1];
    }
    stage0_finish(M, j, sm);
}

template <class Pol>
__device__ void phase_beta(const MemberDev<Pol> &M, const MemberCtl &c, double eta, int j, RowSmem<Pol> &sm)
{
    typedef typename Pol::comp comp;
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    const size_t N = (size_t)nx * M.ny;
    const int s = phys_slot(c, M.k, c.nu);
    const typename Pol::vec *p = M.p + s * N, *Lp = M.Lp + s * N;
    const double beta = c.beta;
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const size_t id = row + i;
        double pv = (double)ldcg(p + id), lv = (double)ldcg(Lp + id);
        M.phi[id] = ldcg(M.phi + id) + beta * pv;
        typename Pol::res rs = (typename Pol::res)((double)ldcg(M.r + id) + beta * lv);
        M.r[id] = rs;
        acc[0] += (double)rs * (double)rs;
        sm.sb[i] = stage0_input(M, eta, (comp)rs, id);
    }
    block_sum(acc, 1, sm.red);
    if (threadIdx.x == 0) M.part[(size_t)j * NSLOT + S_RR] = acc[0];
    stage0_finish(M, j, sm);
}

template <class Pol>
__device__ void phase_prec(const MemberDev<Pol> &M, const MemberCtl &c, double eta, int j, RowSmem<Pol> &sm)
{
    const int mu = c.stage;     // 1 .. nstages-1
    const bool last = (mu == M.nstages - 1);
    const typename Pol::q16 *ih = (mu & 1) ? M.qa : M.qb;
    const float *if32 = (mu & 1) ? M.qa32 : M.qb32;
    const float *is = (mu & 1) ? M.qa_s : M.qb_s;
    typename Pol::q16 *oh = last ? M.e : ((mu & 1) ? M.qb : M.qa);
    float *of32 = last ? M.e32 : ((mu & 1) ? M.qb32 : M.qa32);
    float *os = last ? M.e_s : ((mu & 1) ? M.qb_s : M.qa_s);
    precond_stage(M, eta, j, sm, ih, if32, is, M.r, oh, of32, os);
}

template <class Pol>
__device__ void phase_le(const MemberDev<Pol> &M, const MemberCtl &c, int j, RowSmem<Pol> &sm)
{
    typedef typename Pol::comp comp;
    typedef typename Pol::vec vec;
    const int nx = M.nx, ny = M.ny;
    const size_t row = (size_t)j * nx;
    const size_t N = (size_t)nx * ny;
    stage3_q(sm.s3c, M, M.e, M.e32, M.e_s, j);
    const comp *S = sm.s3c, *X = sm.s3c + nx, *Nn = sm.s3c + 2 * nx;
    double acc[KMAX + 1];
    if (c.start) {
        const int s0 = phys_slot(c, M.k, 0);
        vec *p = M.p + s0 * N, *Lp = M.Lp + s0 * N;
        acc[0] = acc[1] = 0.0;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            comp le = stencil<comp, typename Pol::coef>(S, X, Nn, i, nx, j, ny, M.wax, M.wcx, M.wbx, M.way,
                                                        M.wcy, M.wby, M.wC, true);
            vec lv = (vec)le;
            p[row + i] = (vec)X[i];
            Lp[row + i] = lv;
            acc[0] += (double)lv * (double)lv;
            acc[1] += (double)ldcg(M.r + row + i) * (double)lv;
        }
        block_sum(acc, 2, sm.red);
        if (threadIdx.x == 0) {
            M.part[(size_t)j * NSLOT + S_LPLP] = acc[0];
            M.part[(size_t)j * NSLOT + S_RLP] = acc[1];
        }
    } else {
        const int nd = c.nu + 1;
        for (int l = 0; l < nd; ++l) acc[l] = 0.0;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            comp le = stencil<comp, typename Pol::coef>(S, X, Nn, i, nx, j, ny, M.wax, M.wcx, M.wbx, M.way,
                                                        M.wcy, M.wby, M.wC, true);
            vec lv = (vec)le;
            M.Le[row + i] = lv;
            for (int l = 0; l < nd; ++l) {
                const vec *Lpl = M.Lp + phys_slot(c, M.k, l) * N;
                acc[l] += (double)lv * (double)ldcg(Lpl + row + i);
            }
        }
        block_sum(acc, nd, sm.red);
        if (threadIdx.x == 0)
            for (int l = 0; l < nd; ++l) M.part[(size_t)j * NSLOT + S_DOT0 + l] = acc[l];
    }
    __syncthreads();
}

template <class Pol>
__device__ void phase_upd(const MemberDev<Pol> &M, const MemberCtl &c, int j, RowSmem<Pol> &sm)
{
    typedef typename Pol::comp comp;
    typedef typename Pol::vec vec;
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    const size_t N = (size_t)nx * M.ny;
    const int nd = c.nu + 1;
    const int sn = phys_slot(c, M.k, nd);
    vec *pn = M.p + sn * N, *Lpn = M.Lp + sn * N;
    const float esc = q_scale(M, M.e_s, j);
    double acc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const size_t id = row + i;
        comp pv = q_load(M, M.e, M.e32, esc, j, i);
        comp lv = (comp)ldcg(M.Le + id);
        for (int l = 0; l < nd; ++l) {
            const size_t off = phys_slot(c, M.k, l) * N + id;
            comp a = (comp)c.alpha[l];
            pv += a * (comp)ldcg(M.p + off);
            lv += a * (comp)ldcg(M.Lp + off);
        }
        vec ps = (vec)pv, ls = (vec)lv;
        pn[id] = ps;
        Lpn[id] = ls;
        acc[0] += (double)ls * (double)ls;
        acc[1] += (double)ldcg(M.r + id) * (double)ls;
    }
    block_sum(acc, 2, sm.red);
    if (threadIdx.x == 0) {
        M.part[(size_t)j * NSLOT + S_LPLP] = acc[0];
        M.part[(size_t)j * NSLOT + S_RLP] = acc[1];
    }
}

template <class Pol>
__device__ void phase_zero(const MemberDev<Pol> &M, int j)
{
    const size_t row = (size_t)j * M.nx;
    for (int i = threadIdx.x; i < M.nx; i += blockDim.x) M.phi[row + i] = 0.0;
    if (threadIdx.x == 0) M.part[(size_t)j * NSLOT + S_RR] = 0.0;
}

// ---------------------------------------------------------------------------
// serial section of one member: reduce its row partials (fixed order) and
// advance its state.  Run by the block that finished the member's last row.
// ---------------------------------------------------------------------------
template <class Pol>
__device__ void member_serial(SolverBlock *B, const MemberDev<Pol> &M, MemberCtl &c, RowSmem<Pol> &sm)
{
    int s0 = 0, ns = 0;
    switch (c.phase) {
    case PH_TRUE: s0 = S_RR; ns = c.init ? 2 : 1; break;
    case PH_BETA: s0 = S_RR; ns = 1; break;
    case PH_LE: if (c.start) { s0 = S_LPLP; ns = 2; } else { s0 = S_DOT0; ns = c.nu + 1; } break;
    case PH_UPD: s0 = S_LPLP; ns = 2; break;
    default: break;
    }
    double acc[KMAX + 1];
    for (int s = 0; s < ns; ++s) acc[s] = 0.0;
    for (int r = threadIdx.x; r < M.ny; r += blockDim.x)
        for (int s = 0; s < ns; ++s) acc[s] += ldcg(M.part + (size_t)r * NSLOT + s0 + s);
    if (ns > 0) block_sum(acc, ns, sm.red);
    __shared__ int s_rowres;
    if (threadIdx.x == 0) {
        const int k = M.k;
        bool done = false;
        int ph = c.phase;
        auto to_precond = [&]() { c.stage = 1; c.phase = (M.nstages > 1) ? PH_PREC : PH_LE; };
        auto finish = [&](int st) { c.status = st; done = true; };
        switch (ph) {
        case PH_TRUE: {
            double rn = sqrt(acc[0]);
            if (c.init) {
                c.init = 0;
                c.nR = sqrt(acc[1]);
                c.r0 = rn;
                c.rn_true = c.rn_rec = rn;
                if (M.hist) M.hist[0] = c.nR > 0.0 ? rn / c.nR : 0.0;
                if (c.nR == 0.0) { c.phase = PH_ZERO; break; }
                if (!isfinite(rn) || !isfinite(c.nR)) { finish(ST_NONFINITE); break; }
                if (rn <= M.tol * c.nR && M.min_iters <= 0) { finish(ST_OK); break; }
                c.start = 1;
                to_precond();
            } else {
                c.rn_true = rn;
                if (M.hist) M.hist[c.it] = rn / c.nR;
                if (!isfinite(rn)) { finish(ST_NONFINITE); break; }
                if (rn <= M.tol * c.nR && c.it >= M.min_iters) { finish(ST_OK); break; }
                if (c.it >= M.max_iters) { finish(ST_NOT_CONVERGED); break; }
                to_precond();
            }
            break;
        }
        case PH_PREC:
            c.stage += 1;
            if (c.stage >= M.nstages) c.phase = PH_LE;
            break;
        case PH_LE:
            if (c.start) {
                double lplp = acc[0], rlp = acc[1];
                if (!(lplp > 0.0) || !isfinite(lplp)) { finish(ST_BREAKDOWN); break; }
                c.LpLp[phys_slot(c, k, 0)] = lplp;
                c.beta = -rlp / lplp;
                c.start = 0;
                c.nu = 0;
                c.phase = PH_BETA;
            } else {
                for (int l = 0; l <= c.nu; ++l) c.alpha[l] = -acc[l] / c.LpLp[phys_slot(c, k, l)];
                c.phase = PH_UPD;
            }
            break;
        case PH_UPD: {
            double lplp = acc[0], rlp = acc[1];
            if (!(lplp > 0.0) || !isfinite(lplp)) { finish(ST_BREAKDOWN); break; }
            c.LpLp[phys_slot(c, k, c.nu + 1)] = lplp;
            c.beta = -rlp / lplp;
            c.nu += 1;
            if (c.nu == k) { c.base = phys_slot(c, k, k); c.nu = 0; }
            c.phase = PH_BETA;
            break;
        }
        case PH_BETA: {
            c.it += 1;
            double rn = sqrt(acc[0]);
            c.rn_rec = rn;
            if (M.hist) M.hist[c.it] = rn / c.nR;
            if (!isfinite(rn)) { finish(ST_NONFINITE); break; }
            if ((rn <= M.tol * c.nR && c.it >= M.min_iters) || (M.ru_every > 0 && c.it % M.ru_every == 0) ||
                c.it >= M.max_iters)
                c.phase = PH_TRUE;
            else
                to_precond();
            break;
        }
        case PH_ZERO:
            c.rn_true = c.rn_rec = 0.0;
            finish(ST_OK);
            break;
        default: break;
        }
        s_rowres = (done && (ph == PH_TRUE || ph == PH_ZERO) && M.rowres) ? 1 : 0;
        if (done) c.phase = PH_DONE;
        // publish the new state
        MemberCtl *g = &B->ctl;
        c.arrive = 0;
        const int *src = (const int *)&c;
        int *dst = (int *)g;
        for (int w = 0; w < (int)(sizeof(MemberCtl) / 4); ++w) dst[w] = src[w];
        __threadfence();
    }
    __syncthreads();
    if (s_rowres)
        for (int r = threadIdx.x; r < M.ny; r += blockDim.x)
            M.rowres[r] = sqrt(ldcg(M.part + (size_t)r * NSLOT + S_RR));
    __syncthreads();
}

template <class Pol>
__device__ __forceinline__ double member_eta(const MemberDev<Pol> &M) { return ldcg(M.etap); }

// ---------------------------------------------------------------------------
// the persistent GCR kernel
// ---------------------------------------------------------------------------
template <class Pol>
__global__ void __launch_bounds__(MAX_THREADS) k_gcr(EnsembleParams P, int max_nx)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int s_off[MAX_MEMBERS + 1];
    __shared__ MemberDev<Pol> s_M;
    __shared__ MemberCtl s_c;
    __shared__ int s_last;
    RowSmem<Pol> sm = carve_smem<Pol>(dsm, max_nx);
    GlobalCtl *G = &P.blk[0]->g;
    const int n = P.n;
    const int lane = threadIdx.x & 31;

    for (int step = 0;; ++step) {
        // enumerate the rows of the active members
        if (threadIdx.x < 32) {
            int carry = 0;
            for (int base = 0; base < n; base += 32) {
                int m = base + lane, rows = 0;
                if (m < n) {
                    SolverBlock *b = P.blk[m];
                    if (ldcg(&b->ctl.phase) < PH_DONE) rows = mdev<Pol>(b)->ny;
                }
                int v = rows;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    int o = __shfl_up_sync(0xffffffffu, v, d);
                    if (lane >= d) v += o;
                }
                if (m < n) s_off[m + 1] = carry + v;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            if (lane == 0) s_off[0] = 0;
        }
        __syncthreads();
        const int total = s_off[n];
        if (total == 0) break;
        const int per = (total + gridDim.x - 1) / gridDim.x;
        const int lo = min((int)blockIdx.x * per, total), hi = min(lo + per, total);

        int m = -1, cnt = 0;
        for (int item = lo; item < hi; ++item) {
            if (m < 0 || item >= s_off[m + 1]) {
                if (m >= 0) {
                    // hand over: count my rows of member m
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        __threadfence();
                        int old = atomicAdd(&P.blk[m]->ctl.arrive, cnt);
                        s_last = (old + cnt == s_M.ny);
                    }
                    __syncthreads();
                    if (s_last) { __threadfence(); member_serial<Pol>(P.blk[m], s_M, s_c, sm); }
                }
                int mm = (m < 0) ? 0 : m + 1;
                while (item >= s_off[mm + 1]) ++mm;
                m = mm;
                cnt = 0;
                __syncthreads();
                copy_in(&s_M, mdev<Pol>(P.blk[m]));
                copy_in(&s_c, &P.blk[m]->ctl);
                __syncthreads();
            }
            const int j = item - s_off[m];
            const double eta = member_eta(s_M);
            switch (s_c.phase) {
            case PH_TRUE: phase_true<Pol>(s_M, s_c, eta, j, sm); break;
            case PH_BETA: phase_beta<Pol>(s_M, s_c, eta, j, sm); break;
            case PH_PREC: phase_prec<Pol>(s_M, s_c, eta, j, sm); break;
            case PH_LE: phase_le<Pol>(s_M, s_c, j, sm); break;
            case PH_UPD: phase_upd<Pol>(s_M, s_c, j, sm); break;
            case PH_ZERO: phase_zero<Pol>(s_M, j); break;
            default: break;
            }
            ++cnt;
        }
        if (m >= 0) {
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                int old = atomicAdd(&P.blk[m]->ctl.arrive, cnt);
                s_last = (old + cnt == s_M.ny);
            }
            __syncthreads();
            if (s_last) { __threadfence(); member_serial<Pol>(P.blk[m], s_M, s_c, sm); }
        }
        if (!grid_barrier(G, step)) return;
    }
}

// ---------------------------------------------------------------------------
// standalone kernels: one block per row
// ---------------------------------------------------------------------------
template <class T, class CT>
__global__ void __launch_bounds__(MAX_THREADS) k_operator(OpArgs<CT> a, const T *x, T *y)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    T *s3 = (T *)dsm;
    const int nx = a.nx, ny = a.ny, j = blockIdx.x;
    stage3<T>(s3, nx, ny, j, [&](int jj, int ii) { return x[(size_t)jj * nx + ii]; });
    for (int i = threadIdx.x; i < nx; i += blockDim.x)
        y[(size_t)j * nx + i] = stencil<T, CT>(s3, s3 + nx, s3 + 2 * nx, i, nx, j, ny, a.ax, a.cx, a.bx,
                                                a.ay, a.cy, a.by, a.C, true);
}

// first preconditioner stage from a residual r (type RT)
template <class Pol, class RT>
__global__ void __launch_bounds__(MAX_THREADS) k_precond_first(const MemberDev<Pol> *Mp, const RT *r)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ MemberDev<Pol> s_M;
    copy_in(&s_M, Mp);
    __syncthreads();
    RowSmem<Pol> sm = carve_smem<Pol>(dsm, s_M.nx);
    const int j = blockIdx.x;
    const size_t row = (size_t)j * s_M.nx;
    for (int i = threadIdx.x; i < s_M.nx; i += blockDim.x)
        sm.sb[i] = stage0_input(s_M, ldcg(s_M.etap), (typename Pol::comp)r[row + i], row + i);
    stage0_finish(s_M, j, sm);
}

template <class Pol, class RT>
__global__ void __launch_bounds__(MAX_THREADS) k_precond_stage(const MemberDev<Pol> *Mp, const RT *r, int mu)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ MemberDev<Pol> s_M;
    copy_in(&s_M, Mp);
    __syncthreads();
    RowSmem<Pol> sm = carve_smem<Pol>(dsm, s_M.nx);
    const MemberDev<Pol> &M = s_M;
    const bool last = (mu == M.nstages - 1);
    const typename Pol::q16 *ih = (mu & 1) ? M.qa : M.qb;
    const float *if32 = (mu & 1) ? M.qa32 : M.qb32;
    const float *is = (mu & 1) ? M.qa_s : M.qb_s;
    typename Pol::q16 *oh = last ? M.e : ((mu & 1) ? M.qb : M.qa);
    float *of32 = last ? M.e32 : ((mu & 1) ? M.qb32 : M.qa32);
    float *os = last ? M.e_s : ((mu & 1) ? M.qb_s : M.qa_s);
    precond_stage(M, ldcg(M.etap), (int)blockIdx.x, sm, ih, if32, is, r, oh, of32, os);
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

__global__ void k_fill(double *p, size_t n, double v)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------------------------
// host-side launchers (declared in sw_internal.h)
// ---------------------------------------------------------------------------
template <class Pol>
static cudaError_t launch_gcr_t(const EnsembleParams &P, int max_nx, int threads, int sms, int total_rows,
                                cudaStream_t s, int *grid_used)
{
    size_t smem = row_smem_bytes<Pol>(max_nx, threads);
    cudaError_t e = cudaFuncSetAttribute(k_gcr<Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gcr<Pol>, threads, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    int grid = nb * sms;
    if (grid > total_rows) grid = total_rows;
    if (grid < 1) grid = 1;
    *grid_used = grid;
    EnsembleParams Pc = P;
    int mx = max_nx;
    void *args[] = {(void *)&Pc, (void *)&mx};
    return cudaLaunchCooperativeKernel((const void *)k_gcr<Pol>, dim3(grid), dim3(threads), args, smem, s);
}

cudaError_t launch_gcr(int prec, const EnsembleParams &P, int max_nx, int threads, int sms, int total_rows,
                       cudaStream_t s, int *grid_used)
{
    switch (prec) {
    case 0: return launch_gcr_t<PolFP64>(P, max_nx, threads, sms, total_rows, s, grid_used);
    case 1: return launch_gcr_t<PolF16>(P, max_nx, threads, sms, total_rows, s, grid_used);
    case 2: return launch_gcr_t<PolBF16>(P, max_nx, threads, sms, total_rows, s, grid_used);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_operator_f64(const OpArgs<double> &a, const double *x, double *y, int threads, cudaStream_t s)
{
    size_t smem = 3 * (size_t)a.nx * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_operator<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_operator<double, double><<<a.ny, threads, smem, s>>>(a, x, y);
    return cudaGetLastError();
}

cudaError_t launch_operator_f32(const OpArgs<float> &a, const float *x, float *y, int threads, cudaStream_t s)
{
    size_t smem = 3 * (size_t)a.nx * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_operator<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_operator<float, float><<<a.ny, threads, smem, s>>>(a, x, y);
    return cudaGetLastError();
}

template <class Pol, class RT>
static cudaError_t launch_precond_t(const void *Mdev, int nx, int ny, int nstages, const RT *r, float *qout,
                                    int threads, cudaStream_t s)
{
    const MemberDev<Pol> *M = (const MemberDev<Pol> *)Mdev;
    size_t smem = row_smem_bytes<Pol>(nx, threads);
    cudaError_t e = cudaFuncSetAttribute(k_precond_first<Pol, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_precond_stage<Pol, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_precond_first<Pol, RT><<<ny, threads, smem, s>>>(M, r);
    for (int mu = 1; mu < nstages; ++mu) k_precond_stage<Pol, RT><<<ny, threads, smem, s>>>(M, r, mu);
    if (qout) k_unpack_e<Pol><<<ny, threads, 0, s>>>(M, qout);
    return cudaGetLastError();
}

cudaError_t launch_precond(int prec, const void *Mdev, int nx, int ny, int nstages, const void *r, void *qout,
                           int threads, cudaStream_t s)
{
    switch (prec) {
    case 0: return launch_precond_t<PolFP64, double>(Mdev, nx, ny, nstages, (const double *)r, nullptr, threads, s);
    case 1: return launch_precond_t<PolF16, float>(Mdev, nx, ny, nstages, (const float *)r, (float *)qout, threads, s);
    case 2: return launch_precond_t<PolBF16, float>(Mdev, nx, ny, nstages, (const float *)r, (float *)qout, threads, s);
    default: return cudaErrorInvalidValue;
    }
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
