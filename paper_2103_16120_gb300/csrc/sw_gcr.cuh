// sw_gcr.cuh -- preconditioned GCR(k) (Sec. 2.3) as one persistent,
// cooperative kernel per solve or ensemble of solves.  The kernel template is
// instantiated in one translation unit per precision policy and row mode
// (sw_gcr_*.cu), which nvcc compiles in parallel.
//
// Layout of the work.  Each member (one elliptic problem) owns a group of
// thread blocks for the whole solve; each block owns latitude rows (one row
// when the member's rows fit the co-resident blocks), so the row's face
// coefficients, zonal factors and owner-only vectors (r, L e, p_l, L p_l) can
// stay in shared memory between phases.  Only what other rows read (the
// preconditioner fields q and e, and Phi) goes through global memory, and the
// rows a block needs from there are copied in with one round trip per phase.
//
// The GCR iteration is a state machine whose state every block of the member
// holds in shared memory.  After each phase the block sums its rows' partial
// sums in a fixed order and publishes them; the member's blocks meet at a
// bounded barrier (a monotonic counter with release/acquire semantics); every
// block then adds the published block sums in the same fixed order and applies
// the same transition, so all copies of the state agree.
//
// Phases (the text's algorithmic steps in brackets):
//   PH_TRUE  r = L(Phi) - R in FP64 [step 1 / final check], ||r||^2, and the
//            first preconditioner stage of r
//   PH_PREC  Richardson stage mu >= 1, which needs neighbour rows [step 3]
//   PH_LE    L(e) and the inner products <Le,Le>, <r,Le>, <Le,Lp_l>,
//            <r,Lp_l> [steps 3-4]
//   PH_UB    p_{nu+1} = e + sum alpha_l p_l, Lp_{nu+1} = Le + sum alpha_l Lp_l
//            [step 4], Phi += beta p_{nu+1}, r += beta Lp_{nu+1} [step 2],
//            ||r||^2, <Lp_{nu+1}, Lp_m>, and the first preconditioner stage of
//            the new r [step 3]
// The coefficients alpha_l = -<Le,Lp_l>/<Lp_l,Lp_l> are those of the text;
// beta = -<r,Lp_{nu+1}>/<Lp_{nu+1},Lp_{nu+1}> is evaluated before Lp_{nu+1}
// exists, from the PH_LE inner products and the Gram matrix of the cycle's
// directions (the same value, a different rounding), so the update and the
// step share one pass: three phases per iteration.
#pragma once

#include "sw_split.cuh"
#include "sw_internal.h"

namespace sw {

// longest barrier wait (default 2 s) and arrivals a barrier expects beyond
// the member's blocks (default 0); sw_debug_barrier changes both, so that a
// test can make the wait run out
static __device__ unsigned long long g_wait_limit_ns = 2000000000ull;
static __device__ unsigned long long g_extra_arrivals = 0;

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }

// 1/x for the GCR scalars: a reciprocal approximation refined by two
// Newton-Raphson steps r <- r + r (1 - x r), each of which doubles the number
// of correct bits, so the result agrees with the quotient to about an ulp.
// An FP64 division costs about 600 cycles on this GPU, this about 300.
// Outside a safe exponent range, and for zero, infinities and NaN, it is the
// quotient itself.
__device__ __forceinline__ double recip(double x)
{
    const int ex = (__double2hiint(x) >> 20) & 0x7ff;      // biased exponent
    if (ex < 1023 - 500 || ex > 1023 + 500) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

template <class Pol>
__device__ __forceinline__ const MemberDev<Pol> *mdev(SolverBlock *b) { return (const MemberDev<Pol> *)b->dev; }


// copy a struct from global memory into shared memory, L2-coherent
template <class T>
__device__ __forceinline__ void copy_in(T *dst, const T *src)
{
    static_assert(sizeof(T) % 4 == 0, "");
    const int *s = (const int *)src;
    int *d = (int *)dst;
    for (int k = threadIdx.x; k < (int)(sizeof(T) / 4); k += blockDim.x) d[k] = __ldcg(s + k);
}

// partial-sum slots of each phase (see NSLOT)
__device__ __forceinline__ int phase_slots(int phase, int nd, int *slot)
{
    int ns = 0;
    switch (phase) {
    case PH_TRUE: case PH_ZERO: slot[0] = S_A; slot[1] = S_B; ns = 2; break;
    case PH_UB:
        slot[0] = S_A; slot[1] = S_B; ns = 2;
        for (int l = 0; l < nd; ++l) slot[ns++] = S_C0 + l;
        break;
    case PH_LE:
        slot[0] = S_A; slot[1] = S_B; ns = 2;
        for (int l = 0; l < nd; ++l) slot[ns++] = S_C0 + l;
        for (int l = 0; l < nd; ++l) slot[ns++] = S_T0 + l;
        break;
    default: break;
    }
    return ns;
}

// ---------------------------------------------------------------------------
// phases on one row j (one block).  Each thread adds its share of the phase's
// inner products to part[slot]; the caller sums them over the block.
// ---------------------------------------------------------------------------
template <class Pol, int NP>
__device__ void phase_true(const MemberDev<Pol> &M, const RowView<Pol> &v, typename Pol::comp eta, int j,
                           unsigned char *ws, typename Acc<Pol>::type (&part)[NP])
{
    typedef typename Pol::comp comp;
    const int nx = M.nx, ny = M.ny;
    const size_t row = (size_t)j * nx;
    comp *sb = (comp *)(ws + sb_offset<Pol>(nx));
    // FP64 coefficients: the policy's own (FP64 policy) or the FP64 copies
    RowCoef<double> c;
    if constexpr (Pol::kMixed) {
        const size_t rs = j > 0 ? row - nx : row;
        c = {M.ax + row, M.cx + row, M.bx + row, M.ay + row, M.cy + row, M.by + row,
             M.ay + rs, M.cy + rs, M.by + rs, M.C + row};
    } else {
        c = coef_of(v);
    }
    // the three Phi rows (FP64), unshifted, into the stage + raw region
    double *ph = (double *)ws;
    int src[3], sh[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ghost_row(j - 1 + r, nx, ny, src[r], sh[r]);
        row_copy_issue(ph + (size_t)r * nx, M.phi + (size_t)src[r] * nx, nx * 8);
    }
    row_copy_wait();
    const double *pS = ph, *pX = ph + nx, *pN = ph + 2 * nx;
    auto wrap = [&](int i) { return i >= nx ? i - nx : i; };
    const bool has_n = j < ny - 1, has_s = j > 0;
    double rr = 0.0, RR = 0.0;
    // rows away from the poles (no shifted neighbour row): 4 consecutive points
    // per thread, each zonal face flux formed once for its two points (the same
    // expressions as below, so L(Phi) is unchanged)
    const bool v4 = sh[0] == 0 && sh[2] == 0 && stencil4_ok(c, nx) && al16p(ph) && al16p(M.R + row);
    if (v4) {
        for (int i0 = 4 * threadIdx.x; i0 < nx; i0 += 4 * blockDim.x) {
            double xc[6], xn[6], xs[6];
            ldw6(pX, i0, nx, xc);
            ldw6(pN, i0, nx, xn);
            ldw6(pS, i0, nx, xs);
            const int iw = i0 == 0 ? nx - 1 : i0 - 1;
            double ax[5], cx[5], bx[5], q[4];
            ax[0] = c.ax[iw]; cx[0] = c.cx[iw]; bx[0] = c.bx[iw];
            ldv4(c.ax + i0, q); for (int k = 0; k < 4; ++k) ax[k + 1] = q[k];
            ldv4(c.cx + i0, q); for (int k = 0; k < 4; ++k) cx[k + 1] = q[k];
            ldv4(c.bx + i0, q); for (int k = 0; k < 4; ++k) bx[k + 1] = q[k];
            double cc[4], Rv[4];
            ldv4(c.C + i0, cc);
            ldv4(M.R + row + i0, Rv);
            double ay[4] = {}, cy[4] = {}, by[4] = {}, ays[4] = {}, cys[4] = {}, bys[4] = {};
            if (has_n) { ldv4(c.ay + i0, ay); ldv4(c.cy + i0, cy); ldv4(c.by + i0, by); }
            if (has_s) { ldv4(c.ays + i0, ays); ldv4(c.cys + i0, cys); ldv4(c.bys + i0, bys); }
            // face m: east face of window point m (window k = longitude i0 - 1 + k)
            double F[5];
#pragma unroll
            for (int m = 0; m < 5; ++m)
                F[m] = cx[m] * (xn[m] + xn[m + 1] - xs[m] - xs[m + 1]) + bx[m] * (xc[m] + xc[m + 1]) +
                       ax[m] * (xc[m + 1] - xc[m]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = u + 1, i = i0 + u;
                double lphi = F[u + 1] - F[u];
                if (has_n) lphi += ay[u] * (xn[k] - xc[k]) + cy[u] * (xc[k + 1] + xn[k + 1] - xc[k - 1] - xn[k - 1]) +
                                   by[u] * (xc[k] + xn[k]);
                if (has_s) lphi -= ays[u] * (xc[k] - xs[k]) + cys[u] * (xs[k + 1] + xc[k + 1] - xs[k - 1] - xc[k - 1]) +
                                   bys[u] * (xs[k] + xc[k]);
                lphi -= cc[u] * xc[k];
                const double rv = lphi - Rv[u];
                const typename Pol::res rs = (typename Pol::res)rv;
                v.r[i] = rs;
                rr += rv * rv;
                RR += Rv[u] * Rv[u];
                sb[pidx(i)] = stage0_input(M, v, eta, (comp)rs, i);
            }
        }
    }
    constexpr int U = 2;
    for (int i0 = v4 ? nx : (int)threadIdx.x; i0 < nx; i0 += U * blockDim.x) {
        double cx[U], cxw[U], bx[U], bxw[U], ax[U], axw[U], ay[U], cy[U], by[U], ays[U], cys[U], bys[U], cc[U], Rv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = min(i0 + u * (int)blockDim.x, nx - 1), iw = (i == 0) ? nx - 1 : i - 1;
            cx[u] = c.cx[i]; cxw[u] = c.cx[iw]; bx[u] = c.bx[i]; bxw[u] = c.bx[iw];
            ax[u] = c.ax[i]; axw[u] = c.ax[iw]; cc[u] = c.C[i];
            ay[u] = has_n ? c.ay[i] : 0.0; cy[u] = has_n ? c.cy[i] : 0.0; by[u] = has_n ? c.by[i] : 0.0;
            ays[u] = has_s ? c.ays[i] : 0.0; cys[u] = has_s ? c.cys[i] : 0.0; bys[u] = has_s ? c.bys[i] : 0.0;
            Rv[u] = __ldg(M.R + row + i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= nx) break;
            const int ie = wrap(i + 1), iw = (i == 0) ? nx - 1 : i - 1;
            const double xc = pX[i], xe = pX[ie], xw = pX[iw];
            const double xn = pN[wrap(i + sh[2])], xne = pN[wrap(ie + sh[2])], xnw = pN[wrap(iw + sh[2])];
            const double xs = pS[wrap(i + sh[0])], xse = pS[wrap(ie + sh[0])], xsw = pS[wrap(iw + sh[0])];
            double fe = cx[u] * (xn + xne - xs - xse) + bx[u] * (xc + xe) + ax[u] * (xe - xc);
            double fw = cxw[u] * (xnw + xn - xsw - xs) + bxw[u] * (xw + xc) + axw[u] * (xc - xw);
            double lphi = fe - fw;
            if (has_n) lphi += ay[u] * (xn - xc) + cy[u] * (xe + xne - xw - xnw) + by[u] * (xc + xn);
            if (has_s) lphi -= ays[u] * (xc - xs) + cys[u] * (xse + xe - xsw - xw) + bys[u] * (xs + xc);
            lphi -= cc[u] * xc;
            const double rv = lphi - Rv[u];
            const typename Pol::res rs = (typename Pol::res)rv;
            v.r[i] = rs;
            rr += rv * rv;
            RR += Rv[u] * Rv[u];
            sb[pidx(i)] = stage0_input(M, v, eta, (comp)rs, i);
        }
    }
    part[0] += (typename Acc<Pol>::type)rr;
    part[1] += (typename Acc<Pol>::type)RR;
    stage0_finish(M, v, j, ws);
}

template <class Pol, int KM>
__device__ void phase_le(const MemberDev<Pol> &M, const MemberCtl &c, const RowView<Pol> &v, int j,
                         unsigned char *ws, typename Acc<Pol>::type (&part)[2 + 2 * KM])
{
    typedef typename Pol::comp comp;
    typedef typename Pol::vec vec;
    typedef typename Acc<Pol>::type acc_t;
    const int nx = M.nx, ny = M.ny;
    const int nd = c.nu + 1;
    stage3_q(ws, M, M.e, M.e32, M.e_s, j);
    SW_TRACE(101);
    const comp *stg = (const comp *)ws;
    // L e of the row, straight into the row's L e storage
    if (stencil4_ok(coef_of(v), nx) && ((uintptr_t)v.Le & 15) == 0)
        stencil_row4<comp, typename Pol::coef>(stg, stg + nx, stg + 2 * nx, nx, j, ny, coef_of(v), true, (comp *)v.Le,
                                               false);
    else
        stencil_row<comp, typename Pol::coef>(stg, stg + nx, stg + 2 * nx, nx, j, ny, coef_of(v), true, (comp *)v.Le,
                                              false);
    SW_TRACE(102);
    const vec *Lpl[KM];
#pragma unroll
    for (int l = 0; l < KM; ++l) Lpl[l] = v.Lpb + (size_t)phys_slot(c, M.k, l < nd ? l : 0) * v.vstride;
    // mixed policies: 4 consecutive points per thread, vector reads
    bool v4 = Pol::kMixed && (nx & 3) == 0 && al16p(v.Le) && al16p(v.r);
#pragma unroll
    for (int l = 0; l < KM; ++l) v4 = v4 && al16p(Lpl[l]);
    if (v4) {
        for (int i0 = 4 * threadIdx.x; i0 < nx; i0 += 4 * blockDim.x) {
            vec le4[4], lp4[KM][4];
            typename Pol::res r4[4];
            ldv4(v.Le + i0, le4);
            ldv4(v.r + i0, r4);
#pragma unroll
            for (int l = 0; l < KM; ++l)
                if (l < nd) ldv4(Lpl[l] + i0, lp4[l]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const acc_t la = (acc_t)le4[u], rv = (acc_t)r4[u];
                part[0] += la * la;
                part[1] += rv * la;
#pragma unroll
                for (int l = 0; l < KM; ++l) {
                    if (l < nd) {
                        part[2 + l] += la * (acc_t)lp4[l][u];
                        part[2 + KM + l] += rv * (acc_t)lp4[l][u];
                    }
                }
            }
        }
        return;
    }
    constexpr int U = batch_of<comp>();
    for (int i0 = threadIdx.x; i0 < nx; i0 += U * blockDim.x) {
        acc_t la[U], rv[U], lp[KM][U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = min(i0 + u * (int)blockDim.x, nx - 1);
            la[u] = (acc_t)v.Le[i];
            rv[u] = (acc_t)v.r[i];
#pragma unroll
            for (int l = 0; l < KM; ++l) lp[l][u] = l < nd ? (acc_t)Lpl[l][i] : acc_t(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * (int)blockDim.x >= nx) break;
            part[0] += la[u] * la[u];
            part[1] += rv[u] * la[u];
#pragma unroll
            for (int l = 0; l < KM; ++l) {
                if (l < nd) {
                    part[2 + l] += la[u] * lp[l][u];
                    part[2 + KM + l] += rv[u] * lp[l][u];
                }
            }
        }
    }
}

template <class Pol, int KM>
__device__ void phase_ub(const MemberDev<Pol> &M, const MemberCtl &c, const RowView<Pol> &v,
                         typename Pol::comp eta, int j, unsigned char *ws, typename Acc<Pol>::type (&part)[2 + 2 * KM])
{
    typedef typename Pol::comp comp;
    typedef typename Pol::vec vec;
    typedef typename Acc<Pol>::type acc_t;
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    const int nd = c.nu + 1;                      // directions before the new one
    comp *sb = (comp *)(ws + sb_offset<Pol>(nx));
    // the row of Phi, copied while the direction pointers are set up
    double *phr = (double *)ws;
    row_copy_issue(phr, M.phi + row, nx * 8);
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
    const float esc = q_scale(M, M.e_s, j);
    const double beta = c.beta;
    const comp beta_c = (comp)beta;
    row_copy_wait();
    // mixed policies: 4 consecutive points per thread, vector reads and
    // writes (the FP64 policy keeps the strided loop: the vector form spills
    // registers in the two-blocks-per-SM instantiation)
    bool v4 = Pol::kMixed && (nx & 3) == 0 && al16p(v.Le) && al16p(v.r) && al16p(pn) && al16p(Lpn) &&
              al16p(M.phi + row) && (!v.el || al16p(v.el));
#pragma unroll
    for (int l = 0; l < KM; ++l) v4 = v4 && al16p(pl[l]) && al16p(Lpl[l]);
    if (v4) {
        for (int i0 = 4 * threadIdx.x; i0 < nx; i0 += 4 * blockDim.x) {
            comp ev[4];
            vec le4[4], pv4[KM][4], lp4[KM][4];
            typename Pol::res r4[4];
            double ph4[4];
            if (v.el) {
                ldv4(v.el + i0, ev);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) ev[u] = q_load(M, M.e, M.e32, esc, j, i0 + u);
            }
            ldv4(v.Le + i0, le4);
            ldv4(v.r + i0, r4);
            ldv4(phr + i0, ph4);
#pragma unroll
            for (int l = 0; l < KM; ++l) {
                if (l < nd) {
                    ldv4(pl[l] + i0, pv4[l]);
                    ldv4(Lpl[l] + i0, lp4[l]);
                }
            }
            vec ps4[4], ls4[4];
            typename Pol::res rs4[4];
            double phn[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                comp pv = ev[u], lw = (comp)le4[u];
#pragma unroll
                for (int l = 0; l < KM; ++l) {
                    if (l < nd) {
                        pv += al[l] * (comp)pv4[l][u];
                        lw += al[l] * (comp)lp4[l][u];
                    }
                }
                ps4[u] = (vec)pv;
                ls4[u] = (vec)lw;
                phn[u] = ph4[u] + beta * (double)ps4[u];
                if constexpr (Pol::kMixed) rs4[u] = (typename Pol::res)((comp)r4[u] + beta_c * ls4[u]);
                else rs4[u] = (comp)r4[u] + beta * ls4[u];
                const acc_t ra = (acc_t)rs4[u], la = (acc_t)ls4[u];
                part[0] += ra * ra;
                part[1] += la * la;
#pragma unroll
                for (int l = 0; l < KM; ++l)
                    if (l < nd) part[2 + l] += la * (acc_t)lp4[l][u];
                sb[pidx(i0 + u)] = stage0_input(M, v, eta, (comp)rs4[u], i0 + u);
            }
            stv4(pn + i0, ps4);
            stv4(Lpn + i0, ls4);
            stv4(M.phi + row + i0, phn);
            stv4(v.r + i0, rs4);
        }
        SW_TRACE(201);
        stage0_finish(M, v, j, ws);
        return;
    }
    constexpr int U = batch_of<comp>();
    for (int i0 = threadIdx.x; i0 < nx; i0 += U * blockDim.x) {
        // loads of the batch: e, L e, r, p_l, L p_l
        comp ev[U], lev[U], rv[U], pv_l[KM][U], lp_l[KM][U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = min(i0 + u * (int)blockDim.x, nx - 1);
            ev[u] = v.el ? v.el[i] : q_load(M, M.e, M.e32, esc, j, i);
            lev[u] = (comp)v.Le[i];
            rv[u] = (comp)v.r[i];
#pragma unroll
            for (int l = 0; l < KM; ++l) {
                pv_l[l][u] = l < nd ? (comp)pl[l][i] : comp(0);
                lp_l[l][u] = l < nd ? (comp)Lpl[l][i] : comp(0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= nx) break;
            // p_new = e + sum alpha_l p_l and L p_new = L e + sum alpha_l L p_l
            comp pv = ev[u], lw = lev[u];
#pragma unroll
            for (int l = 0; l < KM; ++l) {
                if (l < nd) {
                    pv += al[l] * pv_l[l][u];
                    lw += al[l] * lp_l[l][u];
                }
            }
            const vec ps = (vec)pv, ls = (vec)lw;
            pn[i] = ps;
            Lpn[i] = ls;
            // the step: Phi += beta p_new, r += beta L p_new
            M.phi[row + i] = phr[i] + beta * (double)ps;
            typename Pol::res rs;
            if constexpr (Pol::kMixed) rs = (typename Pol::res)(rv[u] + beta_c * ls);
            else rs = rv[u] + beta * ls;
            v.r[i] = rs;
            const acc_t ra = (acc_t)rs, la = (acc_t)ls;
            part[0] += ra * ra;
            part[1] += la * la;
#pragma unroll
            for (int l = 0; l < KM; ++l)
                if (l < nd) part[2 + l] += la * (acc_t)lp_l[l][u];
            sb[pidx(i)] = stage0_input(M, v, eta, (comp)rs, i);
        }
    }
    SW_TRACE(201);
    stage0_finish(M, v, j, ws);
}

// first stage of option 3 from the stored r (a learned iteration falling back)
template <class Pol>
__device__ void phase_prec0(const MemberDev<Pol> &M, const RowView<Pol> &v, typename Pol::comp eta, int j,
                            unsigned char *ws)
{
    typedef typename Pol::comp comp;
    comp *sb = (comp *)(ws + sb_offset<Pol>(M.nx));
    for (int i = threadIdx.x; i < M.nx; i += blockDim.x) sb[pidx(i)] = stage0_input(M, v, eta, (comp)v.r[i], i);
    stage0_finish(M, v, j, ws);
}

// ---------------------------------------------------------------------------
// state transition after a phase, from the member-wide sums tot[slot] (FP64).
// The scalars (alpha, beta, the Gram update, norms) are FP64 for every policy.
// (The text's half-precision variant keeps these global sums in single
// precision, Sec. 4.3.)
// ---------------------------------------------------------------------------
// PH_LE scalars on the lanes of warp 0 (lane l < nd holds direction l):
// alpha_l of the text, written to c.alpha, and, in lane 0, <Lp_new, Lp_new>
// and <r, Lp_new> of the direction Lp_new = Le + sum alpha_l Lp_l, from the
// Gram matrix.  An FP64 instruction costs the same for one lane as for 32 on
// this GPU, so the lanes take the O(nd^2) products together.
__device__ __forceinline__ void le_scalars(MemberCtl &c, const double *tot, double &lplp, double &rlp)
{
    const int lane = threadIdx.x & 31, nd = c.nu + 1;
    const bool on = lane < nd;
    const double a = on ? -tot[S_C0 + lane] * c.Ginv[lane] : 0.0;
    double rowv = on ? 2.0 * tot[S_C0 + lane] : 0.0;
    for (int m = 0; m < nd; ++m) {
        const double am = __shfl_sync(0xffffffffu, a, m);
        if (on) rowv = fma(am, c.G[lane][m], rowv);
    }
    double t1 = on ? a * rowv : 0.0, t2 = on ? a * tot[S_T0 + lane] : 0.0;
    // lanes >= nd hold zeros: the tree needs only the levels below nd
#pragma unroll
    for (int o = KMAX / 2; o > 0; o >>= 1) {
        if (o < nd) {
            t1 += __shfl_down_sync(0xffffffffu, t1, o);
            t2 += __shfl_down_sync(0xffffffffu, t2, o);
        }
    }
    if (on) c.alpha[lane] = a;
    lplp = tot[S_A] + t1;
    rlp = tot[S_B] + t2;
}

template <class Pol>
__device__ void advance(const MemberDev<Pol> &M, MemberCtl &c, const double *tot, bool writer, double lplp,
                        double rlp)
{
    typedef double sc;
    const int k = M.k, nd = c.nu + 1;
    bool done = false;
    // the learned preconditioner alternates its directions with option 3's:
    // on the network's turn the launch ends (PH_EXT), the host writes the
    // network's e, and the next launch resumes with L(e)
    const bool learned = (M.pc == PC_LEARNED);
    auto to_precond = [&]() {
        c.stage = 1;
        if (learned && c.net_turn && !c.fb_now) c.phase = PH_EXT;
        else c.phase = M.nstages > 1 ? PH_PREC : PH_LE;
    };
    auto finish = [&](int st) { c.status = st; done = true; };
    switch (c.phase) {
    case PH_TRUE: {
        const double rn = sqrt((double)tot[S_A]);
        if (c.init) {
            c.init = 0;
            c.nR = sqrt((double)tot[S_B]);
            c.r0 = rn;
            c.rn_true = rn;
            c.rn2_rec = c.rn2_cur = (double)tot[S_A];
            c.nu = -1;
            // the mixed policies sum a warp's products in FP32 before the
            // FP64 sums (relative error < 1e-6): their exit test keeps that
            // margin below the tolerance
            c.tolr = M.tol * c.nR * (Pol::kMixed ? (1.0 - 1e-5) : 1.0);
            c.tolr2 = c.tolr * c.tolr;
            if (writer && M.hist) M.hist[0] = c.nR > 0.0 ? rn / c.nR : 0.0;
            if (c.nR == 0.0) { c.phase = PH_ZERO; break; }
            if (!isfinite(rn) || !isfinite(c.nR)) { finish(ST_NONFINITE); break; }
            if (rn <= c.tolr && M.min_iters <= 0) { finish(ST_OK); break; }
            to_precond();
        } else {
            c.rn_true = rn;
            c.rn2_cur = (double)tot[S_A];
            if (writer && M.hist) M.hist[c.it] = rn / c.nR;
            if (!isfinite(rn)) { finish(ST_NONFINITE); break; }
            if (rn <= c.tolr && c.it >= M.min_iters) { finish(ST_OK); break; }
            if (c.it >= M.max_iters) { finish(ST_NOT_CONVERGED); break; }
            to_precond();
        }
        break;
    }
    case PH_PREC:
        c.stage += 1;
        if (c.stage >= M.nstages) c.phase = PH_LE;
        break;
    case PH_PREC0:
        c.stage = 1;
        c.phase = M.nstages > 1 ? PH_PREC : PH_LE;
        break;
    case PH_LE: {
        // alpha (c.alpha), <Lp_new, Lp_new> (lplp) and <r, Lp_new> (rlp)
        // come from le_scalars
        if (learned && c.net_turn && !c.fb_now) {
            // the network's direction would remove rlp^2 / lplp of ||r||^2; it
            // must remove at least fb_ratio times the share the last option-3
            // direction removed, else this iteration takes option 3
            const double gain = (double)rlp * (double)rlp / ((double)lplp * c.rn2_cur);
            if (!(lplp > sc(0)) || !isfinite(lplp) || !isfinite(rlp) || !(gain >= M.fb_ratio * c.g3)) {
                c.fb_now = 1;
                c.fallbacks += 1;
                c.phase = PH_PREC0;
                break;
            }
        }
        if (!(lplp > sc(0)) || !isfinite(lplp) || !isfinite(rlp)) { finish(ST_BREAKDOWN); break; }
        c.beta = -rlp * recip(lplp);
        c.phase = PH_UB;
        break;
    }
    case PH_UB: {
        const int ln = nd;                        // logical index of the new direction
        c.it += 1;
        // squared norms: no square root on the path of every iteration
        const double rn2 = (double)tot[S_A];
        if (learned && (!c.net_turn || c.fb_now) && c.rn2_cur > 0.0)
            c.g3 = 1.0 - rn2 / c.rn2_cur;                           // an option-3 direction
        c.rn2_rec = c.rn2_cur = rn2;
        c.fb_now = 0;
        if (learned) c.net_turn ^= 1;
        if (writer && M.hist) M.hist[c.it] = sqrt(rn2) / c.nR;
        c.G[ln][ln] = (double)tot[S_B];
        c.Ginv[ln] = recip(c.G[ln][ln]);
        for (int m = 0; m < ln; ++m) c.G[ln][m] = c.G[m][ln] = (double)tot[S_C0 + m];
        c.nu = ln;
        if (c.nu == k) {                          // restart: p_0 <- p_k
            c.base = phys_slot(c, k, k);
            c.G[0][0] = c.G[k][k];
            c.Ginv[0] = c.Ginv[k];
            c.nu = 0;
        }
        if (!isfinite(rn2)) { finish(ST_NONFINITE); break; }
        if ((rn2 <= c.tolr2 && c.it >= M.min_iters) || (M.ru_every > 0 && c.it % M.ru_every == 0) ||
            c.it >= M.max_iters)
            c.phase = PH_TRUE;
        else
            to_precond();
        break;
    }
    case PH_ZERO:
        c.rn_true = c.rn2_rec = 0.0;
        finish(ST_OK);
        break;
    default: break;
    }
    if (done) c.phase = PH_DONE;
}

// ---------------------------------------------------------------------------
// the persistent GCR kernel
// ---------------------------------------------------------------------------
// KM: directions a cycle can hold (k <= KM); it sizes the per-thread
// registers of the inner-product and update loops.  MINB: resident blocks
// per SM the register allocation is made for (2 for grids whose blocks own
// several rows each: twice the warps to overlap their memory latency, at the
// price of a few spilled registers)
template <class Pol, int KM, int MINB, int WARP>
__global__ void __launch_bounds__(MAX_THREADS, MINB) k_gcr(const EnsDesc *__restrict__ D, int max_nx)
{
    typedef typename Pol::comp comp;
    typedef typename Acc<Pol>::type acc_t;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ MemberDev<Pol> s_M;
    __shared__ MemberCtl s_c;
    __shared__ int s_m, s_ok;
    __shared__ double s_blk[32];
    __shared__ double s_tot[NSLOT];
    __shared__ dfloat s_totf[NSLOT];
    if (threadIdx.x == 0) {
        int lo = 0, hi = D->n;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (D->cta_begin[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
        }
        s_m = lo;
    }
    __syncthreads();
    const int m = s_m;
    SolverBlock *B = D->blk[m];
    const int nb = D->cta_begin[m + 1] - D->cta_begin[m];
    const int local = (int)blockIdx.x - D->cta_begin[m];
    copy_in(&s_M, mdev<Pol>(B));
    copy_in(&s_c, &B->ctl);
    __syncthreads();
    // a launch that follows the host's application of the network resumes
    // with L(e); every block makes the same change
    if (threadIdx.x == 0 && s_c.phase == PH_EXT) s_c.phase = PH_LE;
    __syncthreads();
    const MemberDev<Pol> &M = s_M;
    const int ny = M.ny, nx = M.nx;
    unsigned char *ws = dsm;
    // warp mode: the warps' row buffers, then the reduction scratch
    // WARP: 0 one block per row; 1 one warp per row (D->warp_rows), rows of
    // any length; m > 1 one warp per row, specialised for rows of 32 m points
    // (only that zonal-solve variant is compiled in: a smaller kernel)
    constexpr bool wmode = WARP != 0;
    // the zonal solve's register chunks: exactly WARP points, or up to 64
    // FP32 points with the register budget of one block per SM, 16 with that
    // of two
    constexpr int SEL = WARP > 1 ? WARP : (MINB == 1 ? -64 : -16);
    const WRow wr = wrow(nx);
    double *scratch;
    typedef typename Pol::fac fac_t;
    WFac<fac_t> wf = {nullptr, nullptr, 0u, 0u, &B->g.abort, -1};
    comp *wb = nullptr;
    if constexpr (wmode) {
        // per warp: row buffer, staged factor rows, mbarrier (warp_slot_bytes)
        const bool stage = D->warp_stage != 0;
        const size_t slot = warp_slot_bytes<Pol>(nx, stage);
        unsigned char *mine = ws + (size_t)(threadIdx.x >> 5) * slot;
        wb = (comp *)mine;
        if (stage) {
            const size_t wbuf = al16((size_t)wbuf_len(nx) * sizeof(comp));
            wf.lf = (fac_t *)(mine + wbuf);
            wf.iD = wf.lf + nx;
            unsigned long long *bar = (unsigned long long *)(mine + wbuf + al16(2 * (size_t)nx * sizeof(fac_t)));
            wf.bar = smem_u32(bar);
            if ((threadIdx.x & 31) == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(wf.bar) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            __syncwarp();
        }
        scratch = (double *)(ws + (size_t)nwarps() * slot);
    } else {
        scratch = (double *)(ws + red_offset<Pol>(nx));
    }
    unsigned char *cslot = dsm + work_bytes<Pol>(max_nx);
    unsigned char *sslot = cslot + (D->cache_const ? const_bytes<Pol>(max_nx) : 0);
    // this block's rows: j = local + t * nb; the first one may be cached
    const int j0 = local;
    const bool single = (j0 + nb >= ny);
    RowView<Pol> vc;
    if (j0 < ny && !wmode) {
        if (D->cache_const && single) view_const_cache(M, j0, cslot, vc); else view_const_global(M, j0, vc);
        if (D->cache_state && single) view_state_cache(M, sslot, vc); else view_state_global(M, j0, vc);
    }
    __syncthreads();
    const comp eta = (comp)(*M.etap);
    GlobalCtl *G = &B->g;
    double *partg = M.part;
    bool ok = true;
    int par = 0;
    for (int step = 0; s_c.phase != PH_DONE && s_c.phase != PH_EXT; ++step) {
        SW_TRACE(10 + s_c.phase);
        constexpr int NP = 2 + 2 * KM;           // A, B, C_0.., T_0..
        acc_t part[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) part[q] = acc_t(0);
        if constexpr (wmode) {
            // one warp per row: warp w of the member's block `local` owns rows
            // w * nb + local + t * (nb * warps)
            const int wi = threadIdx.x >> 5, NW = nb * nwarps();
            for (int j = wi * nb + local; j < ny; j += NW) {
                RowView<Pol> v;
                view_const_global(M, j, v);
                view_state_global(M, j, v);
                switch (s_c.phase) {
                case PH_TRUE:
                    if constexpr (Pol::kMixed) {
                        if (M.split && s_c.init) {
                            // the initial residual by Eq. 14 (split fluid thickness)
                            const bool staged = wf.lf && M.pc >= 3;
                            if (staged) wfac_issue(wf, j, M.lfT + (size_t)j * nx, M.invDT + (size_t)j * nx, nx);
                            const SplitState S = {M.shat, M.sdx, M.scx, M.sdy, M.scy};
                            split_true_row<Pol, NP>(M, S, v, eta, j, threadIdx.x & 31, 32, part,
                                                    [&](int i, comp x) { wb[tpos(wr, i)] = x; });
                            wstage0_finish<Pol, SEL>(M, v, j, wb, wr, wf, staged);
                            break;
                        }
                    }
                    wphase_true<Pol, NP, SEL>(M, v, eta, j, wb, wr, wf, part);
                    break;
                case PH_UB: wphase_ub<Pol, KM, SEL>(M, s_c, v, eta, j, wb, wr, wf, part); break;
                case PH_PREC: wprecond_stage<Pol, SEL>(M, v, eta, s_c.stage, j, wb, wr, wf); break;
                case PH_PREC0: wphase_prec0<Pol, SEL>(M, v, eta, j, wb, wr, wf); break;
                case PH_LE: wphase_le<Pol, KM, SEL>(M, s_c, v, j, wr, part); break;
                case PH_ZERO:
                    for (int i = threadIdx.x & 31; i < nx; i += 32) M.phi[(size_t)j * nx + i] = 0.0;
                    break;
                default: break;
                }
            }
            // the factors of the warp's first row for the next phase's zonal
            // solve, started now so that the copies overlap the member
            // barrier: a solve follows L(e) (the update), the update or the
            // true residual or an earlier stage (a Richardson stage).  In the
            // kernels specialised for one row length (the generic kernel,
            // which runs the ensembles, measured slower with it)
            if (WARP > 1 && wf.lf && M.pc >= 3) {
                const int jf = wi * nb + local, ph = s_c.phase;
                const bool next_solves = ph == PH_LE ||
                                         ((ph == PH_UB || ph == PH_TRUE || ph == PH_PREC0) && M.nstages > 1) ||
                                         (ph == PH_PREC && s_c.stage + 1 < M.nstages);
                if (jf < ny && next_solves) wfac_ahead(wf, jf, M.lfT + (size_t)jf * nx, M.invDT + (size_t)jf * nx, nx);
            }
            __syncthreads();
        } else {
            for (int j = j0; j < ny; j += nb) {
                RowView<Pol> v;
                if (j == j0) v = vc;
                else { view_const_global(M, j, v); view_state_global(M, j, v); }
                switch (s_c.phase) {
                case PH_TRUE:
                    if constexpr (Pol::kMixed) {
                        if (M.split && s_c.init) {
                            // the initial residual by Eq. 14 (split fluid thickness)
                            comp *sb = (comp *)(ws + sb_offset<Pol>(nx));
                            const SplitState S = {M.shat, M.sdx, M.scx, M.sdy, M.scy};
                            split_true_row<Pol, NP>(M, S, v, eta, j, threadIdx.x, blockDim.x, part,
                                                    [&](int i, comp x) { sb[pidx(i)] = x; });
                            stage0_finish(M, v, j, ws);
                            break;
                        }
                    }
                    phase_true<Pol, NP>(M, v, eta, j, ws, part);
                    break;
                case PH_UB: phase_ub<Pol, KM>(M, s_c, v, eta, j, ws, part); break;
                case PH_PREC: precond_stage<Pol>(M, v, eta, s_c.stage, j, ws); break;
                case PH_PREC0: phase_prec0<Pol>(M, v, eta, j, ws); break;
                case PH_LE: phase_le<Pol, KM>(M, s_c, v, j, ws, part); break;
                case PH_ZERO:
                    for (int i = threadIdx.x; i < nx; i += blockDim.x) M.phi[(size_t)j * nx + i] = 0.0;
                    break;
                default: break;
                }
            }
        }
        SW_TRACE(30);
        // block sums of the partials, published slot-major
        int slot[NSLOT];
        const int ns = phase_slots(s_c.phase, s_c.nu + 1, slot);
        double *pbuf = partg + (size_t)par * NSLOT * ny;
        if (ns > 0) {
            if constexpr (Pol::kMixed) block_sum_many_df<NP>(part, (dfloat *)s_blk, (float *)scratch);
            else block_sum_many<NP, acc_t>(part, s_blk, scratch);
            if (threadIdx.x < ns) {
                const int g = slot[threadIdx.x];          // slot of tot; its place in part
                const int at = g < S_T0 ? g : g - S_T0 + 2 + KM;
                if constexpr (Pol::kMixed) ((dfloat *)pbuf)[(size_t)threadIdx.x * ny + local] = ((const dfloat *)s_blk)[at];
                else pbuf[(size_t)threadIdx.x * ny + local] = s_blk[at];
            }
        }
        __syncthreads();
        SW_TRACE(31);
        // member barrier: monotonic arrival counter
        if (threadIdx.x == 0) {
            int okb = 1;
            red_release_add(&G->count, 1ull);
            const unsigned long long target = (unsigned long long)nb * (unsigned long long)(step + 1) + g_extra_arrivals;
            const unsigned long long limit = g_wait_limit_ns;
            if (ld_acquire(&G->count) < target) {
                const unsigned long long t0 = gtimer();
                while (ld_acquire(&G->count) < target) {
                    if (vload(&G->abort)) { okb = 0; break; }
                    if (gtimer() - t0 > limit) {
                        if (atomicExch(&G->abort, 1) == 0) G->where = step;
                        okb = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            s_ok = okb;
        }
        __syncthreads();
        if (!s_ok) { ok = false; break; }
        SW_TRACE(32);
        // member-wide sums, every block in the same order: warp w adds slots
        // w, w + nwarps, ... over the member's blocks, in FP64 (FP64 policy)
        // or in double-float arithmetic (mixed policies, whose magnitudes
        // stay far inside the FP32 range)
        if (ns > 0) {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int q = w; q < ns; q += nw) {
                if constexpr (Pol::kMixed) {
                    const float2 *src = (const float2 *)pbuf + (size_t)q * ny;
                    dfloat t{0.f, 0.f};
#pragma unroll 8
                    for (int b = lane; b < nb; b += 32) {
                        const float2 x = __ldcg(src + b);
                        t = df_add(t, dfloat{x.x, x.y});
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        t = df_add(t, dfloat{__shfl_xor_sync(0xffffffffu, t.hi, o),
                                             __shfl_xor_sync(0xffffffffu, t.lo, o)});
                    if (lane == 0) s_totf[q] = t;
                } else {
                    const double *src = pbuf + (size_t)q * ny;
                    double t = 0;
#pragma unroll 8
                    for (int b = lane; b < nb; b += 32) t += __ldcg(src + b);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                    if (lane == 0) s_tot[slot[q]] = t;
                }
            }
        }
        __syncthreads();
        if constexpr (Pol::kMixed) {
            // the double-float totals to FP64, one slot per lane
            if (threadIdx.x < ns) s_tot[slot[threadIdx.x]] = (double)s_totf[threadIdx.x].hi + (double)s_totf[threadIdx.x].lo;
            __syncthreads();
        }
        SW_TRACE(33);
        if (threadIdx.x < 32) {
            double lplp = 0.0, rlp = 0.0;
            if (s_c.phase == PH_LE) le_scalars(s_c, s_tot, lplp, rlp);
            __syncwarp();
            SW_TRACE(35);
            if (threadIdx.x == 0) advance<Pol>(M, s_c, s_tot, local == 0, lplp, rlp);
            SW_TRACE(36);
        }
        __syncthreads();
        SW_TRACE(34);
        par ^= 1;
    }
    if (local == 0 && threadIdx.x == 0) {
        const int *src = (const int *)&s_c;
        int *dst = (int *)&B->ctl;
        for (int q = 0; q < (int)(sizeof(MemberCtl) / 4); ++q) dst[q] = src[q];
        if (D->stats) {
            // the member's sw_solve_stats (a block that passed every member
            // barrier has seen any abort)
            const int st = vload(&G->abort) ? ST_TIMEOUT : (s_c.phase == PH_DONE ? s_c.status : ST_INTERNAL);
            sw_solve_stats S = {};
            S.iterations = s_c.it;
            S.converged = (st == ST_OK);
            S.status = st;
            S.fallbacks = s_c.fallbacks;
            S.r0_norm = s_c.r0;
            S.R_norm = s_c.nR;
            S.true_rel_residual = s_c.nR > 0 ? s_c.rn_true / s_c.nR : 0.0;
            S.recursive_rel_residual = s_c.nR > 0 ? sqrt(s_c.rn2_rec) / s_c.nR : 0.0;
            S.eta = *M.etap;
            D->stats[m] = S;
        }
    }
    // copies started ahead for a phase that did not come (the solve ended)
    if constexpr (wmode) {
        if (wf.pre >= 0) wfac_wait(wf);
    }
    // per-row norms of the final true residual
    const bool want_rowres = ok && s_c.phase == PH_DONE && M.rowres && (s_c.status == ST_OK || s_c.status == ST_NOT_CONVERGED);
    if constexpr (wmode) {
        if (!want_rowres) return;
        // each warp its own rows (the rows whose r it wrote)
        const int wi = threadIdx.x >> 5, NW = nb * nwarps(), lane = threadIdx.x & 31;
        for (int j = wi * nb + local; j < ny; j += NW) {
            const typename Pol::res *r = M.r + (size_t)j * nx;
            double t = 0.0;
            if (s_c.nR > 0.0)
                for (int i = lane; i < nx; i += 32) { double x = (double)r[i]; t += x * x; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) M.rowres[j] = sqrt(t);
        }
    } else if (want_rowres) {
        for (int j = j0; j < ny; j += nb) {
            const typename Pol::res *r = (j == j0) ? vc.r : M.r + (size_t)j * nx;
            double t = 0.0;
            if (s_c.nR > 0.0)
                for (int i = threadIdx.x; i < nx; i += blockDim.x) { double x = (double)r[i]; t += x * x; }
            double tv[1] = {t};
            block_sum_many<1, double>(tv, s_blk, scratch);
            if (threadIdx.x == 0) M.rowres[j] = sqrt(s_blk[0]);
            __syncthreads();
        }
    }
}

// The host-side entry points of one translation unit's instantiations of
// k_gcr: the kernel for a GCR k and register budget, and the settings of this
// unit's own copies of the device-side globals (the barrier test hook and, in
// traced builds, the time line).
#ifdef SW_PHASE_TRACE
#define SW_GCR_TRACE_FN(TAG)                                                      \
    void gcr_trace_##TAG(unsigned long long *buf, int cap, int block)            \
    {                                                                             \
        int z = 0;                                                                \
        cudaMemcpyToSymbol(g_trace_buf, &buf, sizeof(buf));                       \
        cudaMemcpyToSymbol(g_trace_n, &z, sizeof(z));                             \
        cudaMemcpyToSymbol(g_trace_cap, &cap, sizeof(cap));                       \
        cudaMemcpyToSymbol(g_trace_blk, &block, sizeof(block));                   \
    }
#else
#define SW_GCR_TRACE_FN(TAG)
#endif

#define SW_GCR_DEBUG_FN(TAG)                                                                      \
    cudaError_t gcr_debug_##TAG(unsigned long long extra, unsigned long long limit_ns)            \
    {                                                                                             \
        cudaError_t e = cudaMemcpyToSymbol(g_extra_arrivals, &extra, sizeof(extra));              \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_wait_limit_ns, &limit_ns, sizeof(limit_ns)); \
        return e;                                                                                 \
    }                                                                                             \
    SW_GCR_TRACE_FN(TAG)

#define SW_GCR_UNIT(POL, WARP, TAG)                                                               \
    const void *gcr_kernel_##TAG(int k, int minb)                                                 \
    {                                                                                             \
        if (k <= 4) return minb > 1 ? (const void *)k_gcr<POL, 4, 2, WARP> : (const void *)k_gcr<POL, 4, 1, WARP>; \
        return minb > 1 ? (const void *)k_gcr<POL, KMAX, 2, WARP> : (const void *)k_gcr<POL, KMAX, 1, WARP>;     \
    }                                                                                             \
    SW_GCR_DEBUG_FN(TAG)

// the warp-per-row kernels specialised for one row length (chunks of 32 or 64
// points per lane), GCR k <= 4 and one block per SM
#define SW_GCR_SPEC_UNIT(POL, TAG)                                                                \
    const void *gcr_kernel_##TAG(int m)                                                           \
    {                                                                                             \
        if (m == 64) return (const void *)k_gcr<POL, 4, 1, 64>;                                   \
        if (m == 32) return (const void *)k_gcr<POL, 4, 1, 32>;                                   \
        return nullptr;                                                                           \
    }                                                                                             \
    SW_GCR_DEBUG_FN(TAG)

} // namespace sw
