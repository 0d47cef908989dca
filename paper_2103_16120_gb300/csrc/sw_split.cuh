// sw_split.cuh -- the initial residual r0 = L(Phi) - R in single precision
// with the split fluid thickness of Sec. 4.2, Eq. 14.
//
// Phi is held as Phi_hat + Phi_tilde.  At a refresh (sw_split_refresh),
// Phi_hat = fp32(Phi) is stored with the derivative parts of its face fluxes
// (computed in FP64 from Phi_hat, stored in FP32).  The residual then takes
// Phi_tilde = fp32(Phi - Phi_hat), forms the derivative parts of Phi_tilde in
// FP32 and adds the stored ones of Phi_hat, evaluates the B and C terms on
// the FP32 sum Phi_hat + Phi_tilde, and the divergence in FP32.  The grid
// spacings are folded into the face coefficients (ax = a11/dlam^2,
// cx = a12/(4 dlam dphi), bx = b1/(2 dlam), and the same on the meridional
// faces), so the stored "derivatives" are the differences and cross sums
// those coefficients multiply:
//   zonal face (i+1/2, j):      dx = P[i+1] - P[i],
//                               cx = P[i,j+1] + P[i+1,j+1] - P[i,j-1] - P[i+1,j-1]
//   meridional face (i, j+1/2): dy = P[j+1] - P[j],
//                               cy = P[i+1,j] + P[i+1,j+1] - P[i-1,j] - P[i-1,j+1]
// with the operator's periodic longitude and across-pole continuation.
#pragma once

#include "sw_warp.cuh"

namespace sw {

// the stored split state of a grid: Phi_hat and its four derivative fields
struct SplitState {
    const float *hat, *dx, *cx, *dy, *cy;
};

// what the split operator reads besides the split state: Phi (FP64) and the
// FP32 face coefficients
struct SplitOp {
    int nx, ny;
    const double *phi;
    const float *wax, *wcx, *wbx, *way, *wcy, *wby, *wC;
};

template <class Pol>
__device__ __forceinline__ SplitOp split_op(const MemberDev<Pol> &M)
{
    return SplitOp{M.nx, M.ny, M.phi, (const float *)M.wax, (const float *)M.wcx, (const float *)M.wbx,
                   (const float *)M.way, (const float *)M.wcy, (const float *)M.wby, (const float *)M.wC};
}

// L(Phi) at points i0 .. i0 + 3 of row j by Eq. 14, in FP32 (nx a multiple of 8)
__device__ __forceinline__ void split_quad(const SplitOp &M, const SplitState &S, int j, int i0, float (&L)[4])
{
    const int nx = M.nx, ny = M.ny;
    const size_t row = (size_t)j * nx, rs = j > 0 ? row - nx : row;
    const bool has_n = j < ny - 1, has_s = j > 0;
    int srcS, shS, srcN, shN;
    ghost_row(j - 1, nx, ny, srcS, shS);
    ghost_row(j + 1, nx, ny, srcN, shN);
    int aN = i0 + shN; if (aN >= nx) aN -= nx;
    int aS = i0 + shS; if (aS >= nx) aS -= nx;
    // Phi and Phi_hat windows (longitudes i0 - 1 .. i0 + 4) of rows j, j+1, j-1
    double pc[6], pn[6], ps[6];
    cg6(M.phi + row, i0, nx, pc);
    cg6(M.phi + (size_t)srcN * nx, aN, nx, pn);
    cg6(M.phi + (size_t)srcS * nx, aS, nx, ps);
    float hc[6], hn[6], hs[6];
    cg6(S.hat + row, i0, nx, hc);
    cg6(S.hat + (size_t)srcN * nx, aN, nx, hn);
    cg6(S.hat + (size_t)srcS * nx, aS, nx, hs);
    // Phi_tilde = fp32(Phi - Phi_hat) and Phi_SP = Phi_hat + Phi_tilde
    float tc[6], tn[6], ts[6], sc[6], sn[6], ss[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        tc[k] = (float)(pc[k] - (double)hc[k]);
        tn[k] = (float)(pn[k] - (double)hn[k]);
        ts[k] = (float)(ps[k] - (double)hs[k]);
        sc[k] = hc[k] + tc[k];
        sn[k] = hn[k] + tn[k];
        ss[k] = hs[k] + ts[k];
    }
    // stored derivative parts of Phi_hat: zonal faces i0 - 1 .. i0 + 3 of row
    // j, meridional faces of rows j (north) and j - 1 (south)
    const int iw = i0 == 0 ? nx - 1 : i0 - 1;
    float hdx[5], hcx[5], q[4];
    hdx[0] = __ldg(S.dx + row + iw); hcx[0] = __ldg(S.cx + row + iw);
    ldg4(S.dx + row + i0, q); for (int u = 0; u < 4; ++u) hdx[u + 1] = q[u];
    ldg4(S.cx + row + i0, q); for (int u = 0; u < 4; ++u) hcx[u + 1] = q[u];
    float hdn[4] = {}, hcn[4] = {}, hds[4] = {}, hcs[4] = {};
    if (has_n) { ldg4(S.dy + row + i0, hdn); ldg4(S.cy + row + i0, hcn); }
    if (has_s) { ldg4(S.dy + rs + i0, hds); ldg4(S.cy + rs + i0, hcs); }
    const RowCoef<float> c = {M.wax + row, M.wcx + row, M.wbx + row, M.way + row, M.wcy + row, M.wby + row,
                              M.way + rs, M.wcy + rs, M.wby + rs, M.wC + row};
    Coef4<float> k;
    coef4(c, i0, nx, true, has_n, has_s, k);
    // zonal fluxes: face m between window points m and m + 1
    float F[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const float dx = (tc[m + 1] - tc[m]) + hdx[m];
        const float cr = ((tn[m] + tn[m + 1]) - (ts[m] + ts[m + 1])) + hcx[m];
        F[m] = k.ax[m] * dx + k.cx[m] * cr + k.bx[m] * (sc[m] + sc[m + 1]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int p = u + 1;
        float v = F[u + 1] - F[u];
        if (has_n) {
            const float dy = (tn[p] - tc[p]) + hdn[u];
            const float cr = ((tc[p + 1] + tn[p + 1]) - (tc[p - 1] + tn[p - 1])) + hcn[u];
            v += k.ay[u] * dy + k.cy[u] * cr + k.by[u] * (sc[p] + sn[p]);
        }
        if (has_s) {
            const float dy = (tc[p] - ts[p]) + hds[u];
            const float cr = ((ts[p + 1] + tc[p + 1]) - (ts[p - 1] + tc[p - 1])) + hcs[u];
            v -= k.ays[u] * dy + k.cys[u] * cr + k.bys[u] * (ss[p] + sc[p]);
        }
        L[u] = v - k.cc[u] * sc[p];
    }
}

// the split initial residual of row j for the solver's first phase, by the
// threads (tid, T) of a block or a warp: r (policy type) into the row's r,
// ||r||^2 and ||R||^2 into part, the first preconditioner stage's input to
// put(i, value) (phase_true with the operator of Eq. 14)
template <class Pol, int NP, class PUT>
__device__ __forceinline__ void split_true_row(const MemberDev<Pol> &M, const SplitState &S, const RowView<Pol> &v,
                                               typename Pol::comp eta, int j, int tid, int T,
                                               typename Acc<Pol>::type (&part)[NP], PUT put)
{
    typedef typename Pol::comp comp;
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    const SplitOp op = split_op(M);
    double rr = 0.0, RR = 0.0;
    for (int i0 = 4 * tid; i0 < nx; i0 += 4 * T) {
        float L[4];
        split_quad(op, S, j, i0, L);
        double Rv[4];
        ldg4(M.R + row + i0, Rv);
        typename Pol::res r4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double rv = (double)L[u] - Rv[u];
            r4[u] = (typename Pol::res)rv;
            rr += rv * rv;
            RR += Rv[u] * Rv[u];
            put(i0 + u, stage0_input(M, v, eta, (comp)r4[u], i0 + u));
        }
        stv4(v.r + i0, r4);
    }
    part[0] += (typename Acc<Pol>::type)rr;
    part[1] += (typename Acc<Pol>::type)RR;
}

} // namespace sw
