// sw_rows.cuh -- per-row work of the elliptic solver: the operator stencil
// (Eq. 10), the lagged part P^M (Eq. 13), the preconditioner stages and the
// GCR vector phases.  One thread block processes one latitude row at a time;
// the rows it reads around j (j-1, j, j+1) are staged in shared memory.
#pragma once

#include "sw_common.cuh"

namespace sw {

// shared-memory workspace of one block (carved from dynamic shared memory)
template <class Pol>
struct RowSmem {
    typedef typename Pol::comp comp;
    double *s3d;     // 3 rows, FP64 (true residual)
    comp *s3c;       // 3 rows, policy type (aliases s3d)
    comp *sb;        // 1 row, tridiagonal buffer
    double *red;     // NSLOT * nwarps
    comp *scan;      // 2 * nwarps
    float *redf;     // nwarps
};

template <class Pol>
__host__ __device__ inline size_t row_smem_bytes(int nx, int threads)
{
    size_t nw = threads / 32;
    size_t a = 3 * (size_t)nx * sizeof(double);
    size_t b = (size_t)nx * sizeof(typename Pol::comp);
    size_t c = NSLOT * nw * sizeof(double) + 2 * nw * sizeof(double) + nw * sizeof(float);
    return ((a + 15) & ~(size_t)15) + ((b + 15) & ~(size_t)15) + c + 64;
}

template <class Pol>
__device__ inline RowSmem<Pol> carve_smem(unsigned char *base, int nx)
{
    RowSmem<Pol> s;
    size_t nw = blockDim.x / 32;
    size_t a = ((3 * (size_t)nx * sizeof(double)) + 15) & ~(size_t)15;
    size_t b = (((size_t)nx * sizeof(typename Pol::comp)) + 15) & ~(size_t)15;
    s.s3d = (double *)base;
    s.s3c = (typename Pol::comp *)base;
    s.sb = (typename Pol::comp *)(base + a);
    s.red = (double *)(base + a + b);
    s.scan = (typename Pol::comp *)(s.red + NSLOT * nw);
    s.redf = (float *)((double *)s.scan + 2 * nw);
    return s;
}

// Stage rows j-1, j, j+1 of a field into s3 (row r of s3 = row j-1+r); the row
// beyond a pole is the pole row shifted by nx/2.  ld(row, col) loads one value.
template <class T, class LD>
__device__ __forceinline__ void stage3(T *s3, int nx, int ny, int j, LD ld)
{
    for (int r = 0; r < 3; ++r) {
        int jj = j - 1 + r, src = jj, sh = 0;
        if (jj < 0) { src = 0; sh = nx / 2; }
        else if (jj >= ny) { src = ny - 1; sh = nx / 2; }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            int ii = i + sh;
            if (ii >= nx) ii -= nx;
            s3[r * nx + i] = ld(src, ii);
        }
    }
    __syncthreads();
}

// (L x)_ij (full = true) or (P^M x)_ij (full = false) from the staged rows
// S (j-1), X (j), N (j+1) and the face coefficients of rows j and j-1.
template <class T, class CT>
__device__ __forceinline__ T stencil(const T *S, const T *X, const T *N, int i, int nx, int j, int ny,
                                     const CT *ax, const CT *cx, const CT *bx, const CT *ay,
                                     const CT *cy, const CT *by, const CT *C, bool full)
{
    const int ie = (i + 1 == nx) ? 0 : i + 1;
    const int iw = (i == 0) ? nx - 1 : i - 1;
    const size_t row = (size_t)j * nx;
    const T xc = X[i], xe = X[ie], xw = X[iw];
    const T xn = N[i], xne = N[ie], xnw = N[iw];
    const T xs = S[i], xse = S[ie], xsw = S[iw];
    // zonal fluxes through the east (i+1/2) and west (i-1/2) faces
    T fe = (T)cx[row + i] * (xn + xne - xs - xse) + (T)bx[row + i] * (xc + xe);
    T fw = (T)cx[row + iw] * (xnw + xn - xsw - xs) + (T)bx[row + iw] * (xw + xc);
    if (full) {
        fe += (T)ax[row + i] * (xe - xc);
        fw += (T)ax[row + iw] * (xc - xw);
    }
    T v = fe - fw;
    // meridional fluxes through the north (j+1/2) and south (j-1/2) faces;
    // zero through the pole faces
    if (j < ny - 1)
        v += (T)ay[row + i] * (xn - xc) + (T)cy[row + i] * (xe + xne - xw - xnw) + (T)by[row + i] * (xc + xn);
    if (j > 0) {
        const size_t rs = row - nx;
        v -= (T)ay[rs + i] * (xc - xs) + (T)cy[rs + i] * (xse + xe - xsw - xw) + (T)by[rs + i] * (xs + xc);
    }
    if (full) v -= (T)C[row + i] * xc;
    return v;
}

template <class Pol>
__device__ __forceinline__ bool in_band(const MemberDev<Pol> &M, int j)
{
    return Pol::kMixed && (j < M.band || j >= M.ny - M.band);
}

// value (i) of row j of a preconditioner field (q or e): FP64 for the FP64
// policy; FP32 on pole-band rows or 16-bit times the row scale otherwise.
template <class Pol>
__device__ __forceinline__ typename Pol::comp q_load(const MemberDev<Pol> &M, const typename Pol::q16 *h,
                                                     const float *f32, float sc, int j, int i)
{
    const size_t id = (size_t)j * M.nx + i;
    if constexpr (!Pol::kMixed) {
        return ldcg(h + id);
    } else {
        if (in_band(M, j)) return ldcg(f32 + id);
        return q_to_f(ldcg(h + id)) * sc;
    }
}

template <class Pol>
__device__ __forceinline__ float q_scale(const MemberDev<Pol> &M, const float *sc, int j)
{
    if constexpr (Pol::kMixed) return in_band(M, j) ? 1.f : ldcg(sc + j);
    else return 1.f;
}

template <class Pol>
__device__ __forceinline__ void stage3_q(typename Pol::comp *s3, const MemberDev<Pol> &M,
                                         const typename Pol::q16 *h, const float *f32, const float *sc, int j)
{
    const int nx = M.nx, ny = M.ny;
    for (int r = 0; r < 3; ++r) {
        int jj = j - 1 + r, src = jj, sh = 0;
        if (jj < 0) { src = 0; sh = nx / 2; }
        else if (jj >= ny) { src = ny - 1; sh = nx / 2; }
        const float s = q_scale(M, sc, src);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            int ii = i + sh;
            if (ii >= nx) ii -= nx;
            s3[r * nx + i] = q_load(M, h, f32, s, src, ii);
        }
    }
    __syncthreads();
}

// store row j of a preconditioner field from sb (16-bit storage gets a
// power-of-two row scale so that the stored magnitudes are <= 1)
template <class Pol>
__device__ __forceinline__ void q_store_row(const MemberDev<Pol> &M, typename Pol::q16 *h, float *f32,
                                            float *sc, int j, const typename Pol::comp *sb, float *redf)
{
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    if constexpr (!Pol::kMixed) {
        for (int i = threadIdx.x; i < nx; i += blockDim.x) h[row + i] = sb[i];
    } else {
        if (in_band(M, j)) {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) f32[row + i] = sb[i];
            return;
        }
        float m = 0.f;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) m = fmaxf(m, fabsf(sb[i]));
        m = block_max(m, redf);
        float s = 1.f;
        if (m > 0.f && m <= 3.0e38f) { int e; frexpf(m, &e); s = ldexpf(1.f, e); }
        else if (!(m <= 3.0e38f)) s = m;        // NaN / Inf: propagate
        const float inv = 1.f / s;              // exact: s is a power of two
        for (int i = threadIdx.x; i < nx; i += blockDim.x) h[row + i] = f_to_q<typename Pol::q16>(sb[i] * inv);
        if (threadIdx.x == 0) sc[j] = s;
    }
}

// pointwise first Richardson stage input from the residual value rv:
// option 0: r; 1: r/D; 2: omega r/D (q_1 with q_0 = 0); 3: -eta r (then T^{-1})
template <class Pol>
__device__ __forceinline__ typename Pol::comp stage0_input(const MemberDev<Pol> &M, double eta,
                                                           typename Pol::comp rv, size_t id)
{
    typedef typename Pol::comp comp;
    switch (M.pc) {
    case 0: return rv;
    case 1: return rv / (comp)M.wdiag[id];
    case 2: return (comp)M.omega * rv / (comp)M.wdiag[id];
    default: return -(comp)eta * rv;
    }
}

// finish the first preconditioner stage of row j (sb holds stage0_input):
// option 3 solves the zonal system; the result goes to e (single stage) or qa.
template <class Pol>
__device__ void stage0_finish(const MemberDev<Pol> &M, int j, RowSmem<Pol> &sm)
{
    typedef typename Pol::comp comp;
    __syncthreads();
    const size_t row = (size_t)j * M.nx;
    if (M.pc == 3)
        trisolve_row<comp, typename Pol::fac>(sm.sb, M.nx, M.lf + row, M.invD + row, M.zz + row,
                                              (comp)M.gam[j], (comp)M.ec[j], sm.scan);
    if (M.nstages == 1) q_store_row(M, M.e, M.e32, M.e_s, j, sm.sb, sm.redf);
    else q_store_row(M, M.qa, M.qa32, M.qa_s, j, sm.sb, sm.redf);
    __syncthreads();
}

// preconditioner stage mu >= 1 of row j: reads q_mu (rows j-1..j+1) from
// `in`, writes q_{mu+1} to `out`.
//   option 3 (Eq. 13): [I - eta (P^Z - P^H)] q_{mu+1} = q_mu + eta (P^M q_mu - r)
//   option 2:          q_{mu+1} = q_mu + omega D^{-1} (r - L q_mu)
template <class Pol, class RT>
__device__ void precond_stage(const MemberDev<Pol> &M, double eta, int j, RowSmem<Pol> &sm,
                              const typename Pol::q16 *in_h, const float *in_f, const float *in_s,
                              const RT *r,
                              typename Pol::q16 *out_h, float *out_f, float *out_s)
{
    typedef typename Pol::comp comp;
    const int nx = M.nx, ny = M.ny;
    const size_t row = (size_t)j * nx;
    stage3_q(sm.s3c, M, in_h, in_f, in_s, j);
    const comp *S = sm.s3c, *X = sm.s3c + nx, *N = sm.s3c + 2 * nx;
    const bool opt3 = (M.pc == 3);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        comp rv = (comp)ldcg(r + row + i);
        comp v = stencil<comp, typename Pol::coef>(S, X, N, i, nx, j, ny, M.wax, M.wcx, M.wbx, M.way,
                                                   M.wcy, M.wby, M.wC, !opt3);
        if (opt3) sm.sb[i] = X[i] + (comp)eta * (v - rv);
        else sm.sb[i] = X[i] + (comp)M.omega * (rv - v) / (comp)M.wdiag[row + i];
    }
    __syncthreads();
    if (opt3)
        trisolve_row<comp, typename Pol::fac>(sm.sb, nx, M.lf + row, M.invD + row, M.zz + row,
                                              (comp)M.gam[j], (comp)M.ec[j], sm.scan);
    q_store_row(M, out_h, out_f, out_s, j, sm.sb, sm.redf);
    __syncthreads();
}

} // namespace sw
