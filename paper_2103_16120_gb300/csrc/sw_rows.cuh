// sw_rows.cuh -- per-row work of the elliptic solver, one thread block per
// latitude row: the operator stencil (Eq. 10), the lagged part P^M (Eq. 13)
// and the preconditioner stages.  The field rows a stencil needs (j-1, j,
// j+1) are copied into shared memory in one round trip; the row's constant
// data (face coefficients, zonal factors) and its owner-only vectors (r, L e,
// p_l, L p_l and a copy of e) live either in shared memory for the whole solve
// or in global memory, behind the pointers of a RowView.
#pragma once

#include "sw_block.cuh"

namespace sw {

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// ---------------------------------------------------------------------------
// shared-memory layout of the block (one row at a time)
//   stg   3 staged rows (policy compute type); also 3 FP64 rows of Phi
//   raw   mixed policies: the 16-bit / FP32 rows as copied from global memory
//   sb    one padded row (tridiagonal buffer)
//   red   reduction / scan scratch
//   const 11 coefficient rows + 3 padded factor rows of the owned row (optional)
//   state r, L e, e copy, (k+1) p rows, (k+1) L p rows of the owned row (optional)
// ---------------------------------------------------------------------------
template <class Pol>
__host__ __device__ inline size_t raw_offset(int nx)
{
    return al16(3 * (size_t)nx * sizeof(typename Pol::comp));
}

template <class Pol>
__host__ __device__ inline size_t sb_offset(int nx)
{
    const size_t raw_end = raw_offset<Pol>(nx) + (Pol::kMixed ? al16(3 * (size_t)nx * 4) : 0);
    const size_t phi3 = al16(3 * (size_t)nx * sizeof(double));
    return raw_end > phi3 ? raw_end : phi3;
}

template <class Pol>
__host__ __device__ inline size_t red_offset(int nx)
{
    return sb_offset<Pol>(nx) + al16((size_t)padded_len(nx) * sizeof(typename Pol::comp));
}

constexpr int RED_WORDS = 32 * (MAX_THREADS / 32);   // scratch values (8 bytes each)

template <class Pol>
__host__ __device__ inline size_t work_bytes(int nx)
{
    return red_offset<Pol>(nx) + al16(RED_WORDS * sizeof(double));
}

template <class Pol>
__host__ __device__ inline size_t const_bytes(int nx)
{
    return al16(11 * (size_t)nx * sizeof(typename Pol::coef)) + al16(3 * (size_t)padded_len(nx) * sizeof(typename Pol::fac));
}

template <class Pol>
__host__ __device__ inline size_t state_bytes(int nx, int k)
{
    typedef typename Pol::vec vec;
    return al16((size_t)nx * sizeof(typename Pol::res)) + al16((size_t)nx * sizeof(vec)) +
           al16((size_t)nx * sizeof(typename Pol::comp)) + 2 * al16((size_t)(k + 1) * nx * sizeof(vec));
}

// where the data of one row live
template <class Pol>
struct RowView {
    typedef typename Pol::coef CT;
    typedef typename Pol::fac FT;
    typedef typename Pol::vec VT;
    // constants (coefficient rows unpadded; factor rows padded when fpad)
    const CT *ax, *cx, *bx, *ay, *cy, *by, *ays, *cys, *bys, *C, *diag;
    const FT *lf, *invD, *zz;
    bool fpad;
    double gam, ec;
    // owner-only vectors of the row
    typename Pol::res *r;
    VT *Le;
    typename Pol::comp *el;         // copy of the row of e (nullptr: read e itself)
    VT *pb, *Lpb;                   // slot 0 of p and L p; slot s at + s * vstride
    size_t vstride;
};

template <class CT>
struct RowCoef {
    const CT *ax, *cx, *bx, *ay, *cy, *by, *ays, *cys, *bys, *C;
};

template <class Pol>
__device__ __forceinline__ RowCoef<typename Pol::coef> coef_of(const RowView<Pol> &v)
{
    return {v.ax, v.cx, v.bx, v.ay, v.cy, v.by, v.ays, v.cys, v.bys, v.C};
}

// constants of row j straight from global memory
template <class Pol>
__device__ __forceinline__ void view_const_global(const MemberDev<Pol> &M, int j, RowView<Pol> &v)
{
    const size_t row = (size_t)j * M.nx, rs = j > 0 ? row - M.nx : row;
    v.ax = M.wax + row; v.cx = M.wcx + row; v.bx = M.wbx + row;
    v.ay = M.way + row; v.cy = M.wcy + row; v.by = M.wby + row;
    v.ays = M.way + rs; v.cys = M.wcy + rs; v.bys = M.wby + rs;
    v.C = M.wC + row; v.diag = M.wdiag + row;
    v.lf = M.lf + row; v.invD = M.invD + row; v.zz = M.zz + row;
    v.fpad = false;
    v.gam = M.gam[j]; v.ec = M.ec[j];
}

// copy row j's constants into the block's cache and point the view there
template <class Pol>
__device__ void view_const_cache(const MemberDev<Pol> &M, int j, unsigned char *slot, RowView<Pol> &v)
{
    typedef typename Pol::coef CT;
    typedef typename Pol::fac FT;
    const int nx = M.nx;
    RowView<Pol> g;
    view_const_global(M, j, g);
    CT *c = (CT *)slot;
    const CT *src[11] = {g.ax, g.cx, g.bx, g.ay, g.cy, g.by, g.ays, g.cys, g.bys, g.C, g.diag};
    for (int a = 0; a < 11; ++a)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) c[a * nx + i] = src[a][i];
    const int pl = padded_len(nx);
    FT *f = (FT *)(slot + al16(11 * (size_t)nx * sizeof(CT)));
    const FT *fs[3] = {g.lf, g.invD, g.zz};
    for (int a = 0; a < 3; ++a)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) f[a * pl + pidx(i)] = fs[a][i];
    v.ax = c; v.cx = c + nx; v.bx = c + 2 * nx; v.ay = c + 3 * nx; v.cy = c + 4 * nx; v.by = c + 5 * nx;
    v.ays = c + 6 * nx; v.cys = c + 7 * nx; v.bys = c + 8 * nx; v.C = c + 9 * nx; v.diag = c + 10 * nx;
    v.lf = f; v.invD = f + pl; v.zz = f + 2 * pl;
    v.fpad = true;
    v.gam = g.gam; v.ec = g.ec;
}

template <class Pol>
__device__ __forceinline__ void view_state_global(const MemberDev<Pol> &M, int j, RowView<Pol> &v)
{
    const size_t row = (size_t)j * M.nx;
    v.r = M.r + row;
    v.Le = M.Le + row;
    v.el = nullptr;
    v.pb = M.p + row;
    v.Lpb = M.Lp + row;
    v.vstride = (size_t)M.nx * M.ny;
}

template <class Pol>
__device__ __forceinline__ void view_state_cache(const MemberDev<Pol> &M, unsigned char *slot, RowView<Pol> &v)
{
    typedef typename Pol::vec VT;
    const int nx = M.nx;
    unsigned char *p = slot;
    v.r = (typename Pol::res *)p; p += al16((size_t)nx * sizeof(typename Pol::res));
    v.Le = (VT *)p; p += al16((size_t)nx * sizeof(VT));
    v.el = (typename Pol::comp *)p; p += al16((size_t)nx * sizeof(typename Pol::comp));
    v.pb = (VT *)p; p += al16((size_t)(M.k + 1) * nx * sizeof(VT));
    v.Lpb = (VT *)p;
    v.vstride = nx;
}

// source row and shift of row jj in [-1, ny] (the row beyond a pole is the
// pole row shifted by nx/2)
__device__ __forceinline__ void ghost_row(int jj, int nx, int ny, int &src, int &sh)
{
    src = jj; sh = 0;
    if (jj < 0) { src = 0; sh = nx / 2; }
    else if (jj >= ny) { src = ny - 1; sh = nx / 2; }
}

// ---------------------------------------------------------------------------
// stencils
// ---------------------------------------------------------------------------
// elements per thread whose loads a row loop issues together: enough loads in
// flight to cover the memory latency when the row data are not cached, few
// enough registers for two resident blocks
template <class T>
__host__ __device__ constexpr int batch_of() { return sizeof(T) == 8 ? 2 : 4; }

// y_i = (L x)_i (full) or (P^M x)_i for the whole row from the staged rows
// S (j-1), X (j), N (j+1); y[pidx(i)] when ypad, else y[i].  The coefficients
// of a batch of elements are loaded before any result is stored.
template <class T, class CT>
__device__ __noinline__ void stencil_row(const T *S, const T *X, const T *N, int nx, int j, int ny,
                                         const RowCoef<CT> c, bool full, T *y, bool ypad)
{
    constexpr int U = batch_of<T>();
    const int nt = blockDim.x;
    const bool has_n = j < ny - 1, has_s = j > 0;
    for (int i0 = threadIdx.x; i0 < nx; i0 += U * nt) {
        CT cx[U], cxw[U], bx[U], bxw[U], ax[U], axw[U], ay[U], cy[U], by[U], ays[U], cys[U], bys[U], cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = min(i0 + u * nt, nx - 1), iw = (i == 0) ? nx - 1 : i - 1;
            cx[u] = c.cx[i]; cxw[u] = c.cx[iw]; bx[u] = c.bx[i]; bxw[u] = c.bx[iw];
            ax[u] = full ? c.ax[i] : CT(0); axw[u] = full ? c.ax[iw] : CT(0);
            ay[u] = has_n ? c.ay[i] : CT(0); cy[u] = has_n ? c.cy[i] : CT(0); by[u] = has_n ? c.by[i] : CT(0);
            ays[u] = has_s ? c.ays[i] : CT(0); cys[u] = has_s ? c.cys[i] : CT(0); bys[u] = has_s ? c.bys[i] : CT(0);
            cc[u] = full ? c.C[i] : CT(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * nt;
            if (i >= nx) break;
            const int ie = (i + 1 == nx) ? 0 : i + 1, iw = (i == 0) ? nx - 1 : i - 1;
            const T xc = X[i], xe = X[ie], xw = X[iw];
            const T xn = N[i], xne = N[ie], xnw = N[iw];
            const T xs = S[i], xse = S[ie], xsw = S[iw];
            // zonal fluxes through the east (i+1/2) and west (i-1/2) faces
            T fe = (T)cx[u] * (xn + xne - xs - xse) + (T)bx[u] * (xc + xe) + (T)ax[u] * (xe - xc);
            T fw = (T)cxw[u] * (xnw + xn - xsw - xs) + (T)bxw[u] * (xw + xc) + (T)axw[u] * (xc - xw);
            T v = fe - fw;
            // meridional fluxes through the north (j+1/2) and south (j-1/2)
            // faces; zero through the pole faces
            if (has_n) v += (T)ay[u] * (xn - xc) + (T)cy[u] * (xe + xne - xw - xnw) + (T)by[u] * (xc + xn);
            if (has_s) v -= (T)ays[u] * (xc - xs) + (T)cys[u] * (xse + xe - xsw - xw) + (T)bys[u] * (xs + xc);
            y[ypad ? pidx(i) : i] = v - (T)cc[u] * xc;
        }
    }
    __syncthreads();
}

// stencil_row for rows of a multiple of 4 points (16-byte aligned rows and
// coefficients): a thread takes 4 consecutive points per pass, reads them
// with vector loads, and forms each zonal face flux once for its two points.
// The expressions are those of stencil_row, so the results are the same.
template <class T>
__device__ __forceinline__ void ldv4(const T *p, T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 q = *(const float4 *)p;
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = ((const double2 *)p)[0], q1 = ((const double2 *)p)[1];
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

template <class T>
__device__ __forceinline__ void stv4(T *p, const T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        ((double2 *)p)[0] = make_double2(v[0], v[1]);
        ((double2 *)p)[1] = make_double2(v[2], v[3]);
    }
}

__device__ __forceinline__ bool al16p(const void *p) { return ((uintptr_t)p & 15) == 0; }

template <class T>
__device__ __forceinline__ void ldw6(const T *rowp, int i0, int nx, T (&v)[6])
{
    T m[4];
    ldv4(rowp + i0, m);
    v[1] = m[0]; v[2] = m[1]; v[3] = m[2]; v[4] = m[3];
    v[0] = rowp[i0 == 0 ? nx - 1 : i0 - 1];
    v[5] = rowp[i0 + 4 == nx ? 0 : i0 + 4];
}

template <class T, class CT>
__device__ __noinline__ void stencil_row4(const T *S, const T *X, const T *N, int nx, int j, int ny,
                                          const RowCoef<CT> c, bool full, T *y, bool ypad)
{
    const bool has_n = j < ny - 1, has_s = j > 0;
    for (int i0 = 4 * threadIdx.x; i0 < nx; i0 += 4 * blockDim.x) {
        T xc[6], xn[6], xs[6];
        ldw6(X, i0, nx, xc);
        ldw6(N, i0, nx, xn);
        ldw6(S, i0, nx, xs);
        const int iw = i0 == 0 ? nx - 1 : i0 - 1;
        CT ax[5] = {}, cx[5], bx[5], q[4];
        cx[0] = c.cx[iw]; bx[0] = c.bx[iw];
        ldv4(c.cx + i0, q); for (int k = 0; k < 4; ++k) cx[k + 1] = q[k];
        ldv4(c.bx + i0, q); for (int k = 0; k < 4; ++k) bx[k + 1] = q[k];
        CT cc[4] = {};
        if (full) {
            ax[0] = c.ax[iw];
            ldv4(c.ax + i0, q); for (int k = 0; k < 4; ++k) ax[k + 1] = q[k];
            ldv4(c.C + i0, cc);
        }
        CT ay[4] = {}, cy[4] = {}, by[4] = {}, ays[4] = {}, cys[4] = {}, bys[4] = {};
        if (has_n) { ldv4(c.ay + i0, ay); ldv4(c.cy + i0, cy); ldv4(c.by + i0, by); }
        if (has_s) { ldv4(c.ays + i0, ays); ldv4(c.cys + i0, cys); ldv4(c.bys + i0, bys); }
        // face m (m = 0..4) between window points m - 1 and m (window k = longitude i0 - 1 + k)
        T F[5];
#pragma unroll
        for (int m = 0; m < 5; ++m)
            F[m] = (T)cx[m] * (xn[m] + xn[m + 1] - xs[m] - xs[m + 1]) + (T)bx[m] * (xc[m] + xc[m + 1]) +
                   (T)ax[m] * (xc[m + 1] - xc[m]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = u + 1;
            T v = F[u + 1] - F[u];
            if (has_n) v += (T)ay[u] * (xn[k] - xc[k]) + (T)cy[u] * (xc[k + 1] + xn[k + 1] - xc[k - 1] - xn[k - 1]) +
                            (T)by[u] * (xc[k] + xn[k]);
            if (has_s) v -= (T)ays[u] * (xc[k] - xs[k]) + (T)cys[u] * (xs[k + 1] + xc[k + 1] - xs[k - 1] - xc[k - 1]) +
                            (T)bys[u] * (xs[k] + xc[k]);
            const int i = i0 + u;
            y[ypad ? pidx(i) : i] = v - (T)cc[u] * xc[k];
        }
    }
    __syncthreads();
}

// the vector stencil needs rows of a multiple of 4 points and 16-byte aligned
// coefficient rows
template <class CT>
__device__ __forceinline__ bool stencil4_ok(const RowCoef<CT> &c, int nx)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    return (nx & 3) == 0 && al(c.cx) && al(c.bx) && al(c.ax) && al(c.C) && al(c.ay) && al(c.cy) && al(c.by) &&
           al(c.ays) && al(c.cys) && al(c.bys);
}

template <class Pol>
__device__ __forceinline__ bool in_band(const MemberDev<Pol> &M, int j)
{
    return Pol::kMixed && (j < M.band || j >= M.ny - M.band);
}

template <class Pol>
__device__ __forceinline__ float q_scale(const MemberDev<Pol> &M, const float *sc, int j)
{
    if constexpr (Pol::kMixed) return in_band(M, j) ? 1.f : __ldcg(sc + j);
    else return 1.f;
}

// value (i) of row j of a preconditioner field read straight from global
// memory (rows without a shared-memory copy)
template <class Pol>
__device__ __forceinline__ typename Pol::comp q_load(const MemberDev<Pol> &M, const typename Pol::q16 *h,
                                                     const float *f32, float sc, int j, int i)
{
    const size_t id = (size_t)j * M.nx + i;
    if constexpr (!Pol::kMixed) {
        return __ldcg(h + id);
    } else {
        if (in_band(M, j)) return __ldcg(f32 + id);
        return q_to_f(h[id]) * sc;
    }
}

// stage rows j-1, j, j+1 of a preconditioner field into stg: the three source
// rows are copied as they are (one round trip), then converted with their
// row scales and the pole shift in shared memory
template <class Pol>
__device__ __noinline__ void stage3_q(unsigned char *ws, const MemberDev<Pol> &M, const typename Pol::q16 *h,
                                      const float *f32, const float *sc, int j)
{
    typedef typename Pol::comp comp;
    typedef typename Pol::q16 qt;
    const int nx = M.nx, ny = M.ny;
    comp *stg = (comp *)ws;
    int src[3], sh[3];
    if constexpr (!Pol::kMixed) {
        // FP64: straight into the stage, the pole shift as two half-row copies
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ghost_row(j - 1 + r, nx, ny, src[r], sh[r]);
            const qt *sr = h + (size_t)src[r] * nx;
            comp *d = stg + (size_t)r * nx;
            if (sh[r] == 0) {
                row_copy_issue(d, sr, nx * (int)sizeof(qt));
            } else {
                row_copy_issue(d, sr + sh[r], (nx - sh[r]) * (int)sizeof(qt));
                row_copy_issue(d + (nx - sh[r]), sr, sh[r] * (int)sizeof(qt));
            }
        }
        row_copy_wait();
        return;
    }
    unsigned char *raw = ws + raw_offset<Pol>(nx);
    const size_t rs = (size_t)nx * 4;   // raw row stride
    bool band[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ghost_row(j - 1 + r, nx, ny, src[r], sh[r]);
        band[r] = in_band(M, src[r]);
        const size_t off = (size_t)src[r] * nx;
        if (band[r]) row_copy_issue(raw + r * rs, f32 + off, nx * 4);
        else row_copy_issue(raw + r * rs, h + off, nx * (int)sizeof(qt));
    }
    float s[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) s[r] = q_scale(M, sc, src[r]);
    row_copy_wait();
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const qt *rq = (const qt *)(raw + r * rs);
        const float *rf = (const float *)(raw + r * rs);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            int ii = i + sh[r];
            if (ii >= nx) ii -= nx;
            stg[r * nx + i] = band[r] ? rf[ii] : q_to_f(rq[ii]) * s[r];
        }
    }
    __syncthreads();
}

// store row j of a preconditioner field from the padded buffer sb (16-bit
// storage gets a power-of-two row scale so the stored magnitudes are <= 1);
// el (optional) receives the values as stored
template <class Pol>
__device__ __noinline__ void q_store_row(const MemberDev<Pol> &M, typename Pol::q16 *h, float *f32, float *sc,
                                         int j, const typename Pol::comp *sb, typename Pol::comp *el,
                                         float *scratch)
{
    typedef typename Pol::comp comp;
    const int nx = M.nx;
    const size_t row = (size_t)j * nx;
    if constexpr (!Pol::kMixed) {
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const comp v = sb[pidx(i)];
            h[row + i] = v;
            if (el) el[i] = v;
        }
    } else {
        if (in_band(M, j)) {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const comp v = sb[pidx(i)];
                f32[row + i] = v;
                if (el) el[i] = v;
            }
        } else {
            float m = 0.f;
            for (int i = threadIdx.x; i < nx; i += blockDim.x) m = fmaxf(m, fabsf(sb[pidx(i)]));
            m = block_max(m, scratch);
            float s = 1.f;
            if (m > 0.f && m <= 3.0e38f) { int e; frexpf(m, &e); s = ldexpf(1.f, e); }
            else if (!(m <= 3.0e38f)) s = m;        // NaN / Inf: propagate
            const float inv = 1.f / s;              // exact: s is a power of two
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const typename Pol::q16 q = f_to_q<typename Pol::q16>(sb[pidx(i)] * inv);
                h[row + i] = q;
                if (el) el[i] = q_to_f(q) * s;
            }
            if (threadIdx.x == 0) sc[j] = s;
        }
    }
    __syncthreads();
}

// pointwise first Richardson stage input from the residual value rv:
// option 0: r; 1: r/D; 2: omega r/D (q_1 with q_0 = 0); 3: -eta r (then T^{-1})
template <class Pol>
__device__ __forceinline__ typename Pol::comp stage0_input(const MemberDev<Pol> &M, const RowView<Pol> &v,
                                                           typename Pol::comp eta, typename Pol::comp rv, int i)
{
    typedef typename Pol::comp comp;
    switch (M.pc) {
    case 0: return rv;
    case 1: return rv / (comp)v.diag[i];
    case 2: return (comp)M.omega * rv / (comp)v.diag[i];
    default: return -eta * rv;
    }
}

template <class Pol>
__device__ __forceinline__ void trisolve_view(typename Pol::comp *sb, int nx, const RowView<Pol> &v,
                                              typename Pol::comp *sm)
{
    typedef typename Pol::comp comp;
    if (v.fpad) trisolve_block<comp, typename Pol::fac, true>(sb, nx, v.lf, v.invD, v.zz, (comp)v.gam, (comp)v.ec, sm);
    else trisolve_block<comp, typename Pol::fac, false>(sb, nx, v.lf, v.invD, v.zz, (comp)v.gam, (comp)v.ec, sm);
}

// finish the first preconditioner stage of row j (sb holds stage0_input):
// option 3 solves the zonal system; the result goes to e (single stage) or qa
template <class Pol>
__device__ void stage0_finish(const MemberDev<Pol> &M, const RowView<Pol> &v, int j, unsigned char *ws)
{
    typedef typename Pol::comp comp;
    comp *sb = (comp *)(ws + sb_offset<Pol>(M.nx));
    comp *sm = (comp *)(ws + red_offset<Pol>(M.nx));
    __syncthreads();
    SW_TRACE(401);
    if (M.pc >= 3) trisolve_view(sb, M.nx, v, sm);     // option 3 (also the learned fallback)
    SW_TRACE(402);
    if (M.nstages == 1) q_store_row(M, M.e, M.e32, M.e_s, j, sb, v.el, (float *)sm);
    else q_store_row(M, M.qa, M.qa32, M.qa_s, j, sb, (comp *)nullptr, (float *)sm);
}

// preconditioner stage mu >= 1 of row j: reads q_mu (rows j-1..j+1), writes
// q_{mu+1} (the last stage writes e).
//   option 3 (Eq. 13): [I - eta (P^Z - P^H)] q_{mu+1} = q_mu + eta (P^M q_mu - r)
//   option 2:          q_{mu+1} = q_mu + omega D^{-1} (r - L q_mu)
template <class Pol>
__device__ void precond_stage(const MemberDev<Pol> &M, const RowView<Pol> &v, typename Pol::comp eta, int mu,
                              int j, unsigned char *ws)
{
    typedef typename Pol::comp comp;
    const int nx = M.nx, ny = M.ny;
    const bool last = (mu == M.nstages - 1);
    const typename Pol::q16 *ih = (mu & 1) ? M.qa : M.qb;
    const float *if32 = (mu & 1) ? M.qa32 : M.qb32;
    const float *is = (mu & 1) ? M.qa_s : M.qb_s;
    typename Pol::q16 *oh = last ? M.e : ((mu & 1) ? M.qb : M.qa);
    float *of32 = last ? M.e32 : ((mu & 1) ? M.qb32 : M.qa32);
    float *os = last ? M.e_s : ((mu & 1) ? M.qb_s : M.qa_s);
    comp *stg = (comp *)ws;
    comp *sb = (comp *)(ws + sb_offset<Pol>(nx));
    comp *sm = (comp *)(ws + red_offset<Pol>(nx));
    stage3_q(ws, M, ih, if32, is, j);
    SW_TRACE(301);
    const comp *S = stg, *X = stg + nx, *N = stg + 2 * nx;
    const bool opt3 = (M.pc >= 3);
    if (stencil4_ok(coef_of(v), nx))
        stencil_row4<comp, typename Pol::coef>(S, X, N, nx, j, ny, coef_of(v), !opt3, sb, true);
    else
        stencil_row<comp, typename Pol::coef>(S, X, N, nx, j, ny, coef_of(v), !opt3, sb, true);
    constexpr int U = batch_of<comp>();
    for (int i0 = threadIdx.x; i0 < nx; i0 += U * blockDim.x) {
        comp rv[U], dg[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = min(i0 + u * (int)blockDim.x, nx - 1);
            rv[u] = (comp)v.r[i];
            dg[u] = opt3 ? comp(1) : (comp)v.diag[i];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= nx) break;
            const comp s = sb[pidx(i)], xv = X[i];
            sb[pidx(i)] = opt3 ? xv + eta * (s - rv[u]) : xv + (comp)M.omega * (rv[u] - s) / dg[u];
        }
    }
    __syncthreads();
    SW_TRACE(302);
    if (opt3) trisolve_view(sb, nx, v, sm);
    SW_TRACE(303);
    q_store_row(M, oh, of32, os, j, sb, last ? v.el : (comp *)nullptr, (float *)sm);
}

} // namespace sw
