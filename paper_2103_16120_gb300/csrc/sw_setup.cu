// sw_setup.cu -- work done once per set of coefficients (sw_elliptic_set_coeffs):
//  * face coefficients of the flux-form operator (Eq. 10) in FP64 and FP32,
//    the diagonal of L (preconditioner options 1 and 2) and, per row, the
//    largest |diag(P^M)| (for the automatic pseudo time step of Eq. 13);
//  * the factorised zonal operator T = I - eta (P^Z - P^H) of every row: a
//    symmetric cyclic tridiagonal matrix, split by Sherman-Morrison into its
//    plain tridiagonal part T' = L D L^T and a rank-one wrap correction.
// The pivots D_i follow the continued fraction D_i = d_i - o_{i-1}^2 / D_{i-1};
// written as the three-term recurrence of the leading minors it is a product
// of 2x2 transfer matrices, which a block computes with a parallel scan.
#include "sw_common.cuh"
#include "sw_internal.h"

namespace sw {

__global__ void __launch_bounds__(MAX_THREADS) k_faces(FaceArgs a)
{
    __shared__ double red[MAX_THREADS / 32];
    const int nx = a.nx, ny = a.ny, j = blockIdx.x;
    // the face scales, each with the 1/2 of the face mean folded in (a power
    // of two: the products round exactly as (a + b)/2 times the scale)
    const double idl2 = 0.5 / (a.dlam * a.dlam), idp2 = 0.5 / (a.dphi * a.dphi);
    const double i4 = 0.5 / (4.0 * a.dlam * a.dphi), i2l = 0.5 / (2.0 * a.dlam), i2p = 0.5 / (2.0 * a.dphi);
    const size_t row = (size_t)j * nx;
    double m = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int ip = (i + 1 == nx) ? 0 : i + 1, im = (i == 0) ? nx - 1 : i - 1;
        const size_t id = row + i;
        // x faces i+1/2 and i-1/2 of row j
        double ax = (a.A11[id] + a.A11[row + ip]) * idl2;
        double cx = (a.A12[id] + a.A12[row + ip]) * i4;
        double bx = (a.B1[id] + a.B1[row + ip]) * i2l;
        double axm = (a.A11[row + im] + a.A11[id]) * idl2;
        double bxm = (a.B1[row + im] + a.B1[id]) * i2l;
        // y faces j+1/2 and j-1/2 (zero through the pole faces)
        double ay = 0.0, cy = 0.0, by = 0.0, ays = 0.0, bys = 0.0;
        if (j < ny - 1) {
            ay = (a.A22[id] + a.A22[id + nx]) * idp2;
            cy = (a.A21[id] + a.A21[id + nx]) * i4;
            by = (a.B2[id] + a.B2[id + nx]) * i2p;
        }
        if (j > 0) {
            ays = (a.A22[id - nx] + a.A22[id]) * idp2;
            bys = (a.B2[id - nx] + a.B2[id]) * i2p;
        }
        const double c = a.C[id];
        // diagonal of P^M = L - P^Z + P^H, and of L
        const double dpm = (bx - bxm) - (ay + ays) + (by - bys);
        const double dl = -(ax + axm) + dpm - c;
        a.ax[id] = ax; a.cx[id] = cx; a.bx[id] = bx;
        a.ay[id] = ay; a.cy[id] = cy; a.by[id] = by;
        a.C64[id] = c; a.diag[id] = dl;
        a.wax[id] = (float)ax; a.wcx[id] = (float)cx; a.wbx[id] = (float)bx;
        a.way[id] = (float)ay; a.wcy[id] = (float)cy; a.wby[id] = (float)by;
        a.wC[id] = (float)c; a.wdiag[id] = (float)dl;
        m = fmax(m, fabs(dpm));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) mm = fmax(mm, red[ww]);
        a.rowmax[j] = mm;
    }
}

// 2x2 matrix [[m00, m01], [m10, m11]]
template <class T> struct M2 { T m00, m01, m10, m11; };

template <class T>
__device__ __forceinline__ M2<T> mul(const M2<T> &A, const M2<T> &B)   // A B
{
    return {A.m00 * B.m00 + A.m01 * B.m10, A.m00 * B.m01 + A.m01 * B.m11,
            A.m10 * B.m00 + A.m11 * B.m10, A.m10 * B.m01 + A.m11 * B.m11};
}

// scale by a power of two so that the largest entry is O(1) (ratios unchanged)
template <class T>
__device__ __forceinline__ void renorm(M2<T> &A)
{
    T m = fmax(fmax(fabs(A.m00), fabs(A.m01)), fmax(fabs(A.m10), fabs(A.m11)));
    if (m > T(0) && isfinite(m)) {
        int e;
        frexp(m, &e);
        A.m00 = ldexp(A.m00, -e); A.m01 = ldexp(A.m01, -e);
        A.m10 = ldexp(A.m10, -e); A.m11 = ldexp(A.m11, -e);
    }
}

template <class T>
__device__ __forceinline__ M2<T> shfl_up(const M2<T> &A, int d)
{
    return {__shfl_up_sync(0xffffffffu, A.m00, d), __shfl_up_sync(0xffffffffu, A.m01, d),
            __shfl_up_sync(0xffffffffu, A.m10, d), __shfl_up_sync(0xffffffffu, A.m11, d)};
}

// exclusive block scan of matrices in thread order: returns the product of
// the matrices of all earlier threads (later ones on the left)
template <class T>
__device__ M2<T> scan_mat_excl(M2<T> A, M2<T> *sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    M2<T> inc = A;
    for (int d = 1; d < 32; d <<= 1) {
        M2<T> o = shfl_up(inc, d);
        if (lane >= d) { inc = mul(inc, o); renorm(inc); }
    }
    M2<T> ex = shfl_up(inc, 1);
    if (lane == 0) ex = {T(1), T(0), T(0), T(1)};
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    M2<T> pre = {T(1), T(0), T(0), T(1)};
    for (int ww = 0; ww < w; ++ww) { pre = mul(sm[ww], pre); renorm(pre); }
    M2<T> out = mul(ex, pre);
    renorm(out);
    __syncthreads();
    return out;
}

// the zonal factors of every row in the arithmetic of T: FP64 factors for the
// FP64 solver (lf, invD, zz, gam, ec), FP32 ones for the mixed solvers (lf32,
// invD32, zz32, gam32, ec32).  An FP64 instruction costs about 64 cycles per
// warp on this GPU against about 5 for FP32, so the mixed path's factors are
// computed in FP32 and the FP64 ones only when an FP64 solve needs them.
template <class T>
__global__ void __launch_bounds__(MAX_THREADS) k_factor(FactorArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    T *sb = (T *)dsm;                                    // nx
    __shared__ M2<T> smat[MAX_THREADS / 32];
    __shared__ T sscan[2 * (MAX_THREADS / 32)];
    __shared__ double red[MAX_THREADS / 32];
    __shared__ double s_eta;
    const int nx = a.nx, ny = a.ny, j = blockIdx.x;
    const size_t row = (size_t)j * nx;
    constexpr bool f64 = sizeof(T) == 8;

    // eta: explicit, or 1 / max |diag(P^M)| over the grid (FP64 in both)
    if (a.eta_explicit > 0.0) {
        if (threadIdx.x == 0) s_eta = a.eta_explicit;
    } else {
        double m = 0.0;
        for (int r = threadIdx.x; r < ny; r += blockDim.x) m = fmax(m, a.rowmax[r]);
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double mm = 0.0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) mm = fmax(mm, red[ww]);
            s_eta = mm > 0.0 ? 1.0 / mm : 1.0;
        }
    }
    __syncthreads();
    const double eta64 = s_eta;
    if (j == 0 && threadIdx.x == 0) *a.eta_out = eta64;
    const T eta = (T)eta64;

    // row of T: diag_i = 1 + eta (ax_i + ax_{i-1} + C_i); coupling of i and
    // i+1: o_i = -eta ax_i (o_{nx-1} couples the last point to the first)
    const double *ax = a.ax + row, *C = a.C + row;
    auto diagT = [&](int i) {
        int im = (i == 0) ? nx - 1 : i - 1;
        return T(1) + eta * ((T)ax[i] + (T)ax[im] + (T)C[i]);
    };
    const T ec = -eta * (T)ax[nx - 1];
    const T d0 = diagT(0);
    const T gam = -d0;
    // T' = T minus the rank-one wrap term w w^T / gam, w = (gam, 0, .., 0, ec)
    auto dprime = [&](int i) {
        T d = diagT(i);
        if (i == 0) d -= gam;
        if (i == nx - 1) d -= ec * ec / gam;
        return d;
    };
    int c0, c1;
    row_chunk(nx, c0, c1);
    // product of the transfer matrices [[d'_i, -o_{i-1}^2], [1, 0]] of my chunk
    M2<T> P = {T(1), T(0), T(0), T(1)};
    for (int i = c0; i < c1; ++i) {
        T o = (i == 0) ? T(0) : -eta * (T)ax[i - 1];
        M2<T> Mi = {dprime(i), -o * o, T(1), T(0)};
        P = mul(Mi, P);
        renorm(P);
    }
    M2<T> Q = scan_mat_excl(P, smat);
    // pivot before my chunk: D_{c0-1} = theta_{c0-1} / theta_{c0-2} = Q00 / Q10
    T Dprev = (c0 > 0) ? Q.m00 / Q.m10 : T(0);
    double *lf64 = a.lf + row, *iD64 = a.invD + row;
    float *lf32 = a.lf32 + row, *iD32 = a.invD32 + row;
    // the transposed copies of the warp-per-row solver: point i at
    // (i % m) * 32 + i / m of the row, m = nx / 32 (nx a power of two)
    T *lfT = f64 ? (T *)a.lfT : (T *)a.lf32T, *iDT = f64 ? (T *)a.invDT : (T *)a.invD32T;
    T *zT = f64 ? (T *)a.zzT : (T *)a.zz32T;
    const int mT = nx >> 5, lmT = mT > 0 ? __ffs(mT) - 1 : 0;
    auto tp = [&](int i) { return (size_t)((i & (mT - 1)) * 32 + (i >> lmT)); };
    for (int i = c0; i < c1; ++i) {
        T l = T(0), D;
        if (i == 0) {
            D = dprime(0);
        } else {
            T o = -eta * (T)ax[i - 1];
            l = o / Dprev;
            D = dprime(i) - l * o;
        }
        const T iD = T(1) / D;
        if constexpr (f64) { lf64[i] = l; iD64[i] = iD; }
        else { lf32[i] = l; iD32[i] = iD; }
        if (lfT) { lfT[row + tp(i)] = l; iDT[row + tp(i)] = iD; }
        Dprev = D;
    }
    __syncthreads();
    // z = T'^{-1} w
    for (int i = threadIdx.x; i < nx; i += blockDim.x) sb[i] = (i == 0) ? gam : ((i == nx - 1) ? ec : T(0));
    __syncthreads();
    if constexpr (f64) trisolve_row<T, T>(sb, nx, lf64, iD64, (const T *)nullptr, T(0), T(0), sscan);
    else trisolve_row<T, T>(sb, nx, lf32, iD32, (const T *)nullptr, T(0), T(0), sscan);
    const T g = T(1) / (gam + gam * sb[0] + ec * sb[nx - 1]);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const T z = sb[i] * g;
        if constexpr (f64) a.zz[row + i] = z;
        else a.zz32[row + i] = z;
        if (zT) zT[row + tp(i)] = z;
    }
    if (threadIdx.x == 0) {
        if constexpr (f64) { a.gam[j] = gam; a.ec[j] = ec; }
        else { a.gam32[j] = gam; a.ec32[j] = ec; }
    }
}

cudaError_t launch_faces(const FaceArgs &a, int threads, cudaStream_t s)
{
    k_faces<<<a.ny, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_factor(const FactorArgs &a, bool fp64, int threads, cudaStream_t s)
{
    const size_t smem = (size_t)a.nx * (fp64 ? sizeof(double) : sizeof(float));
    if (smem > 48 * 1024) {
        cudaError_t e = fp64 ? cudaFuncSetAttribute(k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                             : cudaFuncSetAttribute(k_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (fp64) k_factor<double><<<a.ny, threads, smem, s>>>(a);
    else k_factor<float><<<a.ny, threads, smem, s>>>(a);
    return cudaGetLastError();
}

} // namespace sw
