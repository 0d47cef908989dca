// sw_swe.cu -- semi-implicit shallow-water time stepping around the elliptic
// solve (Sec. 2.2, Eqs. 1-10): the explicit part of a step, the right-hand
// side of the increment solve and the recovery of the momenta, as FP64
// stencil kernels over the collocated grid, and the C ABI (sw_swe_*) that
// runs them with the solver.
//
// Every kernel takes one cell per thread: blocks of 128 consecutive
// longitudes of one latitude row (coalesced rows; the four neighbours come
// from L1/L2), rows strided by gridDim.y.  A step moves about 90 doubles per
// cell through these kernels (two passes of the coefficient and right-hand
// side kernels), against about 350 B per cell per iteration of the FP64
// solve: the two solves dominate whenever they take more than a few
// iterations.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/sw_elliptic.h"
#include "sw_internal.h"

namespace sw {

constexpr int SWE_THREADS = 128;

// FP64 arithmetic issues slowly on this GPU (one warp instruction per 64
// cycles per SM sub-partition; a division is about ten of them), so the
// per-row factors come from tables made on the host and each cell divides
// twice per step (1/Phi for the winds, 1/D of the 2x2 system), both in the
// forcing kernel.
struct Geom {
    int nx, ny;
    double a, dt, grav, omega;
    double inv2dlam, inv2dphi, invdlam, invdphi;   // 1/(2 dlam), 1/(2 dphi), 1/dlam, 1/dphi
    const double *cosr, *sinr, *tanr;   // per latitude row
    const double *invcos;               // 1 / cos(phi_j)
    const double *Crow;                 // C of Eq. 10: a^2 cos(phi_j) / (dt/2)
    const double *tscale;               // dt / (a^2 cos(phi_j)): transport over dt
    const double *gx;                   // g / (a cos(phi_j)): zonal pressure gradient
};

// centre and its four neighbours; beyond a pole, the pole row half a circle away
struct Nbr {
    size_t c, e, w, n, s;
};

__device__ __forceinline__ Nbr neighbours(int i, int j, int nx, int ny)
{
    Nbr r;
    const size_t row = (size_t)j * nx;
    const int ih = i + nx / 2 >= nx ? i + nx / 2 - nx : i + nx / 2;
    r.c = row + i;
    r.e = row + (i + 1 == nx ? 0 : i + 1);
    r.w = row + (i == 0 ? nx - 1 : i - 1);
    r.n = j + 1 < ny ? row + nx + i : row + ih;
    r.s = j > 0 ? row - nx + i : row + ih;
    return r;
}

// ---------------------------------------------------------------------------
// 1. winds at n, advective velocity at n + 1/2, Q + dt/2 R^n (Eqs. 4-5),
//    b = dt/2 (f + u* tan(phi)/a) of the implicit Coriolis term and 1/D of
//    the 2x2 system of Eq. 8 (D = c^2 + b^2, c = 1 + dt/2 alpha)
// ---------------------------------------------------------------------------
struct ForcingArgs {
    Geom G;
    const double *phi, *qx, *qy, *up, *vp, *h0, *alpha, *qbx, *qby;
    int has_prev;
    double *U, *V, *psx, *psy, *bb, *invD, *un, *vn;
};

__global__ void __launch_bounds__(SWE_THREADS) k_swe_forcing(ForcingArgs A)
{
    const int nx = A.G.nx, ny = A.G.ny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double a = A.G.a, delta = 0.5 * A.G.dt, ga = A.G.grav / a, inva = 1.0 / a;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const Nbr q = neighbours(i, j, nx, ny);
        const double cj = A.G.cosr[j], sj = A.G.sinr[j], tja = A.G.tanr[j] * inva;
        const double ph = A.phi[q.c], qx = A.qx[q.c], qy = A.qy[q.c];
        const double rph = 1.0 / ph;
        const double u = qx * rph, v = qy * rph;
        const double upv = A.has_prev ? A.up[q.c] : u;
        const double vpv = A.has_prev ? A.vp[q.c] : v;
        A.U[q.c] = a * (1.5 * u - 0.5 * upv);
        A.V[q.c] = a * cj * (1.5 * v - 0.5 * vpv);
        const double he = A.phi[q.e] + A.h0[q.e], hw = A.phi[q.w] + A.h0[q.w];
        const double hn = A.phi[q.n] + A.h0[q.n], hs = A.phi[q.s] + A.h0[q.s];
        const double f = 2.0 * A.G.omega * sj;
        const double fn = f + u * tja;
        const double al = A.alpha[q.c];
        const double Rx = -A.G.gx[j] * ph * ((he - hw) * A.G.inv2dlam) + fn * qy - al * (qx - A.qbx[q.c]);
        const double Ry = -ga * ph * ((hn - hs) * A.G.inv2dphi) - fn * qx - al * (qy - A.qby[q.c]);
        A.psx[q.c] = qx + delta * Rx;
        A.psy[q.c] = qy + delta * Ry;
        const double ustar = 2.0 * u - upv;
        const double b = delta * (f + ustar * tja);
        const double c = 1.0 + delta * al;
        A.bb[q.c] = b;
        A.invD[q.c] = 1.0 / (c * c + b * b);
        A.un[q.c] = u;
        A.vn[q.c] = v;
    }
}

// ---------------------------------------------------------------------------
// 2. donor-cell transport of Q + dt/2 R^n over dt (Eq. 6): face velocity =
//    mean of the two cells, nothing through the pole faces
// ---------------------------------------------------------------------------
struct TransportArgs {
    Geom G;
    const double *U, *V, *psx, *psy;
    double *qhx, *qhy;
};

__device__ __forceinline__ double donor(double vel, double up, double down)
{
    return fmax(vel, 0.0) * up + fmin(vel, 0.0) * down;
}

__global__ void __launch_bounds__(SWE_THREADS) k_swe_transport(TransportArgs A)
{
    const int nx = A.G.nx, ny = A.G.ny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const Nbr q = neighbours(i, j, nx, ny);
        const double scale = A.G.tscale[j];
        const double Uc = A.U[q.c];
        const double ue = 0.5 * (Uc + A.U[q.e]);
        const double uw = 0.5 * (A.U[q.w] + Uc);
        const double Vc = A.V[q.c];
        const double vn = j + 1 < ny ? 0.5 * (Vc + A.V[q.n]) : 0.0;
        const double vs = j > 0 ? 0.5 * (A.V[q.s] + Vc) : 0.0;
        const double *src[2] = {A.psx, A.psy};
        double *dst[2] = {A.qhx, A.qhy};
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const double *p = src[f];
            const double pc = p[q.c];
            const double fe = donor(ue, pc, p[q.e]);
            const double fw = donor(uw, p[q.w], pc);
            const double fnf = j + 1 < ny ? donor(vn, pc, p[q.n]) : 0.0;
            const double fsf = j > 0 ? donor(vs, p[q.s], pc) : 0.0;
            const double div = (fe - fw) * A.G.invdlam + (fnf - fsf) * A.G.invdphi;
            dst[f][q.c] = pc - scale * div;
        }
    }
}

// ---------------------------------------------------------------------------
// 3. coefficients of Eq. 10 from the predictor Phi* = pbase + pinc (Eq. 7;
//    pinc may be null), the explicit momenta X0, Y0 at n+1 and the mass flux
//    F^n + F0 (Eq. 8 inverted in closed form)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pred(const double *base, const double *inc, size_t k)
{
    return inc ? base[k] + inc[k] : base[k];
}

struct CoeffArgs {
    Geom G;
    const double *pbase, *pinc, *h0, *alpha, *qbx, *qby, *qhx, *qhy, *bb, *invD, *qx, *qy;
    double *A11, *A12, *A21, *A22, *B1, *B2, *C;
    double *X0, *Y0, *fsx, *fsy;
};

__global__ void __launch_bounds__(SWE_THREADS) k_swe_coeffs(CoeffArgs A)
{
    const int nx = A.G.nx, ny = A.G.ny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double a = A.G.a, g = A.G.grav, delta = 0.5 * A.G.dt;
    const double hdg = 0.5 * delta * g, hga = 0.5 * g / a;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const Nbr q = neighbours(i, j, nx, ny);
        const double cj = A.G.cosr[j], ic = A.G.invcos[j];
        const double al = A.alpha[q.c];
        const double c = 1.0 + delta * al;
        const double b = A.bb[q.c];
        const double iD = A.invD[q.c];
        const double ps = pred(A.pbase, A.pinc, q.c);
        const double kappa = hdg * ps;
        const double dhl = ((pred(A.pbase, A.pinc, q.e) + A.h0[q.e]) - (pred(A.pbase, A.pinc, q.w) + A.h0[q.w]))
                           * A.G.inv2dlam;
        const double dhp = ((pred(A.pbase, A.pinc, q.n) + A.h0[q.n]) - (pred(A.pbase, A.pinc, q.s) + A.h0[q.s]))
                           * A.G.inv2dphi;
        const double kci = kappa * c * iD, kbi = kappa * b * iD, hgi = hdg * iD;
        A.A11[q.c] = kci * ic;
        A.A12[q.c] = kbi;
        A.A21[q.c] = -kbi;
        A.A22[q.c] = kci * cj;
        A.B1[q.c] = hgi * (c * dhl * ic + b * dhp);
        A.B2[q.c] = hgi * (c * cj * dhp - b * dhl);
        A.C[q.c] = A.G.Crow[j];
        const double d0l = (A.h0[q.e] - A.h0[q.w]) * A.G.inv2dlam;
        const double d0p = (A.h0[q.n] - A.h0[q.s]) * A.G.inv2dphi;
        const double X0 = A.qhx[q.c] + delta * al * A.qbx[q.c] - delta * (0.5 * A.G.gx[j]) * ps * d0l;
        const double Y0 = A.qhy[q.c] + delta * al * A.qby[q.c] - delta * hga * ps * d0p;
        A.X0[q.c] = X0;
        A.Y0[q.c] = Y0;
        A.fsx[q.c] = a * A.qx[q.c] + a * (c * X0 + b * Y0) * iD;
        A.fsy[q.c] = a * cj * A.qy[q.c] + a * cj * (c * Y0 - b * X0) * iD;
    }
}

// ---------------------------------------------------------------------------
// 4. R' = div(F^n + F0) - C Phi^n - L(Phi^n); rhs holds L(Phi^n) on entry
//    and R' on return (same cell, read before written)
// ---------------------------------------------------------------------------
struct RhsArgs {
    Geom G;
    const double *fsx, *fsy, *phi;
    double *rhs;
};

__global__ void __launch_bounds__(SWE_THREADS) k_swe_rhs(RhsArgs A)
{
    const int nx = A.G.nx, ny = A.G.ny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const Nbr q = neighbours(i, j, nx, ny);
        const double xc = A.fsx[q.c], yc = A.fsy[q.c];
        const double fe = 0.5 * (xc + A.fsx[q.e]);
        const double fw = 0.5 * (A.fsx[q.w] + xc);
        const double fn = j + 1 < ny ? 0.5 * (A.fsy[q.n] + yc) : 0.0;
        const double fs = j > 0 ? 0.5 * (yc + A.fsy[q.s]) : 0.0;
        const double div = (fe - fw) * A.G.invdlam + (fn - fs) * A.G.invdphi;
        A.rhs[q.c] = div - A.G.Crow[j] * A.phi[q.c] - A.rhs[q.c];
    }
}

// ---------------------------------------------------------------------------
// 6. Phi^{n+1} = Phi^n + dPhi and the momenta of Eq. 8 with the pressure
//    gradient of Eq. 7
// ---------------------------------------------------------------------------
struct RecoverArgs {
    Geom G;
    const double *phi, *dphi, *pinc, *h0, *alpha, *bb, *invD, *X0, *Y0;   // Phi* = phi + pinc
    double *phi1, *qx1, *qy1;
};

__global__ void __launch_bounds__(SWE_THREADS) k_swe_recover(RecoverArgs A)
{
    const int nx = A.G.nx, ny = A.G.ny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double delta = 0.5 * A.G.dt, hga = 0.5 * A.G.grav / A.G.a;
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const Nbr q = neighbours(i, j, nx, ny);
        const double p1c = A.phi[q.c] + A.dphi[q.c];
        const double p1e = A.phi[q.e] + A.dphi[q.e], p1w = A.phi[q.w] + A.dphi[q.w];
        const double p1n = A.phi[q.n] + A.dphi[q.n], p1s = A.phi[q.s] + A.dphi[q.s];
        const double ps = pred(A.phi, A.pinc, q.c);
        const double dhl = ((pred(A.phi, A.pinc, q.e) + A.h0[q.e]) - (pred(A.phi, A.pinc, q.w) + A.h0[q.w]))
                           * A.G.inv2dlam;
        const double dhp = ((pred(A.phi, A.pinc, q.n) + A.h0[q.n]) - (pred(A.phi, A.pinc, q.s) + A.h0[q.s]))
                           * A.G.inv2dphi;
        const double Px = -(0.5 * A.G.gx[j]) * (p1c * dhl + ps * ((p1e - p1w) * A.G.inv2dlam));
        const double Py = -hga * (p1c * dhp + ps * ((p1n - p1s) * A.G.inv2dphi));
        const double X = A.X0[q.c] + delta * Px;
        const double Y = A.Y0[q.c] + delta * Py;
        const double c = 1.0 + delta * A.alpha[q.c];
        const double b = A.bb[q.c];
        const double iD = A.invD[q.c];
        A.phi1[q.c] = p1c;
        A.qx1[q.c] = (c * X + b * Y) * iD;
        A.qy1[q.c] = (c * Y - b * X) * iD;
    }
}

// ---------------------------------------------------------------------------
// first guess of the predictor solve: the increment extrapolated from the
// last two steps, 2 dPhi^(n-1) - dPhi^(n-2)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_swe_guess(size_t n, const double *d1, const double *d2, double *out)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        out[k] = 2.0 * d1[k] - d2[k];
}

}  // namespace sw

using namespace sw;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
enum SweField {
    F_PHI0, F_PHI1, F_QX0, F_QX1, F_QY0, F_QY1,   // state, double-buffered
    F_UP, F_VP, F_UN, F_VN,                      // winds of levels n-1 and n
    F_H0, F_ALPHA, F_QBX, F_QBY,                 // fixed forcing fields
    F_U, F_V, F_PSX, F_PSY, F_BB, F_IND,         // step 1
    F_QHX, F_QHY,                                // step 2
    F_A11, F_A12, F_A21, F_A22, F_B1, F_B2, F_C, // step 3
    F_X0, F_Y0, F_FSX, F_FSY,
    F_RHS, F_DPH1, F_DPHI,                       // right-hand side, first and second increments
    F_DH1, F_DH2,                                // final increments of the last two steps
    F_COUNT
};

struct sw_swe_s {
    sw_grid grid;
    int nx, ny, sms;
    size_t N;
    sw_swe_params p;
    double radius;
    double *mem = nullptr;       // F_COUNT fields, then the NROWTAB row tables
    double *f[F_COUNT];
    double *rows = nullptr;
    int cur = 0;                 // state buffer holding level n
    bool has_state = false, has_prev = false;
    int n_dhist = 0;             // final increments kept from earlier steps (0..2)
    sw_solve_stats *dstats = nullptr;
    int dstats_n = 0;
};

namespace {

sw_status swe_cuda(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return sw::api_fail(e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA, m.c_str());
}

#define SWE_CK(call)                                               \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return swe_cuda(e_, #call);         \
    } while (0)

constexpr int NROWTAB = 7;   // cos, sin, tan, 1/cos, C, dt/(a^2 cos), g/(a cos)

Geom geom(const sw_swe_s *m)
{
    Geom G;
    const double dlam = 2.0 * M_PI / m->nx, dphi = M_PI / m->ny;
    G.nx = m->nx; G.ny = m->ny; G.a = m->radius;
    G.dt = m->p.dt; G.grav = m->p.gravity; G.omega = m->p.omega;
    G.inv2dlam = 1.0 / (2.0 * dlam); G.inv2dphi = 1.0 / (2.0 * dphi);
    G.invdlam = 1.0 / dlam; G.invdphi = 1.0 / dphi;
    const double *r = m->rows;
    const size_t ny = (size_t)m->ny;
    G.cosr = r; G.sinr = r + ny; G.tanr = r + 2 * ny; G.invcos = r + 3 * ny;
    G.Crow = r + 4 * ny; G.tscale = r + 5 * ny; G.gx = r + 6 * ny;
    return G;
}

dim3 swe_grid(const sw_swe_s *m)
{
    return dim3((unsigned)((m->nx + SWE_THREADS - 1) / SWE_THREADS), (unsigned)(m->ny < 65535 ? m->ny : 65535));
}

double *fld(sw_swe_s *m, int k) { return m->f[k]; }

// steps 1-2 of a step: winds, forcing, transported momenta
sw_status run_forcing(sw_swe m, cudaStream_t s)
{
    const Geom G = geom(m);
    const int c = m->cur;
    ForcingArgs fa{G, fld(m, F_PHI0 + c), fld(m, F_QX0 + c), fld(m, F_QY0 + c), fld(m, F_UP), fld(m, F_VP),
                   fld(m, F_H0), fld(m, F_ALPHA), fld(m, F_QBX), fld(m, F_QBY), m->has_prev ? 1 : 0, fld(m, F_U),
                   fld(m, F_V), fld(m, F_PSX), fld(m, F_PSY), fld(m, F_BB), fld(m, F_IND), fld(m, F_UN),
                   fld(m, F_VN)};
    k_swe_forcing<<<swe_grid(m), SWE_THREADS, 0, s>>>(fa);
    SWE_CK(cudaGetLastError());
    TransportArgs ta{G, fld(m, F_U), fld(m, F_V), fld(m, F_PSX), fld(m, F_PSY), fld(m, F_QHX), fld(m, F_QHY)};
    k_swe_transport<<<swe_grid(m), SWE_THREADS, 0, s>>>(ta);
    SWE_CK(cudaGetLastError());
    return SW_OK;
}

// steps 3-4 for the predictor Phi* = pbase + pinc: coefficients on the grid,
// R' in F_RHS
sw_status run_pass(sw_swe m, const double *pbase, const double *pinc, cudaStream_t s)
{
    const Geom G = geom(m);
    const int c = m->cur;
    const double *phi = fld(m, F_PHI0 + c), *qx = fld(m, F_QX0 + c), *qy = fld(m, F_QY0 + c);
    CoeffArgs ca{G, pbase, pinc, fld(m, F_H0), fld(m, F_ALPHA), fld(m, F_QBX), fld(m, F_QBY), fld(m, F_QHX),
                 fld(m, F_QHY), fld(m, F_BB), fld(m, F_IND), qx, qy, fld(m, F_A11), fld(m, F_A12), fld(m, F_A21), fld(m, F_A22),
                 fld(m, F_B1), fld(m, F_B2), fld(m, F_C), fld(m, F_X0), fld(m, F_Y0), fld(m, F_FSX), fld(m, F_FSY)};
    k_swe_coeffs<<<swe_grid(m), SWE_THREADS, 0, s>>>(ca);
    SWE_CK(cudaGetLastError());
    sw_status st = sw_elliptic_set_coeffs(m->grid, fld(m, F_A11), fld(m, F_A12), fld(m, F_A21), fld(m, F_A22),
                                          fld(m, F_B1), fld(m, F_B2), fld(m, F_C), s);
    if (st) return st;
    st = sw_operator_apply(m->grid, SW_PREC_FP64, phi, fld(m, F_RHS), s);
    if (st) return st;
    RhsArgs ra{G, fld(m, F_FSX), fld(m, F_FSY), phi, fld(m, F_RHS)};
    k_swe_rhs<<<swe_grid(m), SWE_THREADS, 0, s>>>(ra);
    SWE_CK(cudaGetLastError());
    return SW_OK;
}

}  // namespace

extern "C" sw_status sw_swe_create(sw_grid g, const sw_swe_params *p, sw_swe *out)
{
    if (!out) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_create: out is NULL");
    *out = nullptr;
    if (!g || !p) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_create: NULL grid or params");
    if (!(p->dt > 0.0) || !std::isfinite(p->dt) || !(p->gravity > 0.0) || !std::isfinite(p->gravity) ||
        !std::isfinite(p->omega))
        return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_create: dt and gravity must be > 0, omega finite");
    const sw::GridGeom gg = sw::grid_geom(g);
    sw_swe m = new (std::nothrow) sw_swe_s();
    if (!m) return sw::api_fail(SW_ERR_OOM, "sw_swe_create: host allocation failed");
    m->grid = g; m->nx = gg.nx; m->ny = gg.ny; m->sms = gg.sms; m->radius = gg.radius; m->p = *p;
    m->N = (size_t)gg.nx * gg.ny;
    const size_t stride = (m->N + 31) & ~(size_t)31;     // 256-byte aligned fields
    cudaError_t e = cudaMalloc((void **)&m->mem, (F_COUNT * stride + NROWTAB * (size_t)m->ny) * sizeof(double));
    if (e != cudaSuccess) {
        delete m;
        return swe_cuda(e, "sw_swe_create: cudaMalloc");
    }
    for (int k = 0; k < F_COUNT; ++k) m->f[k] = m->mem + k * stride;
    m->rows = m->mem + F_COUNT * stride;
    const size_t ny = (size_t)m->ny;
    std::vector<double> rows(NROWTAB * ny);
    const double dphi = M_PI / m->ny, a = m->radius, delta = 0.5 * p->dt;
    for (size_t j = 0; j < ny; ++j) {
        const double lat = -0.5 * M_PI + (j + 0.5) * dphi;
        const double c = std::cos(lat), sn = std::sin(lat);
        rows[j] = c;
        rows[ny + j] = sn;
        rows[2 * ny + j] = sn / c;
        rows[3 * ny + j] = 1.0 / c;
        rows[4 * ny + j] = (a * a * c) / delta;
        rows[5 * ny + j] = p->dt / (a * a * c);
        rows[6 * ny + j] = p->gravity / (a * c);
    }
    e = cudaMemcpy(m->rows, rows.data(), rows.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->mem, 0, F_COUNT * stride * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(m->mem);
        delete m;
        return swe_cuda(e, "sw_swe_create: initialise");
    }
    *out = m;
    return SW_OK;
}

extern "C" sw_status sw_swe_destroy(sw_swe m)
{
    if (!m) return SW_OK;
    cudaFree(m->mem);
    if (m->dstats) cudaFree(m->dstats);
    delete m;
    return SW_OK;
}

extern "C" sw_status sw_swe_set_state(sw_swe m, const double *Phi, const double *Qx, const double *Qy,
                                      const double *H0, const double *alpha, const double *Qbar_x,
                                      const double *Qbar_y, void *stream)
{
    if (!m || !Phi || !Qx || !Qy) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_set_state: NULL stepper or state");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = m->N * sizeof(double);
    m->cur = 0;
    SWE_CK(cudaMemcpyAsync(fld(m, F_PHI0), Phi, bytes, cudaMemcpyDeviceToDevice, s));
    SWE_CK(cudaMemcpyAsync(fld(m, F_QX0), Qx, bytes, cudaMemcpyDeviceToDevice, s));
    SWE_CK(cudaMemcpyAsync(fld(m, F_QY0), Qy, bytes, cudaMemcpyDeviceToDevice, s));
    const double *opt[4] = {H0, alpha, Qbar_x, Qbar_y};
    const int dst[4] = {F_H0, F_ALPHA, F_QBX, F_QBY};
    for (int k = 0; k < 4; ++k) {
        if (opt[k]) SWE_CK(cudaMemcpyAsync(fld(m, dst[k]), opt[k], bytes, cudaMemcpyDeviceToDevice, s));
        else SWE_CK(cudaMemsetAsync(fld(m, dst[k]), 0, bytes, s));
    }
    m->has_state = true;
    m->has_prev = false;
    m->n_dhist = 0;
    return SW_OK;
}

extern "C" sw_status sw_swe_set_history(sw_swe m, const double *u_prev, const double *v_prev, void *stream)
{
    if (!m || !u_prev || !v_prev) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_set_history: NULL argument");
    if (!m->has_state) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_set_history: no state set");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = m->N * sizeof(double);
    SWE_CK(cudaMemcpyAsync(fld(m, F_UP), u_prev, bytes, cudaMemcpyDeviceToDevice, s));
    SWE_CK(cudaMemcpyAsync(fld(m, F_VP), v_prev, bytes, cudaMemcpyDeviceToDevice, s));
    m->has_prev = true;
    return SW_OK;
}

extern "C" sw_status sw_swe_get_state(sw_swe m, double *Phi, double *Qx, double *Qy, void *stream)
{
    if (!m) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_get_state: NULL stepper");
    if (!m->has_state) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_get_state: no state set");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = m->N * sizeof(double);
    double *dst[3] = {Phi, Qx, Qy};
    const int src[3] = {F_PHI0, F_QX0, F_QY0};
    for (int k = 0; k < 3; ++k)
        if (dst[k]) SWE_CK(cudaMemcpyAsync(dst[k], fld(m, src[k] + m->cur), bytes, cudaMemcpyDeviceToDevice, s));
    return SW_OK;
}

extern "C" sw_status sw_swe_explicit(sw_swe m, const double *phi_star, double *const *coeffs, double *rhs,
                                     void *stream)
{
    if (!m) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_explicit: NULL stepper");
    if (!m->has_state) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_explicit: no state set");
    cudaStream_t s = (cudaStream_t)stream;
    sw_status st = run_forcing(m, s);
    if (st) return st;
    st = run_pass(m, phi_star ? phi_star : fld(m, F_PHI0 + m->cur), nullptr, s);
    if (st) return st;
    const size_t bytes = m->N * sizeof(double);
    if (coeffs)
        for (int k = 0; k < 7; ++k)
            if (coeffs[k]) SWE_CK(cudaMemcpyAsync(coeffs[k], fld(m, F_A11 + k), bytes, cudaMemcpyDeviceToDevice, s));
    if (rhs) SWE_CK(cudaMemcpyAsync(rhs, fld(m, F_RHS), bytes, cudaMemcpyDeviceToDevice, s));
    return SW_OK;
}

extern "C" sw_status sw_swe_step(sw_swe m, const sw_solve_opts *o, int nsteps, sw_solve_stats *stats,
                                 void *stream)
{
    if (!m || !o) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_step: NULL stepper or options");
    if (!m->has_state) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_step: no state set");
    if (nsteps < 1) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_step: nsteps must be >= 1");
    if (o->pc == SW_PC_LEARNED) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_swe_step: SW_PC_LEARNED is not supported");
    cudaStream_t s = (cudaStream_t)stream;
    const int nsolves = 2 * nsteps;
    if (stats && m->dstats_n < nsolves) {
        if (m->dstats) {
            SWE_CK(cudaStreamSynchronize(s));
            SWE_CK(cudaFree(m->dstats));
            m->dstats = nullptr;
            m->dstats_n = 0;
        }
        SWE_CK(cudaMalloc((void **)&m->dstats, (size_t)nsolves * sizeof(sw_solve_stats)));
        m->dstats_n = nsolves;
    }
    const size_t bytes = m->N * sizeof(double);
    const Geom G = geom(m);
    const double *R = fld(m, F_RHS);
    for (int k = 0; k < nsteps; ++k) {
        const int c = m->cur, n = 1 - c;
        const double *phi = fld(m, F_PHI0 + c);
        sw_status st = run_forcing(m, s);
        if (st) return st;
        // predictor pass: Phi* = Phi^n, increment from zero
        st = run_pass(m, phi, nullptr, s);
        if (st) return st;
        // first guess: the increment extrapolated from the last two steps
        double *d1 = fld(m, F_DPH1), *d2 = fld(m, F_DPHI);
        if (m->n_dhist >= 2) {
            k_swe_guess<<<m->sms * 4, 256, 0, s>>>(m->N, fld(m, F_DH1), fld(m, F_DH2), d1);
            SWE_CK(cudaGetLastError());
        } else if (m->n_dhist == 1) {
            SWE_CK(cudaMemcpyAsync(d1, fld(m, F_DH1), bytes, cudaMemcpyDeviceToDevice, s));
        } else {
            SWE_CK(cudaMemsetAsync(d1, 0, bytes, s));
        }
        st = sw_ensemble_solve_async(1, &m->grid, o, &R, &d1, stats ? m->dstats + 2 * k : nullptr, s);
        if (st) return st;
        // corrector pass: Phi* = Phi^n + dPhi_1, increment warm-started from dPhi_1
        st = run_pass(m, phi, d1, s);
        if (st) return st;
        SWE_CK(cudaMemcpyAsync(d2, d1, bytes, cudaMemcpyDeviceToDevice, s));
        st = sw_ensemble_solve_async(1, &m->grid, o, &R, &d2, stats ? m->dstats + 2 * k + 1 : nullptr, s);
        if (st) return st;
        RecoverArgs ra{G, phi, d2, d1, fld(m, F_H0), fld(m, F_ALPHA), fld(m, F_BB), fld(m, F_IND), fld(m, F_X0),
                       fld(m, F_Y0),
                       fld(m, F_PHI0 + n), fld(m, F_QX0 + n), fld(m, F_QY0 + n)};
        k_swe_recover<<<swe_grid(m), SWE_THREADS, 0, s>>>(ra);
        SWE_CK(cudaGetLastError());
        m->cur = n;
        // the applied increment becomes the newest history entry (pointer rotation)
        double *h2 = m->f[F_DH2];
        m->f[F_DH2] = m->f[F_DH1];
        m->f[F_DH1] = m->f[F_DPHI];
        m->f[F_DPHI] = h2;
        if (m->n_dhist < 2) ++m->n_dhist;
        double *t = m->f[F_UP]; m->f[F_UP] = m->f[F_UN]; m->f[F_UN] = t;
        t = m->f[F_VP]; m->f[F_VP] = m->f[F_VN]; m->f[F_VN] = t;
        m->has_prev = true;
    }
    if (stats) {
        SWE_CK(cudaMemcpyAsync(stats, m->dstats, (size_t)nsolves * sizeof(sw_solve_stats), cudaMemcpyDeviceToHost, s));
        SWE_CK(cudaStreamSynchronize(s));
    }
    return SW_OK;
}
