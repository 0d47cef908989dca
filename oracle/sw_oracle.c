/*
 * sw_oracle.c -- plain, slow, FP64 CPU oracle of the preconditioned GCR(k)
 * elliptic solve of Ackmann, Dueben, Palmer & Smolarkiewicz (2021),
 * "Mixed-precision for linear solvers in global geophysical flows".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file; the library never does.  It
 * shares no code with the CUDA path.
 *
 * What it computes, and where it comes from:
 *   swo_operator      generalised Laplacian L (Eq. 10) in compact flux form
 *   swo_apply_PZ      zonal second-derivative part P^Z of L (Sec. 2.3, Eq. 13)
 *   swo_apply_PM      the remainder P^M = L - (P^Z - P^H), P^H = C (Eq. 13)
 *   swo_diag_L        the diagonal D of L (preconditioner option 1, Sec. 2.3)
 *   swo_eta_auto      pseudo-time step eta from the stability of the lagged P^M
 *   swo_cyclic_solve  cyclic (periodic) tridiagonal solve, Sherman-Morrison
 *   swo_precond       preconditioner options 0-3 (Sec. 2.3, Eq. 13)
 *   swo_gcr           preconditioned GCR(k) with restarts, exit test Eq. 12,
 *                     residual Eq. 11, optional true-residual replacement
 *
 * Readings of points the paper leaves open (the discrete stencil, the pole
 * treatment, eta, the cyclic wrap, the GCR restart):
 *   - flux form: L x = (Fx[i+1/2] - Fx[i-1/2])/dlam + (Fy[j+1/2] - Fy[j-1/2])/dphi - C x,
 *       Fx[i+1/2,j] = a11 (x[i+1,j]-x[i,j])/dlam
 *                   + a12 (x[i,j+1]+x[i+1,j+1]-x[i,j-1]-x[i+1,j-1])/(4 dphi)
 *                   + b1 (x[i,j]+x[i+1,j])/2,
 *       Fy[i,j+1/2] = a22 (x[i,j+1]-x[i,j])/dphi
 *                   + a21 (x[i+1,j]+x[i+1,j+1]-x[i-1,j]-x[i-1,j+1])/(4 dlam)
 *                   + b2 (x[i,j]+x[i,j+1])/2,
 *     face coefficients (a11 ...) are means of the two adjacent cell values;
 *   - periodic in longitude; Fy = 0 on the two pole faces (h_x = a cos(phi)
 *     vanishes there); the row beyond a pole is the pole row shifted by half
 *     a circle, x[i,-1] = x[i+nx/2,0] and x[i,ny] = x[i+nx/2,ny-1] (even nx);
 *   - eta = 1 / max |diag(P^M)| unless given;
 *   - the zonal problem of Eq. 13 is cyclic (periodic longitude) and is solved
 *     exactly;
 *   - GCR restart keeps the last direction: p_0 <- p_k, L(p_0) <- L(p_k);
 *   - exit when ||r|| <= eps ||R|| (equal to Eq. 12 for a zero first guess)
 *     and at least min_iters iterations were done; the residual that decides
 *     is always the true residual L(Phi) - R recomputed from Phi (Sec. 4).
 *
 * Fields are [ny][nx] row-major, longitude fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny;
    const double *A11, *A12, *A21, *A22, *B1, *B2, *C;
} swo_problem;

typedef struct {
    int k;          /* GCR(k): directions kept before a restart */
    double tol;     /* eps of the exit condition, relative to ||R|| */
    int max_iters;
    int min_iters;
    int pc;         /* preconditioner option 0..3 */
    int n_rich;     /* Richardson iterations for options 2 and 3 */
    double eta;     /* pseudo time step of option 3 (<= 0: automatic) */
    double omega;   /* relaxation of option 2 */
    int ru_every;   /* recompute the true residual every ru_every iterations (0: never) */
} swo_opts;

typedef struct {
    int iterations;
    int converged;
    int status;     /* 0 ok, 4 not converged, 5 breakdown */
    double r0_norm;
    double R_norm;
    double true_rel_residual;
    double recursive_rel_residual;
    double eta_used;
} swo_stats;

#define PI 3.14159265358979323846

static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* x at (i, j) with periodic longitude and the across-pole continuation. */
static inline double xat(const swo_problem *P, const double *x, int i, int j)
{
    int nx = P->nx, ny = P->ny;
    if (j < 0)        { j = 0;      i += nx / 2; }
    else if (j >= ny) { j = ny - 1; i += nx / 2; }
    return x[(size_t)j * nx + wrapi(i, nx)];
}

static inline double cat(const double *c, int nx, int i, int j)
{
    return c[(size_t)j * nx + wrapi(i, nx)];
}

/* zonal flux through the face (i+1/2, j) */
static double flux_x(const swo_problem *P, const double *x, int i, int j,
                     double dlam, double dphi)
{
    int nx = P->nx;
    double a11 = 0.5 * (cat(P->A11, nx, i, j) + cat(P->A11, nx, i + 1, j));
    double a12 = 0.5 * (cat(P->A12, nx, i, j) + cat(P->A12, nx, i + 1, j));
    double b1  = 0.5 * (cat(P->B1,  nx, i, j) + cat(P->B1,  nx, i + 1, j));
    double dxl = (xat(P, x, i + 1, j) - xat(P, x, i, j)) / dlam;
    double dxp = (xat(P, x, i, j + 1) + xat(P, x, i + 1, j + 1)
                - xat(P, x, i, j - 1) - xat(P, x, i + 1, j - 1)) / (4.0 * dphi);
    double xm  = 0.5 * (xat(P, x, i, j) + xat(P, x, i + 1, j));
    return a11 * dxl + a12 * dxp + b1 * xm;
}

/* meridional flux through the face (i, j+1/2); zero on the pole faces */
static double flux_y(const swo_problem *P, const double *x, int i, int j,
                     double dlam, double dphi)
{
    int nx = P->nx, ny = P->ny;
    if (j < 0 || j >= ny - 1) return 0.0;
    double a22 = 0.5 * (cat(P->A22, nx, i, j) + cat(P->A22, nx, i, j + 1));
    double a21 = 0.5 * (cat(P->A21, nx, i, j) + cat(P->A21, nx, i, j + 1));
    double b2  = 0.5 * (cat(P->B2,  nx, i, j) + cat(P->B2,  nx, i, j + 1));
    double dxp = (xat(P, x, i, j + 1) - xat(P, x, i, j)) / dphi;
    double dxl = (xat(P, x, i + 1, j) + xat(P, x, i + 1, j + 1)
                - xat(P, x, i - 1, j) - xat(P, x, i - 1, j + 1)) / (4.0 * dlam);
    double xm  = 0.5 * (xat(P, x, i, j) + xat(P, x, i, j + 1));
    return a22 * dxp + a21 * dxl + b2 * xm;
}

/* Eq. 10:  y = L(x) = sum_I d/dx^I (sum_J A^IJ dx/dx^J + B^I x) - C x */
void swo_operator(const swo_problem *P, const double *x, double *y)
{
    int nx = P->nx, ny = P->ny;
    double dlam = 2.0 * PI / nx, dphi = PI / ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double dfx = flux_x(P, x, i, j, dlam, dphi) - flux_x(P, x, i - 1, j, dlam, dphi);
            double dfy = flux_y(P, x, i, j, dlam, dphi) - flux_y(P, x, i, j - 1, dlam, dphi);
            size_t id = (size_t)j * nx + i;
            y[id] = dfx / dlam + dfy / dphi - P->C[id] * x[id];
        }
}

/* zonal part P^Z: the A11 second-derivative term of Eq. 10 */
void swo_apply_PZ(const swo_problem *P, const double *x, double *y)
{
    int nx = P->nx, ny = P->ny;
    double dlam = 2.0 * PI / nx;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double ae = 0.5 * (cat(P->A11, nx, i, j) + cat(P->A11, nx, i + 1, j));
            double aw = 0.5 * (cat(P->A11, nx, i - 1, j) + cat(P->A11, nx, i, j));
            double xe = xat(P, x, i + 1, j), xc = xat(P, x, i, j), xw = xat(P, x, i - 1, j);
            y[(size_t)j * nx + i] = (ae * (xe - xc) - aw * (xc - xw)) / (dlam * dlam);
        }
}

/* P^M is what remains of L once the implicit part P^Z - P^H is removed (Eq. 13):
 * P^M x = L x - P^Z x + C x */
void swo_apply_PM(const swo_problem *P, const double *x, double *y)
{
    size_t n = (size_t)P->nx * P->ny;
    double *t = malloc(n * sizeof(double));
    swo_operator(P, x, y);
    swo_apply_PZ(P, x, t);
    for (size_t id = 0; id < n; ++id) y[id] = y[id] - t[id] + P->C[id] * x[id];
    free(t);
}

/* diagonal of L: the coefficient of x[i,j] in (L x)[i,j] */
void swo_diag_L(const swo_problem *P, double *d)
{
    int nx = P->nx, ny = P->ny;
    double dlam = 2.0 * PI / nx, dphi = PI / ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double a11e = 0.5 * (cat(P->A11, nx, i, j) + cat(P->A11, nx, i + 1, j));
            double a11w = 0.5 * (cat(P->A11, nx, i - 1, j) + cat(P->A11, nx, i, j));
            double b1e  = 0.5 * (cat(P->B1, nx, i, j) + cat(P->B1, nx, i + 1, j));
            double b1w  = 0.5 * (cat(P->B1, nx, i - 1, j) + cat(P->B1, nx, i, j));
            double zonal = (-a11e / dlam + 0.5 * b1e - (a11w / dlam + 0.5 * b1w)) / dlam;
            double merid = 0.0;
            if (j < ny - 1) {   /* north face */
                double a22n = 0.5 * (cat(P->A22, nx, i, j) + cat(P->A22, nx, i, j + 1));
                double b2n  = 0.5 * (cat(P->B2, nx, i, j) + cat(P->B2, nx, i, j + 1));
                merid += (-a22n / dphi + 0.5 * b2n) / dphi;
            }
            if (j > 0) {        /* south face */
                double a22s = 0.5 * (cat(P->A22, nx, i, j - 1) + cat(P->A22, nx, i, j));
                double b2s  = 0.5 * (cat(P->B2, nx, i, j - 1) + cat(P->B2, nx, i, j));
                merid -= (a22s / dphi + 0.5 * b2s) / dphi;
            }
            size_t id = (size_t)j * nx + i;
            d[id] = zonal + merid - P->C[id];
        }
}

/* eta = 1 / max |diag(P^M)|, diag(P^M) = diag(L) - diag(P^Z) + C:
 * the forward-Euler step limit for the lagged (explicit) part of Eq. 13 */
double swo_eta_auto(const swo_problem *P)
{
    int nx = P->nx, ny = P->ny;
    double dlam = 2.0 * PI / nx;
    size_t n = (size_t)nx * ny;
    double *d = malloc(n * sizeof(double));
    swo_diag_L(P, d);
    double m = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double ae = 0.5 * (cat(P->A11, nx, i, j) + cat(P->A11, nx, i + 1, j));
            double aw = 0.5 * (cat(P->A11, nx, i - 1, j) + cat(P->A11, nx, i, j));
            size_t id = (size_t)j * nx + i;
            double dpm = d[id] + (ae + aw) / (dlam * dlam) + P->C[id];
            if (fabs(dpm) > m) m = fabs(dpm);
        }
    free(d);
    return m > 0.0 ? 1.0 / m : 1.0;
}

/* Tridiagonal solve without pivoting (the matrices here are strictly
 * diagonally dominant):  a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i],
 * a[0] and c[n-1] ignored. */
static void thomas(int n, const double *a, const double *b, const double *c,
                   const double *d, double *x, double *cp, double *dp)
{
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; ++i) {
        double m = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / m;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* Cyclic tridiagonal solve, n >= 3:
 *   sub[i] x[i-1] + diag[i] x[i] + sup[i] x[i+1] = rhs[i],  indices mod n
 * (sub[0] couples x[0] to x[n-1], sup[n-1] couples x[n-1] to x[0]).
 * Sherman-Morrison: T = T' + u v^T with gamma = -diag[0],
 * u = (gamma, 0, .., 0, sup[n-1]), v = (1, 0, .., 0, sub[0]/gamma), T' the
 * plain tridiagonal part with diag'[0] = diag[0] - gamma and
 * diag'[n-1] = diag[n-1] - sub[0] sup[n-1] / gamma;
 * x = y - z (v.y)/(1 + v.z) with T' y = rhs, T' z = u. */
void swo_cyclic_solve(int n, const double *sub, const double *diag, const double *sup,
                      const double *rhs, double *x)
{
    double *bb = malloc(6 * (size_t)n * sizeof(double));
    double *u = bb + n, *z = bb + 2 * n, *y = bb + 3 * n, *cp = bb + 4 * n, *dp = bb + 5 * n;
    double gamma = -diag[0];
    memcpy(bb, diag, n * sizeof(double));
    bb[0] = diag[0] - gamma;
    bb[n - 1] = diag[n - 1] - sub[0] * sup[n - 1] / gamma;
    thomas(n, sub, bb, sup, rhs, y, cp, dp);
    for (int i = 0; i < n; ++i) u[i] = 0.0;
    u[0] = gamma;
    u[n - 1] = sup[n - 1];
    thomas(n, sub, bb, sup, u, z, cp, dp);
    double vy = y[0] + sub[0] / gamma * y[n - 1];
    double vz = z[0] + sub[0] / gamma * z[n - 1];
    double f = vy / (1.0 + vz);
    for (int i = 0; i < n; ++i) x[i] = y[i] - f * z[i];
    free(bb);
}

/* Row j of T = I - eta (P^Z - P^H), the implicit zonal operator of Eq. 13. */
void swo_row_T(const swo_problem *P, int j, double eta, double *sub, double *diag, double *sup)
{
    int nx = P->nx;
    double dlam = 2.0 * PI / nx, s = eta / (dlam * dlam);
    for (int i = 0; i < nx; ++i) {
        double ae = 0.5 * (cat(P->A11, nx, i, j) + cat(P->A11, nx, i + 1, j));
        double aw = 0.5 * (cat(P->A11, nx, i - 1, j) + cat(P->A11, nx, i, j));
        sub[i] = -s * aw;
        sup[i] = -s * ae;
        diag[i] = 1.0 + s * (ae + aw) + eta * P->C[(size_t)j * nx + i];
    }
}

/* Solve T q = b row by row (Eq. 13, left-hand side). */
static void solve_T(const swo_problem *P, double eta, const double *b, double *q)
{
    int nx = P->nx, ny = P->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        double *w = malloc(3 * (size_t)nx * sizeof(double));
        swo_row_T(P, j, eta, w, w + nx, w + 2 * nx);
        swo_cyclic_solve(nx, w, w + nx, w + 2 * nx, b + (size_t)j * nx, q + (size_t)j * nx);
        free(w);
    }
}

/* q ~ L^{-1} r by the preconditioner option o->pc (Sec. 2.3):
 *   0: q = r                         (P = I)
 *   1: q = D^{-1} r                  (P = D, the diagonal of L)
 *   2: q_0 = 0, q_{mu+1} = q_mu + omega D^{-1} (r - L q_mu),  n_rich times
 *   3: q_0 = 0, [I - eta (P^Z - P^H)] q_{mu+1} = q_mu + eta (P^M q_mu - r),  n_rich times
 */
void swo_precond(const swo_problem *P, const swo_opts *o, double eta,
                 const double *r, double *q)
{
    size_t n = (size_t)P->nx * P->ny;
    if (o->pc == 0) { memcpy(q, r, n * sizeof(double)); return; }
    double *d = malloc(n * sizeof(double));
    double *t = malloc(n * sizeof(double));
    if (o->pc == 1) {
        swo_diag_L(P, d);
        for (size_t id = 0; id < n; ++id) q[id] = r[id] / d[id];
    } else if (o->pc == 2) {
        swo_diag_L(P, d);
        for (size_t id = 0; id < n; ++id) q[id] = 0.0;
        for (int mu = 0; mu < o->n_rich; ++mu) {
            swo_operator(P, q, t);
            for (size_t id = 0; id < n; ++id) q[id] += o->omega * (r[id] - t[id]) / d[id];
        }
    } else {
        for (size_t id = 0; id < n; ++id) q[id] = 0.0;
        for (int mu = 0; mu < o->n_rich; ++mu) {
            swo_apply_PM(P, q, t);
            for (size_t id = 0; id < n; ++id) d[id] = q[id] + eta * (t[id] - r[id]);
            solve_T(P, eta, d, q);
        }
    }
    free(d);
    free(t);
}

static double dot(size_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* r = L(phi) - R   (Eq. 11) */
static void residual(const swo_problem *P, const double *phi, const double *R, double *r)
{
    size_t n = (size_t)P->nx * P->ny;
    swo_operator(P, phi, r);
    for (size_t i = 0; i < n; ++i) r[i] -= R[i];
}

/*
 * Preconditioned GCR(k) (Sec. 2.3; Eisenstat et al. 1983):
 *   r_0 = L(Phi_0) - R;  p_0 = P^{-1}(r_0);  compute L(p_0)
 *   for nu = 0 .. k-1:
 *     beta = -<r_nu, L p_nu> / <L p_nu, L p_nu>
 *     Phi_{nu+1} = Phi_nu + beta p_nu;   r_{nu+1} = r_nu + beta L p_nu
 *     exit test (Eq. 12)
 *     e = P^{-1}(r_{nu+1});  compute L(e)
 *     alpha_l = -<L e, L p_l> / <L p_l, L p_l>,   l = 0..nu
 *     p_{nu+1} = e + sum_l alpha_l p_l;   L p_{nu+1} = L e + sum_l alpha_l L p_l
 *   restart with p_0 <- p_k, L p_0 <- L p_k.
 * The residual is replaced by the true one, L(Phi) - R, when the recursive
 * one meets the tolerance, every ru_every iterations and at max_iters.
 * hist (optional, max_iters+1 entries): ||r|| / ||R|| after each iteration
 * (entry 0: the initial residual).  orth (optional, max_iters entries): the
 * largest |cos| between the new L p_{nu+1} and the earlier L p_l of the cycle.
 */
int swo_gcr(const swo_problem *P, const swo_opts *o, const double *R, double *phi,
            swo_stats *st, double *hist, double *orth)
{
    size_t n = (size_t)P->nx * P->ny;
    int k = o->k, it = 0, nu = 0;
    memset(st, 0, sizeof(*st));
    double eta = o->eta > 0.0 ? o->eta : swo_eta_auto(P);
    st->eta_used = eta;
    double nR = sqrt(dot(n, R, R));
    st->R_norm = nR;
    if (nR == 0.0) {
        memset(phi, 0, n * sizeof(double));
        st->converged = 1;
        if (hist) hist[0] = 0.0;
        return 0;
    }
    double *r = malloc(n * sizeof(double));
    double *e = malloc(n * sizeof(double));
    double *Le = malloc(n * sizeof(double));
    double *p = malloc((size_t)(k + 1) * n * sizeof(double));
    double *Lp = malloc((size_t)(k + 1) * n * sizeof(double));
    double *alpha = malloc((size_t)(k + 1) * sizeof(double));

    residual(P, phi, R, r);
    double rn = sqrt(dot(n, r, r));
    st->r0_norm = rn;
    st->true_rel_residual = st->recursive_rel_residual = rn / nR;
    if (hist) hist[0] = rn / nR;
    if (rn <= o->tol * nR && o->min_iters <= 0) {
        st->converged = 1;
        goto done;
    }
    swo_precond(P, o, eta, r, p);
    swo_operator(P, p, Lp);

    for (;;) {
        double *pn = p + (size_t)nu * n, *Lpn = Lp + (size_t)nu * n;
        double LpLp = dot(n, Lpn, Lpn);
        if (!(LpLp > 0.0)) { st->status = 5; break; }
        double beta = -dot(n, r, Lpn) / LpLp;
        for (size_t i = 0; i < n; ++i) { phi[i] += beta * pn[i]; r[i] += beta * Lpn[i]; }
        ++it;
        rn = sqrt(dot(n, r, r));
        st->recursive_rel_residual = rn / nR;
        int is_true = 0;
        if ((rn <= o->tol * nR && it >= o->min_iters) ||
            (o->ru_every > 0 && it % o->ru_every == 0) || it >= o->max_iters) {
            residual(P, phi, R, r);
            rn = sqrt(dot(n, r, r));
            is_true = 1;
        }
        if (hist) hist[it] = rn / nR;
        if (is_true) st->true_rel_residual = rn / nR;
        if (is_true && rn <= o->tol * nR && it >= o->min_iters) { st->converged = 1; break; }
        if (it >= o->max_iters) { st->status = 4; break; }

        swo_precond(P, o, eta, r, e);
        swo_operator(P, e, Le);
        for (int l = 0; l <= nu; ++l) {
            double *Lpl = Lp + (size_t)l * n;
            alpha[l] = -dot(n, Le, Lpl) / dot(n, Lpl, Lpl);
        }
        double *pnew = p + (size_t)(nu + 1) * n, *Lpnew = Lp + (size_t)(nu + 1) * n;
        for (size_t i = 0; i < n; ++i) {
            double sp = e[i], sl = Le[i];
            for (int l = 0; l <= nu; ++l) {
                sp += alpha[l] * p[(size_t)l * n + i];
                sl += alpha[l] * Lp[(size_t)l * n + i];
            }
            pnew[i] = sp;
            Lpnew[i] = sl;
        }
        if (orth) {
            double m = 0.0, nn = sqrt(dot(n, Lpnew, Lpnew));
            for (int l = 0; l <= nu; ++l) {
                double *Lpl = Lp + (size_t)l * n;
                double c = fabs(dot(n, Lpnew, Lpl)) / (nn * sqrt(dot(n, Lpl, Lpl)));
                if (c > m) m = c;
            }
            orth[it - 1] = m;
        }
        ++nu;
        if (nu == k) {
            memcpy(p, p + (size_t)k * n, n * sizeof(double));
            memcpy(Lp, Lp + (size_t)k * n, n * sizeof(double));
            nu = 0;
        }
    }
done:
    st->iterations = it;
    free(r); free(e); free(Le); free(p); free(Lp); free(alpha);
    return st->status;
}

/* Round x to p significand bits (p counts the explicit fraction bits, so p = 10
 * is IEEE half's precision and p = 23 single's), round-to-nearest-even, with
 * an unbounded exponent: the reduced-precision emulation of Sec. 3.4, which
 * keeps double's exponent range. */
double swo_round_bits(double x, int p)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int ex;
    double m = frexp(x, &ex);                 /* x = m 2^ex, 0.5 <= |m| < 1 */
    double s = ldexp(m, p + 1);               /* p+1 significant bits before the point */
    double r = nearbyint(s);                  /* default mode: nearest, ties to even */
    return ldexp(r, ex - p - 1);
}

/* Host threads of the OpenMP row loops (timing only: the row loops and their
 * fixed-order per-row partial sums give the same results for any count). */
#ifdef _OPENMP
#include <omp.h>
#endif
void swo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
