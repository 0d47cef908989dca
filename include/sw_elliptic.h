/*
 * sw_elliptic.h -- C ABI of the GB300 elliptic solver for the semi-implicit
 * shallow-water model on the longitude/latitude sphere.
 *
 * The library solves the Helmholtz problem of Eq. 9,
 *     L(Phi) - R = 0,
 *     L(Phi) = sum_I d/dx^I ( sum_J A^IJ dPhi/dx^J + B^I Phi ) - C Phi   (Eq. 10),
 * with the preconditioned generalised conjugate residual method GCR(k)
 * (Sec. 2.3) and the preconditioners of Sec. 2.3 (option 3: the
 * semi-implicit Richardson iteration of Eq. 13).
 *
 * Grid.  nx longitudes lambda_i = 2 pi i / nx (periodic), ny latitudes
 * phi_j = -pi/2 + (j + 1/2) pi / ny (rows half a cell from the poles).
 * Every field is a dense [ny][nx] row-major array, longitude fastest.
 *
 * Discretisation (the paper does not print it; this library's reading):
 * compact flux form, face coefficients are means of the two adjacent cell
 * values, zero meridional flux through the two pole faces, and the row beyond
 * a pole is the pole row shifted by nx/2 (hence nx must be even).
 *
 * Conventions for every call:
 *  - pointers to fields are DEVICE pointers owned by the caller, unless a
 *    comment says "host";
 *  - `stream` is a cudaStream_t (NULL = legacy default stream); every call is
 *    ordered on it, and only sw_gcr_solve / sw_ensemble_solve (to fill their
 *    host-side stats) and sw_elliptic_set_coeffs (to read back the automatic
 *    eta) synchronise it;
 *  - errors are reported by the returned status only, never by exceptions or
 *    aborts; sw_last_error() gives a message for the calling thread;
 *  - a grid handle must not be used by two host threads at once.
 */
#ifndef SW_ELLIPTIC_H
#define SW_ELLIPTIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sw_grid_s *sw_grid;    /* opaque, owned by the library */

typedef enum {
    SW_OK = 0,
    SW_ERR_INVALID_ARG = 1,    /* bad size, pointer, option or state */
    SW_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SW_ERR_OOM = 3,            /* device allocation failed */
    SW_ERR_NOT_CONVERGED = 4,  /* max_iters reached; stats are filled in */
    SW_ERR_BREAKDOWN = 5,      /* <L p, L p> not positive: GCR cannot continue */
    SW_ERR_NONFINITE = 6,      /* NaN or Inf in a residual norm */
    SW_ERR_TIMEOUT = 7,        /* a bounded device-side wait ran out */
    SW_ERR_INTERNAL = 8
} sw_status;

/* Precision layouts of the solver (Sec. 4.2-4.3 describe the paper's own
 * CPU/emulator choices; these are this library's GB300 layouts). */
typedef enum {
    SW_PREC_FP64 = 0,        /* everything in FP64 */
    SW_PREC_MIXED_FP16 = 1,  /* preconditioner in FP16 storage / FP32 math with
                                per-row scaling, operator and recursive residual
                                in FP32, FP64 reductions, Phi and true residual */
    SW_PREC_MIXED_BF16 = 2,  /* as MIXED_FP16 with BF16 storage in the preconditioner */
    SW_PREC_FP32 = 3         /* sw_operator_apply only: FP32 x and y */
} sw_precision;

/* Preconditioner options of Sec. 2.3. */
typedef enum {
    SW_PC_NONE = 0,             /* option 0: P = I */
    SW_PC_DIAG = 1,             /* option 1: P = D, the diagonal of L */
    SW_PC_DIAG_RICHARDSON = 2,  /* option 2: diagonally preconditioned explicit Richardson */
    SW_PC_SI_RICHARDSON = 3     /* option 3: semi-implicit Richardson, Eq. 13 */
} sw_precond_kind;

typedef struct {
    int k;               /* GCR(k): directions kept before a restart (1..8) */
    double tol;          /* exit when ||L(Phi) - R||_2 <= tol ||R||_2 (Eq. 12 with
                            ||R|| in place of ||r_0||; equal for a zero first guess) */
    int max_iters;       /* >= 1 */
    int min_iters;       /* iterations done before the exit test may stop (the
                            paper forces one full GCR(3) cycle) */
    int pc;              /* sw_precond_kind */
    int n_richardson;    /* Richardson iterations, options 2 and 3 (1..16) */
    double eta;          /* option 3 pseudo time step; <= 0: the grid's automatic
                            eta = 1 / max|diag(P^M)| set by sw_elliptic_set_coeffs */
    double omega;        /* option 2 relaxation factor */
    int prec;            /* sw_precision (FP64 or MIXED_*) */
    int pole_band_rows;  /* mixed precision: rows next to each pole whose
                            preconditioner runs in FP32 (Sec. 4.3); -1: automatic */
    int ru_every;        /* recompute the true residual every ru_every
                            iterations (0: only when the exit test is met) */
    int threads_per_row; /* launch shape: threads of the block that works on one
                            latitude row (multiple of 32, <= 256); 0: automatic */
    double *res_history; /* device, optional (NULL): max_iters+1 doubles, the
                            relative residual after each iteration (entry 0:
                            the initial one), NaN where not reached */
    double *row_residual;/* device, optional (NULL): ny doubles, the final true
                            residual's 2-norm per latitude row */
} sw_solve_opts;

typedef struct {
    int iterations;
    int converged;                 /* 1 if the true residual met tol */
    int status;                    /* sw_status of this solve */
    int fallbacks;                 /* reserved (learned preconditioner) */
    double r0_norm;                /* ||L(Phi_0) - R||_2 */
    double R_norm;                 /* ||R||_2 */
    double true_rel_residual;      /* ||L(Phi) - R|| / ||R|| at exit, FP64 */
    double recursive_rel_residual; /* the GCR recursive residual at exit */
    double eta;                    /* eta used by option 3 */
} sw_solve_stats;

/* Fills *o with the defaults: k = 4, tol = 1e-8, max_iters = 1000,
 * min_iters = 0, option 3 with 2 Richardson iterations, automatic eta,
 * omega = 1, FP64, automatic pole band, no periodic true residual. */
void sw_solve_opts_default(sw_solve_opts *o);

/* Create a grid of nx x ny points on a sphere of the given radius (m).
 * nx even, 4 <= nx <= 4096, 2 <= ny <= 65536.  The grid takes the current
 * CUDA device.  Allocates the coefficient storage. */
sw_status sw_grid_create(int nx, int ny, double radius, sw_grid *out);
sw_status sw_grid_destroy(sw_grid g);

/* Workspace needed by a solve with options o (NULL: defaults). */
sw_status sw_grid_workspace_bytes(sw_grid g, const sw_solve_opts *o, size_t *bytes);
/* Lend the grid a caller-owned device buffer (256-byte aligned) for solver
 * workspace; it must stay valid until detached (dev_ptr = NULL) or the grid
 * is destroyed.  Without one the grid allocates its own on first use. */
sw_status sw_grid_attach_workspace(sw_grid g, void *dev_ptr, size_t bytes);

/* Give the grid the seven cell-centred coefficient fields of Eq. 10 (device,
 * FP64, [ny][nx]).  The library copies what it needs (face coefficients in
 * FP64 and FP32, the diagonal of L, and the factorised zonal operators of
 * Eq. 13) and computes the automatic eta = 1/max|diag(P^M)|. */
sw_status sw_elliptic_set_coeffs(sw_grid g, const double *A11, const double *A12,
                                 const double *A21, const double *A22,
                                 const double *B1, const double *B2,
                                 const double *C, void *stream);

/* Set eta explicitly (eta > 0) or return to the automatic value (eta <= 0);
 * refactorises the zonal operators.  Needs coefficients. */
sw_status sw_grid_set_eta(sw_grid g, double eta, void *stream);
/* The eta currently in use (host). */
sw_status sw_grid_get_eta(sw_grid g, double *eta);

/* y = L(x) (Eq. 10).  prec SW_PREC_FP64: x, y are double; SW_PREC_FP32: float
 * (FP32 coefficients and arithmetic).  x and y must not overlap. */
sw_status sw_operator_apply(sw_grid g, int prec, const void *x, void *y, void *stream);

/* q = P^{-1}(r), the preconditioner o->pc with o->n_richardson iterations
 * (Sec. 2.3, Eq. 13).  FP64 when o->prec is SW_PREC_FP64 (r, q double),
 * otherwise r and q are float and the sweeps use o->prec's 16-bit storage.
 * r and q must not overlap. */
sw_status sw_precond_apply(sw_grid g, const sw_solve_opts *o, const void *r, void *q,
                           void *stream);

/* Solve L(Phi) = R by preconditioned GCR(k).  R: device FP64; phi: device
 * FP64, the first guess on entry and the solution on return.  stats: host,
 * may be NULL.  Returns SW_OK when converged, SW_ERR_NOT_CONVERGED when
 * max_iters was reached (phi then holds the last iterate).  A zero R gives
 * phi = 0 after 0 iterations. */
sw_status sw_gcr_solve(sw_grid g, const sw_solve_opts *o, const double *R, double *phi,
                       sw_solve_stats *stats, void *stream);

/* Solve n (1..480) independent problems (grids may differ in size) in one persistent
 * launch; each member stops at its own convergence.  grids, R, phi and stats
 * are host arrays of n entries (R[m], phi[m] device pointers).  The grids must
 * be distinct.  Returns the first non-OK member status, else SW_OK. */
sw_status sw_ensemble_solve(int n, const sw_grid *grids, const sw_solve_opts *o,
                            const double *const *R, double *const *phi,
                            sw_solve_stats *stats, void *stream);

/* Size of the fixed device scratch used by sw_gcr_solve_noalloc. */
#define SW_NOALLOC_SCRATCH_BYTES (16u << 20)

/* sw_gcr_solve without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory in the
 * middle of their time step.  Examples are a model that has already handed
 * all of its device memory to its own pool, and a pipeline that must not
 * stall: cudaMalloc and cudaFree can synchronise the whole device.
 *
 * Arguments, results, statuses and the solution are those of sw_gcr_solve with
 * the same grid and options.  The difference is where the solver's work
 * vectors live.  They are not in the grid's workspace, and nothing is
 * allocated for them.  They go in one fixed array of SW_NOALLOC_SCRATCH_BYTES
 * per device, built into the library and shared by every grid on that device.
 * The call makes no device or pinned-host allocation of any kind.  On a
 * failing call, the error message text may use the host heap.
 *  - Size limit: sw_grid_workspace_bytes(g, o) must not exceed
 *    SW_NOALLOC_SCRATCH_BYTES.  A larger grid is rejected with
 *    SW_ERR_INVALID_ARG before anything runs.  For example, 512 x 256 with
 *    k <= 4 fits in FP64 and in the mixed precisions.
 *  - Nothing has to start at zero.  The solver writes every scratch value
 *    before it reads it, and each call resets the grid's own barrier
 *    counters.
 *  - Overlapping calls race.  Two calls on one device that can run at the
 *    same time share the scratch and corrupt each other's results: for
 *    example, calls from two host threads or calls on two streams.  Issue
 *    them one after another.  Each call waits for its own solve on `stream`
 *    before it returns.
 *  - The first call on each device looks up the scratch's device address.
 *    That is a one-time setup step and may load the library's device code.
 *    Make this first call, with that device current, before any stream
 *    capture begins. */
sw_status sw_gcr_solve_noalloc(sw_grid g, const sw_solve_opts *o, const double *R, double *phi,
                               sw_solve_stats *stats, void *stream);

/* Message describing the last error on the calling host thread. */
const char *sw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SW_ELLIPTIC_H */
