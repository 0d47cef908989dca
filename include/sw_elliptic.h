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
 *    ordered on it, and only sw_gcr_solve, sw_gcr_solve_noalloc,
 *    sw_ensemble_solve and sw_swe_step with stats (to fill host-side stats)
 *    synchronise it;
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
    SW_PC_SI_RICHARDSON = 3,    /* option 3: semi-implicit Richardson, Eq. 13 */
    SW_PC_LEARNED = 4           /* not in the paper: flexible GCR whose
                                   directions alternate between option 3 and
                                   a sw_model's network (opts.model), e = s y / d;
                                   a network direction that does not help is
                                   replaced by option 3.  The network turns of
                                   a single-grid solve run on the device, in a
                                   CUDA graph with a conditional node that the
                                   grid builds once per configuration (and
                                   rebuilds when the grid's workspace, the
                                   model's activations or the launch change),
                                   with no host synchronisation per turn */
} sw_precond_kind;

typedef struct sw_model_s *sw_model;  /* opaque, owned by the library */

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
                            iterations (0: only when the exit test is met).
                            The exit is always decided by the FP64 true
                            residual.  With 0, a mixed-precision solve whose
                            recursive residual stalls above tol (its FP32
                            recursion drifting from the true residual) gets
                            no intermediate FP64 check and runs to max_iters;
                            ru_every = k recomputes it at every cycle
                            restart, at the cost of one FP64 operator pass
                            per cycle (measured at 2048 x 1024 in the design
                            notes) */
    int threads_per_row; /* launch shape: threads of the block that works on one
                            latitude row (multiple of 32, <= 256); 0: automatic */
    double *res_history; /* device, optional (NULL): max_iters+1 doubles, the
                            relative residual after each iteration (entry 0:
                            the initial one), NaN where not reached */
    double *row_residual;/* device, optional (NULL): ny doubles, the final true
                            residual's 2-norm per latitude row */
    sw_model model;      /* SW_PC_LEARNED: the trained network */
    double fb_ratio;     /* SW_PC_LEARNED: a network iteration falls back to
                            option 3 when its direction would remove less of
                            ||r||^2 than fb_ratio times the share the last
                            option-3 direction removed (or is not finite);
                            default 0.5 */
    int row_mode;        /* launch shape of the solver kernel: 0 automatic (one
                            thread block per latitude row while the rows fit the
                            resident blocks, else, in the mixed precisions, one
                            warp per row when nx is a power of two >= 128 and a
                            single grid is solved without the learned
                            preconditioner, else blocks cycling over rows);
                            1 thread blocks only; 2 one warp per row
                            (SW_ERR_INVALID_ARG where not possible).  The
                            results agree to rounding: the inner products sum
                            in another order. */
    int split_r0;        /* mixed precisions: 1 computes the solve's initial
                            residual r0 = L(Phi_0) - R in FP32 with the split
                            fluid thickness of Sec. 4.2, Eq. 14, from the
                            grid's last sw_split_refresh (SW_ERR_INVALID_ARG
                            without one); 0 (default) computes it in FP64.
                            Every later true residual, and so the exit test,
                            stays FP64. */
} sw_solve_opts;

typedef struct {
    int iterations;
    int converged;                 /* 1 if the true residual met tol */
    int status;                    /* sw_status of this solve */
    int fallbacks;                 /* SW_PC_LEARNED: iterations that fell back to option 3 */
    double r0_norm;                /* ||L(Phi_0) - R||_2 */
    double R_norm;                 /* ||R||_2 */
    double true_rel_residual;      /* ||L(Phi) - R|| / ||R|| at exit, FP64 */
    double recursive_rel_residual; /* the GCR recursive residual at exit */
    double eta;                    /* eta used by option 3 */
    int network_turns;             /* SW_PC_LEARNED: applications of the network (its
                                    * proposed directions, fallbacks included); 0 otherwise */
} sw_solve_stats;

/* Fills *o with the defaults: k = 4, tol = 1e-8, max_iters = 1000,
 * min_iters = 0, option 3 with 2 Richardson iterations, automatic eta,
 * omega = 1, FP64, automatic pole band, no periodic true residual, no model,
 * fb_ratio = 0.5, automatic row mode. */
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

/* Split fluid thickness of Sec. 4.2, Eq. 14 (refresh step).  Phi is held as
 * Phi_hat + Phi_tilde: this call stores Phi_hat = fp32(phi) in the grid with
 * the derivative parts of its face fluxes, computed in FP64 from Phi_hat and
 * stored in FP32: on the zonal face (i+1/2, j) the difference
 * Phi_hat[i+1] - Phi_hat[i] and the cross sum Phi_hat[i,j+1] + Phi_hat[i+1,j+1]
 * - Phi_hat[i,j-1] - Phi_hat[i+1,j-1]; on the meridional face (i, j+1/2) the
 * difference Phi_hat[j+1] - Phi_hat[j] and the cross sum Phi_hat[i+1,j] +
 * Phi_hat[i+1,j+1] - Phi_hat[i-1,j] - Phi_hat[i-1,j+1] (with the operator's
 * periodic and across-pole continuation).  These are the paper's stored
 * derivatives of Phi_hat with the grid spacings folded into the face
 * coefficients.  phi: device FP64 [ny][nx].  Allocates 20 bytes per point on
 * the first call (SW_ERR_OOM if that fails); the paper refreshes every 100
 * solves. */
sw_status sw_split_refresh(sw_grid g, const double *phi, void *stream);

/* r = L(Phi) - R with L evaluated in FP32 by Eq. 14 (the difference with R
 * taken in FP64, r stored as float): Phi_tilde = fp32(phi - Phi_hat), the
 * flux derivative parts as the stored ones of Phi_hat plus those of
 * Phi_tilde in FP32, the B and C terms on Phi_hat + Phi_tilde in FP32, the
 * face coefficients of the grid's FP32 copies.  phi, R: device FP64;
 * r: device float; all [ny][nx].  SW_ERR_INVALID_ARG before the first
 * sw_split_refresh.  A refresh survives new coefficients: Phi_hat belongs
 * to the state, not to the operator. */
sw_status sw_split_residual(sw_grid g, const double *phi, const double *R, float *r, void *stream);

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

/* sw_ensemble_solve without host synchronisation: every step is enqueued on
 * `stream` and the call returns at once.  stats_dev (device, n entries, may
 * be NULL) receives the members' sw_solve_stats when the solve completes on
 * the stream; the return value reports only argument and enqueue errors.
 * Calls may follow one another without synchronisation, on the same grids
 * too: each grid stages the descriptors of a call in one of four pinned host
 * slots, and a call waits on the host only while the stream is four calls
 * behind.  Nothing is allocated once each grid's workspace exists, i.e.
 * after one solve with the same precision and k (or an attached workspace),
 * so the call can then be recorded in a CUDA graph and replayed.  With one
 * member (n = 1) the descriptors travel as kernel parameters, with no host
 * staging and no copies, and a recorded call keeps them for the graph's
 * lifetime.  With more, a recorded call stages into a slot of its own, which
 * replays read; it stays valid until the grid's next recorded
 * sw_ensemble_solve_async.  Not for SW_PC_LEARNED. */
sw_status sw_ensemble_solve_async(int n, const sw_grid *grids, const sw_solve_opts *o,
                                  const double *const *R, double *const *phi,
                                  sw_solve_stats *stats_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Learned preconditioner (no counterpart in the paper).  A three-level U-Net
 * of 3x3 convolutions (4 -> 32, pool, 32 -> 64, pool, 64 -> 64, up + skip,
 * 128 -> 64, up + skip, 96 -> 32, 32 -> 1; ReLU after all but the last),
 * padded like the operator: periodic in longitude, across the poles the pole
 * row shifted by half a circle.  Weights and activations are BF16, products
 * accumulate in FP32 on the tensor cores; master weights and AdamW moments
 * are FP32.  Grid sizes: nx = 64, 128 or a multiple of 256; ny a multiple of
 * 4 and >= 8.
 *
 * Inputs x0 (4 channels) of a residual r on a grid: r / s, the zonal and the
 * meridional couplings (ax_w + ax_e) / d and (ay_s + ay_n) / d of L's faces,
 * and sin(latitude), with d = |diag(L)| and s = rms(r).  Output: the network's
 * y; as a preconditioner e = s y / d, trained on y* = d L^-1(R) / rms(R).
 * Parameters are one flat FP32 vector of
 * SW_MODEL_PARAMS values: per layer the weights [out][in][ky][kx], then the
 * biases.
 * ------------------------------------------------------------------------- */
#define SW_MODEL_PARAMS 158369

typedef struct {
    double lr, beta1, beta2, eps, weight_decay;   /* AdamW; decay on weights only */
} sw_adamw;

/* Create a model on the current device (parameters zero, AdamW state zero). */
sw_status sw_model_create(sw_model *out);
sw_status sw_model_destroy(sw_model m);
/* Set (and reset the AdamW state) / read the parameters; host, SW_MODEL_PARAMS floats. */
sw_status sw_model_set_params(sw_model m, const float *params);
sw_status sw_model_get_params(sw_model m, float *params);
/* x0 (device FP32 [4][ny][nx]) for the residual r (device FP32 [ny][nx]) on grid g. */
sw_status sw_model_features(sw_model m, sw_grid g, const float *r, float *x0, void *stream);
/* y = network(x0) for a batch: x0 device FP32 [batch][4][ny][nx], y device FP32 [batch][ny][nx]. */
sw_status sw_model_forward(sw_model m, int batch, int ny, int nx, const float *x0, float *y, void *stream);
/* Mean squared error of y against target (device FP32 [batch][ny][nx]) and
 * its gradient with respect to the parameters (host, SW_MODEL_PARAMS floats;
 * NULL to skip); loss: host. */
sw_status sw_model_loss_grad(sw_model m, int batch, int ny, int nx, const float *x0, const float *target,
                             double *loss, float *grad, void *stream);
/* One AdamW step on that loss; loss (host, may be NULL) receives the loss
 * before the step.  Synchronises the stream only when loss is not NULL. */
sw_status sw_model_train_step(sw_model m, int batch, int ny, int nx, const float *x0, const float *target,
                              const sw_adamw *hp, double *loss, void *stream);
/* e = s y / d: the preconditioner applied to r (device FP32 [ny][nx]). */
sw_status sw_model_apply(sw_model m, sw_grid g, const float *r, float *e, void *stream);
/* The inverse scaling, y = d e / s with s = rms(r): the training target of a
 * pair (r, e = L^-1 r).  Device FP32 [ny][nx] each. */
sw_status sw_model_target(sw_model m, sw_grid g, const float *r, const float *e, float *y, void *stream);

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
 *  - Every call looks up the scratch's device address in the current
 *    context (it can move when a context is destroyed and created again).
 *    The first call on a device may also load the library's device code, a
 *    one-time setup step: make this first call, with that device current,
 *    before any stream capture begins.
 *  - The launch shape is the one sw_gcr_solve picks for the same grid and
 *    options, so the two give the same results. */
sw_status sw_gcr_solve_noalloc(sw_grid g, const sw_solve_opts *o, const double *R, double *phi,
                               sw_solve_stats *stats, void *stream);

/* Test hook for failure detection (no counterpart in the paper).  Every
 * barrier of the solver kernel waits for the arrivals of its member's blocks
 * for at most a limit (2 s), then stops the solve, which returns
 * SW_ERR_TIMEOUT with the CUDA context intact.  This call makes later solves
 * on the current device expect extra_arrivals more arrivals than any block
 * provides, with a limit of wait_limit_s seconds (0: the default 2 s), so a
 * test can make that wait run out without any fault.  sw_debug_barrier(0, 0)
 * restores normal operation. */
sw_status sw_debug_barrier(int extra_arrivals, double wait_limit_s);

/* ---------------------------------------------------------------------------
 * Semi-implicit shallow-water time stepping around the solve (Sec. 2.2,
 * Eqs. 1-10).  A stepper owns the model state on one grid: thickness Phi (m)
 * and momenta Qx = Phi u, Qy = Phi v (m^2/s), plus the fixed fields of the
 * forcing (Eqs. 4-5): orography H0, relaxation rate alpha (1/s) and
 * relaxation target (Qbar_x, Qbar_y).  All fields are device FP64 [ny][nx].
 *
 * One step n -> n+1 (all on the stream, FP64 except inside the solves):
 *  1. winds u, v at n; the advective velocity (a u, a cos(phi) v) at n + 1/2
 *     by linear extrapolation from n and n-1;
 *  2. R^n of Eqs. 4-5 and Q^ = Q^n + dt/2 R^n carried over dt by donor-cell
 *     fluxes (first-order upwind in flux form; MPDATA is not provided), Eq. 6;
 *  3. for a thickness predictor Phi*: the coefficient fields of Eq. 10 with
 *     Eq. 7's pressure gradient, Coriolis and relaxation implicit and the
 *     metric force folded into the Coriolis parameter f + u* tan(phi)/a,
 *     u* = 2u^n - u^(n-1); they are given to the grid with
 *     sw_elliptic_set_coeffs;
 *  4. the right-hand side of the increment solve L(dPhi) = R' with
 *     R' = div(F^n + F0) - (G/(dt/2)) Phi^n - L(Phi^n), F = (a Qx, a cos(phi) Qy)
 *     and F0 the explicit part of F at n+1 (face values are means of the two
 *     cells, no flux through the pole faces); o->tol bounds
 *     ||L(dPhi) - R'|| / ||R'||, the paper's ||r|| / ||r0|| with first guess
 *     Phi^n;
 *  5. steps 3-4 and the solve run twice: with Phi* = Phi^n, then with
 *     Phi* = Phi^n + that increment (warm-started from it).  The first solve
 *     starts from the increment extrapolated from the last two steps
 *     (2 dPhi^(n-1) - dPhi^(n-2); after sw_swe_set_state: zero, then the last
 *     increment), which changes its iteration count, not its tolerance.
 *     This one outer iteration replaces the explicit transport predictor of
 *     Eq. 7, which amplifies short zonal waves at the external-mode Courant
 *     numbers of the pole rows;
 *  6. Phi^{n+1} = Phi^n + dPhi and the momenta from Eq. 8.
 * Cell-centred derivatives are centred differences, periodic in longitude,
 * with the pole row shifted by half a circle beyond each pole.  Winds must
 * keep the zonal Courant number u dt / (a cos(phi) dlam) below 1 on every
 * row, pole rows included.
 * ------------------------------------------------------------------------- */
typedef struct sw_swe_s *sw_swe;

typedef struct {
    double dt;        /* time step (s), > 0 */
    double gravity;   /* g (m s^-2), > 0 */
    double omega;     /* rotation rate Omega (1/s) */
} sw_swe_params;

/* Create a stepper on grid g (which must outlive it); allocates 38 fields of
 * nx*ny doubles on the grid's device.  The grid's coefficients are
 * replaced at every step. */
sw_status sw_swe_create(sw_grid g, const sw_swe_params *p, sw_swe *out);
sw_status sw_swe_destroy(sw_swe m);
/* Copy a state in (device pointers; H0, alpha, Qbar_x, Qbar_y may be NULL,
 * meaning zero).  Phi must be positive.  Clears the history: the first step
 * takes the winds of level n-1 equal to those of level n. */
sw_status sw_swe_set_state(sw_swe m, const double *Phi, const double *Qx, const double *Qy,
                           const double *H0, const double *alpha, const double *Qbar_x,
                           const double *Qbar_y, void *stream);
/* Set the winds of level n-1 (device, m/s) used by the next step. */
sw_status sw_swe_set_history(sw_swe m, const double *u_prev, const double *v_prev, void *stream);
/* Copy the current state out (device pointers; any may be NULL). */
sw_status sw_swe_get_state(sw_swe m, double *Phi, double *Qx, double *Qy, void *stream);
/* Steps 1-4 of the next step for the predictor phi_star (device; NULL:
 * Phi^n), without advancing the state: on return (on the stream) the grid
 * holds those coefficients.  coeffs: NULL or 7 device pointers (A11, A12,
 * A21, A22, B1, B2, C; entries may be NULL) that receive copies of the
 * coefficient fields; rhs: NULL or a device buffer for R'. */
sw_status sw_swe_explicit(sw_swe m, const double *phi_star, double *const *coeffs, double *rhs,
                          void *stream);
/* Advance nsteps (>= 1) steps, two solves each, with options o (FP64 or a
 * mixed precision; not SW_PC_LEARNED).  Nothing synchronises when stats is
 * NULL.  Otherwise stats (host, 2 * nsteps entries: each step's predictor and
 * corrector solves) receives every solve's sw_solve_stats after the call
 * waits for the stream; a solve that did not converge is reported there (its
 * status), and the step went on with its last iterate.  Returns argument and
 * CUDA errors only. */
sw_status sw_swe_step(sw_swe m, const sw_solve_opts *o, int nsteps, sw_solve_stats *stats,
                      void *stream);

/* Message describing the last error on the calling host thread. */
const char *sw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SW_ELLIPTIC_H */
