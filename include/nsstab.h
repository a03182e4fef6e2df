/*
 * nsstab.h - C ABI of the GB300-native matrix-free stability library.
 *
 * The library implements the data-parallel hot path of the time-stepper
 * approach to hydrodynamic stability (Loiseau, Bucci, Cherubini, Robinet,
 * "Time-stepping and Krylov methods for large-scale instability problems"):
 *   - a 2D incompressible Navier-Stokes time-stepper in vorticity-
 *     streamfunction form that applies the nonlinear map G (Sec. 2, Eq. 2;
 *     Sec. 3.1.2, Eq. 41) and the exponential propagator
 *     M v = exp(T A) v of the linearised equations (Sec. 3, Eqs. 29-30;
 *     Sec. 3.1.2, Eq. 42; Sec. 3.2, Eq. 55);
 *   - the Arnoldi factorisation (Sec. 3.2.1, Algorithm 1, Eq. 57) with
 *     CGS2 orthogonalisation and the Krylov-Schur restart (Sec. 3.2.2,
 *     Eqs. 60-63) that consume M;
 *   - selective frequency damping (Sec. 3.1.1, Eq. 40) for the base flow.
 *
 * Conventions for every entry point:
 *   - Fields are float64, row-major [ny][nx] (x fastest), contiguous, in
 *     DEVICE memory owned by the caller, unless an argument says "host".
 *   - All device work is enqueued on the stream given to stepper_create
 *     (a cudaStream_t passed as void*; NULL = legacy default stream).
 *   - Return value: NSSTAB_OK (0) on success, a negative NSSTAB_ERR_* code
 *     on failure (nothing is guaranteed about outputs then), a positive
 *     soft status (NSSTAB_NOT_CONVERGED, NSSTAB_DIVERGED) when the call ran
 *     to completion but did not meet its target.  nsstab_last_error()
 *     returns a message for the calling thread's last failure.
 *   - Calls marked "asynchronous" only enqueue work: results are valid
 *     after the stream is synchronised.  All other calls synchronise the
 *     stream before returning.
 *   - A stepper is not thread-safe: one host thread at a time per stepper.
 *
 * Grid: nx, ny powers of two in [8, 4096]; x_i = i Lx/nx, y_j = j Ly/ny; the
 * box is doubly periodic.
 */
#ifndef NSSTAB_H
#define NSSTAB_H

#ifdef __cplusplus
extern "C" {
#endif

#define NSSTAB_OK 0
#define NSSTAB_NOT_CONVERGED 1      /* target not met within the budget */
#define NSSTAB_DIVERGED 2           /* non-finite values appeared */
#define NSSTAB_ERR_INVALID_ARG (-1)
#define NSSTAB_ERR_CUDA (-2)
#define NSSTAB_ERR_OUT_OF_MEMORY (-3)
#define NSSTAB_ERR_NUMERICAL (-4)   /* dense eigen-solver failed */

/* Physical and numerical parameters of one stepper.  See
 * nsstab_config_default for the 128x64 cylinder-wake values. */
typedef struct nsstab_config {
    int nx, ny;             /* grid points in x and y (powers of two)          */
    double Lx, Ly;          /* box size (16, 8)                                 */
    double dt;              /* time step                                        */
    double Re;              /* Reynolds number; viscosity nu = 1/Re             */
    double Uinf;            /* free-stream velocity along x (1)                 */
    double cyl_x, cyl_y;    /* cylinder centre (4, 4)                           */
    double cyl_D;           /* cylinder diameter (1); <= 0 disables it          */
    double eta;             /* Brinkman permeability (1e-3)                     */
    double mask_cells;      /* width of the smoothed mask edge in x-cells (2)   */
    double sponge_frac;     /* fringe occupies x >= (1 - frac) Lx (0.1)         */
    double sponge_sigma;    /* peak fringe strength (10); <= 0 disables it      */
    int precision;          /* 64: FP64 stepper; 32: FP32 stepper (FP64 I/O)    */
} nsstab_config;

typedef struct nsstab_stepper nsstab_stepper;   /* opaque */

/* Fill *cfg with the 128x64 cylinder defaults (Re 50, dt 0.01, FP64). */
void nsstab_config_default(nsstab_config* cfg);

/* Create a stepper for cfg; it allocates and owns its device workspace
 * (about 13 fields of nx*ny values of the stepper's precision).
 * stream: cudaStream_t (as void*) on which all of this stepper's work runs.
 * Errors: INVALID_ARG (bad sizes or parameters), OUT_OF_MEMORY, CUDA. */
int stepper_create(const nsstab_config* cfg, void* stream, nsstab_stepper** out);

/* Batched stepper: B = nsets * per_set members on one grid, advanced
 * together by every call below (each kernel launch covers all members).
 * Member m belongs to parameter set m / per_set, which has its own Reynolds
 * number Re[k] and cylinder diameter cyl_D[k] (host arrays of nsets; NULL
 * takes cfg's value for every set) and its own base flow for the linearised
 * step.  Uses: Reynolds/geometry sweeps (per_set = 1), several start
 * vectors or perturbations per parameter set (per_set > 1), independent
 * stability solves served together.  For a batched stepper every field
 * argument of the calls below is [B][ny][nx] (base flows [nsets][ny][nx]),
 * stepper_residual and sfd_baseflow write B residuals, and arnoldi_eigs is
 * replaced by batch_arnoldi_eigs.  A stepper from stepper_create is the
 * batch nsets = per_set = 1.  Errors: INVALID_ARG (nsets < 1, per_set < 1,
 * B > 65535, Re <= 0, cyl_D < 0), OUT_OF_MEMORY, CUDA. */
int batch_create(const nsstab_config* cfg, int nsets, const double* Re, const double* cyl_D,
                 int per_set, void* stream, nsstab_stepper** out);

/* Number of members B and of parameter sets of a stepper (host ints). */
int stepper_members(nsstab_stepper* st, int* members, int* sets);

/* Release the stepper and its device memory (synchronises its stream). */
void stepper_destroy(nsstab_stepper* st);

/* Step a1 alone: psi with 5-point Laplacian(psi) = -omega (mean removed),
 * solved in Fourier space.  omega, psi: device [ny][nx].  Asynchronous. */
int stepper_poisson(nsstab_stepper* st, const double* omega, double* psi);

/* March the nonlinear equations (Sec. 3, Eq. 28) nsteps steps of a1-a4:
 * omega <- G^nsteps(omega).  AB1 on the first step, AB2 after.  omega:
 * device [ny][nx], in/out.  Asynchronous. */
int step_nonlinear(nsstab_stepper* st, double* omega, int nsteps);

/* Set the frozen base flow (vorticity Omega_b, device [ny][nx]) used by the
 * linearised stepper.  The stepper keeps its own copy.  Asynchronous. */
int stepper_set_base(nsstab_stepper* st, const double* base_omega);

/* M v = exp(T A) v (Eq. 42 / Eq. 55): T/dt linearised steps about the base
 * flow, AB1 start, so M is a fixed linear map of v.  base_omega: device
 * [ny][nx] (it is then also kept as the stepper's base), or NULL to use the
 * base of the last stepper_set_base.  v_in, v_out: device [ny][nx]; they
 * may alias.  T must be a whole number of steps.  Asynchronous. */
int apply_expTL(nsstab_stepper* st, const double* base_omega,
                const double* v_in, double* v_out, double T);

/* Base-flow residual r(q) = ||G_1(q) - q||_h / dt with G_1 one AB1 step
 * and ||f||_h = sqrt(sum f^2 dx dy) (fixed point of Eq. 32).  q: device.
 * *r: host.  Synchronous. */
int stepper_residual(nsstab_stepper* st, const double* q, double* r);

/* Selective frequency damping (Sec. 3.1.1, Eq. 40): march
 *   X* = G(X^n),  X^{n+1} = X* - dt chi (X* - Y^n),
 *   Y^{n+1} = Y^n + dt (X* - Y^n) / Delta,   Y^0 = X^0,
 * evaluating r(X) every check_every steps, until r <= tol or max_steps.
 * omega: device [ny][nx], in: X^0, out: last X.  *residual, *steps: host.
 * Returns NSSTAB_OK, NSSTAB_NOT_CONVERGED or NSSTAB_DIVERGED.  Synchronous. */
int sfd_baseflow(nsstab_stepper* st, double* omega, double chi, double Delta,
                 double tol, long max_steps, int check_every,
                 double* residual, long* steps);

/* Steady base flow by Newton-Krylov (Sec. 3.1.2, Eq. 43): iterate
 *   q <- q - (I - M)^{-1} (q - Phi_T(q)),
 * Phi_T = T/dt nonlinear steps (AB1 start), M = dPhi_T/dq at the current
 * iterate: the exact discrete tangent (see apply_tangent), the linear system
 * solved by GMRES(gmres_m) with CGS2 to the relative residual 1e-3 (at
 * most 2 restarts), until the base-flow residual r(q) of stepper_residual is
 * <= tol or max_newton Newton steps were made.  Unlike SFD it also
 * converges to unstable steady states with real (non-oscillating) unstable
 * eigenvalues.  omega: device [ny][nx], in: initial guess, out: last
 * iterate.  *residual (r of the last iterate), *newton_iters, *matvecs
 * (products with M): host.  Allocates n (gmres_m + 5) doubles and a
 * two-member stepper of st's configuration during the call.  Single
 * steppers only.  Returns NSSTAB_OK, NSSTAB_NOT_CONVERGED or
 * NSSTAB_DIVERGED.  Synchronous. */
int newton_krylov_fixedpoint(nsstab_stepper* st, double* omega, double T, int gmres_m,
                             double tol, int max_newton, double* residual,
                             int* newton_iters, int* matvecs);

/* The same with the Krylov products taken in lin_st's arithmetic (same
 * grid and dt; NULL = st), e.g. FP32 while st (FP64) evaluates Phi_T and
 * the residual, with the GMRES relative tolerance and restart count given,
 * and the Jacobian chosen: jacobian = NSSTAB_JACOBIAN_TANGENT (the exact
 * discrete tangent, marched by a two-member stepper of lin_st's
 * configuration made for the call) or NSSTAB_JACOBIAN_FROZEN (lin_st's
 * linearised propagator about the current iterate: exact only at the fixed
 * point, one march per product instead of two). */
#define NSSTAB_JACOBIAN_TANGENT 0
#define NSSTAB_JACOBIAN_FROZEN 1
int newton_krylov_fixedpoint_ex(nsstab_stepper* st, nsstab_stepper* lin_st, double* omega,
                                double T, int gmres_m, double gmres_rtol, int gmres_restarts,
                                double tol, int max_newton, int jacobian, double* residual,
                                int* newton_iters, int* matvecs);

/* Exact discrete tangent of Phi_T (T/dt nonlinear steps, AB1 start) at q,
 * applied to v_in: v_out = dPhi_T(q)/dq v_in.  Computed by co-integration:
 * member 0 of st marches q with the nonlinear step while member 1 marches
 * v with the step linearised about member 0's state of the same step (the
 * AB2 history term linearised about the previous state), which is the
 * derivative of the discrete scheme itself, not of the continuous
 * equations.  st: a batch of two members and one parameter set
 * (batch_create(cfg, 1, Re, D, 2, ...)); its base fields are overwritten
 * (set a base again before a frozen-base product).  q, v_in, v_out: device
 * [ny][nx]; v_out may alias v_in.  Asynchronous. */
int apply_tangent(nsstab_stepper* st, const double* q, const double* v_in, double* v_out, double T);

/* Leading eigenvalues of M = exp(T A) about base_omega (Sec. 3.2).
 * max_restarts == 0: one m-step Arnoldi factorisation (Algorithm 1) with
 * CGS2.  max_restarts > 0: Krylov-Schur (Sec. 3.2.2) of order m, restarted
 * until the leading values have Ritz residual |b^T y| <= tol (Eq. 63) or
 * max_restarts restarts were made.  Wanted set on restart: values with
 * |mu| >= 1 - 0.05, clamped to [nev, m/2], never splitting a conjugate pair.
 *   base_omega: device [ny][nx] or NULL (use the current base)
 *   v0:         device [ny][nx] starting vector (need not be normalised)
 *   m:          Krylov dimension, 2 <= m <= min(nx*ny - 1, 1024)
 *   nev:        number of leading values wanted (rounded up by one when the
 *               last one would split a complex-conjugate pair)
 *   eig_re, eig_im, resid: host arrays of at least nev+1 entries: Ritz
 *               values mu (eigenvalues of M, |mu| descending, then Im mu
 *               descending) and their residuals
 *   eigvecs:    device [nev+1][ny][nx] or NULL: Ritz vectors V y, unit
 *               norm; a conjugate pair k, k+1 is stored as Re in slot k and
 *               Im in slot k+1
 *   n_eig:      host, number of values written (nev or nev+1)
 *   n_conv:     host, how many of them have residual <= tol
 *   n_matvec:   host, products with M made
 * Allocates (n (m+1)) doubles of device memory for the basis for the
 * duration of the call.  Returns NSSTAB_OK when all n_eig values converged,
 * NSSTAB_NOT_CONVERGED otherwise.  Synchronous. */
int arnoldi_eigs(nsstab_stepper* st, const double* base_omega, const double* v0,
                 int m, int nev, double tol, int max_restarts, double T,
                 double* eig_re, double* eig_im, double* resid, double* eigvecs,
                 int* n_eig, int* n_conv, int* n_matvec);

/* Largest basis size j accepted by cgs2_orthogonalize_noalloc. */
#define NSSTAB_NOALLOC_MAX_COLS 256

/* cgs2_orthogonalize for callers that cannot allocate device memory at the
 * point of the call: frameworks whose memory pool owns the device memory and
 * forbids side allocations, and real-time loops that must not take the
 * allocator's locks or meet an out-of-memory error mid-run.  The paper has
 * no counterpart: it is a deployment variant of the Gram-Schmidt step above.
 * Same arguments, results and synchronisation as cgs2_orthogonalize, but
 * all scratch (partial dot products per block, the two coefficient vectors)
 * lives in one fixed file-scope device array of about 0.3 MB that every GPU
 * loading the library holds until the process exits; the call makes no
 * cudaMalloc, cudaFree or other allocating call.  j > NSSTAB_NOALLOC_MAX_COLS
 * is rejected with NSSTAB_ERR_INVALID_ARG.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) for that device, with
 * that device current.  A reset of the device's primary context after that first call is not
 * supported.  All calls on a device share the array, so calls whose GPU
 * work overlaps (other streams, other host threads) race: serialise them.
 * Nothing needs clearing between calls: each call writes every scratch
 * value before reading it. */
int cgs2_orthogonalize_noalloc(const double* V, long ldv, long n, int j, double* w,
                               double* h, double* beta, void* stream);

/* Measurement helper for the propagator of Eq. 42: run nsteps linearised
 * steps from v (device [ny][nx]) about the current base flow, recording a
 * CUDA event on the stepper's stream between consecutive kernels, and add
 * the elapsed milliseconds of each of the six kernels of a step to
 * kernel_ms[0..5] (host): column Poisson pass, row inverse of psi, row
 * forward of the advection term, column AB2/CN update, row inverse of
 * (omega*, psi*), row forward of the penalised vorticity.  The state the
 * steps leave behind is discarded.  Synchronous. */
int stepper_profile_linear(nsstab_stepper* st, const double* v, int nsteps, double* kernel_ms);

/* Launch plans of the six step kernels (ids 0..5 in the order of
 * stepper_profile_linear).  A plan is (log2_elems, per_block): each thread
 * of the FFT passes owns 2^log2_elems elements (1, 2 or 3), and a block
 * handles per_block row pairs or columns (a power of two).  Plans change
 * the launch shape and the radix of the transforms, not the method; results
 * agree to rounding.  stepper_create picks a default from the grid size.
 * stepper_autotune times every valid plan of each kernel (reps launches
 * each) and keeps the fastest; it overwrites the stepper's workspace (not
 * its base flow) and, if plans is not NULL, stores the chosen
 * (log2_elems, per_block) of kernel k in plans[2k], plans[2k+1] (host, 12
 * ints).  stepper_set_plan rejects a plan that does not fit the grid
 * (INVALID_ARG).  All synchronous. */
int stepper_autotune(nsstab_stepper* st, int reps, int* plans);
int stepper_set_plan(nsstab_stepper* st, int kernel, int log2_elems, int per_block);

/* FP32 steppers: run each time step as four kernels instead of six, the two
 * row passes (Sec. 3's nonlinear/linearised right-hand side, and the
 * penalisation split) each fused into one pass that walks strips of
 * rows_per_strip rows and keeps the neighbouring rows the centred y
 * differences need in shared memory.  Same discrete operator, FP32
 * rounding.  rows_per_strip = 0 selects the six-kernel step; otherwise it
 * must be even and divide ny, and the grid must have 64 <= nx <= 2048
 * (INVALID_ARG otherwise, also for FP64 and double-float steppers).
 * Off by default.  With it on, stepper_profile_linear reports the fused
 * passes in slots 2 (right-hand side) and 5 (penalisation) and 0 ms in
 * slots 1 and 4.  Synchronous. */
int stepper_set_fused_rows(nsstab_stepper* st, int rows_per_strip);
int stepper_get_fused_rows(nsstab_stepper* st, int* rows_per_strip);
int stepper_get_plan(nsstab_stepper* st, int kernel, int* log2_elems, int* per_block);

/* arnoldi_eigs for every member of a batched stepper at once: member b runs
 * its own Arnoldi / Krylov-Schur process (same m, nev, tol, max_restarts, T)
 * from v0[b] about the base flow of its parameter set.  The processes
 * advance in lockstep rounds of one batched product with M and one batched
 * CGS2; a member leaves the batch when it has converged or used its
 * restarts.  base_omegas: device [nsets][ny][nx] or NULL (current bases);
 * v0: device [B][ny][nx]; eig_re, eig_im, resid: host [B][nev+1]; eigvecs:
 * device [B][nev+1][ny][nx] or NULL; n_eig, n_conv, n_matvec: host [B].
 * Allocates B (n (m+1)) doubles for the bases during the call.  Returns
 * NSSTAB_OK when every member converged, else NSSTAB_NOT_CONVERGED.
 * Synchronous. */
int batch_arnoldi_eigs(nsstab_stepper* st, const double* base_omegas, const double* v0,
                       int m, int nev, double tol, int max_restarts, double T,
                       double* eig_re, double* eig_im, double* resid, double* eigvecs,
                       int* n_eig, int* n_conv, int* n_matvec);

/* Block Krylov-Schur: an eigenproblem of M = exp(T A) about the base flow
 * of each parameter set, built with a block of b vectors per product with M,
 * so that every product is one batched run of the step kernels over b
 * fields per set (b times the parallelism of arnoldi_eigs on the same
 * grid).  Each new basis column is orthogonalised by CGS2 against every
 * column before it (Algorithm 1's Gram-Schmidt step); the projected matrix
 * is then banded with b sub-diagonals, and the residual of a Ritz pair
 * (mu, V y) is ||R y|| with R the b rows below its square part.  The
 * restart keeps the wanted Schur vectors and the b residual columns
 * (Sec. 3.2.2 with a rank-b instead of a rank-1 remainder).  The paper's
 * Algorithm 1 is the case b = 1.  The S parameter sets of a batch (a
 * Reynolds or geometry sweep) are S independent block eigenproblems run in
 * lockstep rounds: one batched product over all S b new columns, then one
 * batched CGS2 across the sets per column; a set leaves the rounds when it
 * has converged or used its restarts.
 *   st:   a batch of S parameter sets and b = per_set members
 *         (batch_create(cfg, S, Re, D, b, ...)); S = b = 1 is a plain stepper
 *   base_omega: device [S][ny][nx] or NULL (current bases)
 *   v0:   device [S][b][ny][nx], each set's start block (linearly independent)
 *   m:    basis size per set, 2 (nev + 1) + 2 b <= m <= 1024; the blocked
 *         Gram-Schmidt also needs b <= 8 and (m + b) b <= 6144 (its
 *         coefficients of one pass held in 48 KB of shared memory), so
 *         m <= 760 at b = 8; other values give NSSTAB_ERR_INVALID_ARG
 *   eig_re, eig_im, resid: host [S][nev+1]; eigvecs: device [S][nev+1][ny][nx]
 *   or NULL; n_eig, n_conv, n_matvec: host [S] (n_matvec counts single
 *   products, b per round).  With S = 1 these are the arrays of arnoldi_eigs.
 * Allocates about S (m + 2 b) n + (m + 2 b) n doubles during the call.
 * Returns NSSTAB_OK when every set converged, else NSSTAB_NOT_CONVERGED.
 * Synchronous. */
int block_arnoldi_eigs(nsstab_stepper* st, const double* base_omega, const double* v0,
                       int m, int nev, double tol, int max_restarts, double T,
                       double* eig_re, double* eig_im, double* resid, double* eigvecs,
                       int* n_eig, int* n_conv, int* n_matvec);

/* ------------------------------------------------------------------------
 * Serving batch: many independent eigen-solves on mixed grids.
 *
 * The paper analyses one flow at a time (Sec. 3.2); a parameter study or an
 * analysis service runs many, on grids of different sizes.  serve_eigs takes
 * a list of solves that may differ in grid, time step, Reynolds number and
 * cylinder diameter.  Solves that share (nx, ny, dt) are grouped into
 * batched steppers (one member per solve, as batch_create with per_set = 1),
 * split further where a group would not fit the memory budget.  The groups
 * run concurrently, each on its own CUDA stream and host thread, largest
 * grids first; a group is admitted only while the device memory held by
 * the running groups (an upper estimate of stepper workspace plus Krylov
 * basis) stays within mem_budget.  Every solve is the Krylov-Schur
 * eigen-solve of batch_arnoldi_eigs (same m, nev, tol, max_restarts, T),
 * so its Ritz values equal those of arnoldi_eigs on a single stepper of
 * the same configuration, up to rounding.
 * --------------------------------------------------------------------- */

/* Ritz values kept per solve: nev <= NSSTAB_SERVE_MAX_EIG - 1. */
#define NSSTAB_SERVE_MAX_EIG 33

typedef struct {
    int nx, ny;           /* grid: powers of two, as in nsstab_config */
    double dt;            /* time step; T / dt must be a whole number */
    double Re, cyl_D;     /* Reynolds number (> 0), cylinder diameter (>= 0) */
    const double* base;   /* device [ny][nx]: base-flow vorticity (read only) */
    const double* v0;     /* device [ny][nx]: starting vector, non-zero (read only) */
} nsstab_eig_job;

typedef struct {
    int status;           /* NSSTAB_OK, NSSTAB_NOT_CONVERGED, or an error code < 0 */
    int n_eig, n_conv, n_matvec;
    int group;            /* index of the batch the solve ran in */
    double latency_s;     /* seconds from the call's start to the solve's completion */
    double eig_re[NSSTAB_SERVE_MAX_EIG];   /* Ritz values mu, |mu| descending */
    double eig_im[NSSTAB_SERVE_MAX_EIG];
    double resid[NSSTAB_SERVE_MAX_EIG];    /* their residuals */
} nsstab_eig_result;

/* Run njobs eigen-solves as described above.
 *   cfg:        shared physical parameters (Lx, Ly, Uinf, cylinder centre,
 *               eta, mask_cells, sponge, precision); its nx, ny, dt, Re and
 *               cyl_D are ignored (each job gives its own)
 *   jobs:       host array of njobs >= 1 solves
 *   m, nev, tol, max_restarts, T: as arnoldi_eigs, for every solve
 *   mem_budget: device bytes the running groups may hold; <= 0 takes 80% of
 *               the device memory free at the call
 *   max_concurrent: most groups in flight at once (>= 1; <= 0 means 4)
 *   results:    host array of njobs, written for every job
 *   ngroups:    host, number of batches formed (may be NULL)
 * A job whose single-member batch would exceed mem_budget fails with
 * NSSTAB_ERR_OUT_OF_MEMORY in its result; the others still run.  The jobs'
 * base and v0 buffers must hold their values when the call is made (its
 * own streams do not wait on the caller's streams) and stay valid and
 * unmodified until it returns; the call uses the current device of the
 * calling thread, synchronises every stream it creates and returns when
 * all solves are done.  Returns
 * the first error code (< 0) of any job, else NSSTAB_NOT_CONVERGED if any
 * solve did not converge, else NSSTAB_OK.  Argument errors (INVALID_ARG)
 * are reported before any device work.  Synchronous. */
int serve_eigs(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
               double tol, int max_restarts, double T, long long mem_budget, int max_concurrent,
               nsstab_eig_result* results, int* ngroups);

/* The same batch of solves (FP32 stepper only: cfg->precision must be 32)
 * with every grid advanced by one persistent launch per step kernel instead
 * of one batched stepper per grid on its own stream.  Solves that share
 * (nx, ny, dt) form a group as in serve_eigs; groups are admitted by device
 * memory in waves (largest grids first, while the estimated footprint fits
 * mem_budget, at most 8 grids a wave), and all solves of a wave run in
 * lockstep Krylov-Schur rounds of Sec. 3.2.2: each round one product with M
 * for every unfinished solve, made of T/dt_g steps of its own grid g, all
 * grids stepped by the same launches (a grid sits out the steps beyond its
 * own T/dt), captured once as a CUDA graph; then one batched CGS2 over all
 * solves (vectors of different lengths).  Arguments, results and status as
 * serve_eigs; results[i].group is the wave index and *nwaves (if not NULL)
 * the number of waves.  Synchronous. */
int serve_eigs_persistent(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
                          double tol, int max_restarts, double T, long long mem_budget,
                          nsstab_eig_result* results, int* nwaves);

/* ------------------------------------------------------------------------
 * Learned initial guess for the base-flow solve.
 *
 * The paper has no counterpart: the Newton-Krylov fixed-point solve
 * (Sec. 3.1.2, Eq. 43) converges in fewer iterations from a start closer to
 * the fixed point, and this network predicts such a start from the flow's
 * parameters.  It is a 4-level U-Net: at level l (width c_l = width 2^l,
 * grid (ny, nx) / 2^l) two 3x3 convolutions with periodic wrap + ReLU;
 * 2x2 average pooling down; nearest 2x upsampling up, concatenated with
 * the encoder's output of that level (upsampled channels first); a 1x1
 * output convolution to one channel.  Activations are stored in bfloat16
 * (round to nearest even), weights as FP32 masters with a bfloat16 copy
 * used by the convolutions, all sums in FP32.
 *
 * Parameters are one flat FP32 vector: for each convolution in the order
 * enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, enc3a, enc3b, dec2a, dec2b,
 * dec1a, dec1b, dec0a, dec0b, out, the weight [out][in][3][3] ([1][c_0]
 * for out) followed by the bias [out].
 * Fields: x is [B][in_ch][ny][nx] FP32, targets and outputs [B][ny][nx]
 * FP32, all device memory owned by the caller.  Calls are enqueued on the
 * network's stream; unet_gradient and unet_train_step synchronise it (they
 * return the loss).
 * --------------------------------------------------------------------- */
typedef struct nsstab_unet nsstab_unet;

/* Number of FP32 parameters of the network (-1 for bad arguments). */
long unet_param_count(int in_ch, int width);

/* Create a network for inputs of in_ch channels on an ny x nx grid (powers
 * of two >= 8) and batches of up to max_batch; parameters start at zero.
 * stream: cudaStream_t as void*.  Errors: INVALID_ARG, OUT_OF_MEMORY. */
int unet_create(int in_ch, int width, int ny, int nx, int max_batch, void* stream, nsstab_unet** out);
void unet_destroy(nsstab_unet* net);

/* Copy the parameters in (device, unet_param_count floats; also resets
 * Adam's moments and step count) or out. */
int unet_set_params(nsstab_unet* net, const float* theta);
int unet_get_params(nsstab_unet* net, float* theta);

/* y = net(x) for a batch of 1 <= batch <= max_batch.  Asynchronous. */
int unet_forward(nsstab_unet* net, const float* x, int batch, float* y);

/* Loss = mean over all outputs of (net(x) - target)^2 (host, *loss) and
 * its gradient with respect to the parameters (device, param_count
 * floats).  Synchronous. */
int unet_gradient(nsstab_unet* net, const float* x, const float* target, int batch, float* grad,
                  double* loss);

/* One Adam step (moments m, v; step t counted from unet_set_params):
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), for the
 * gradient g of the loss above; *loss is the loss before the step.
 * Synchronous. */
int unet_train_step(nsstab_unet* net, const float* x, const float* target, int batch, float lr,
                    float beta1, float beta2, float eps, double* loss);

/* One CGS2 orthogonalisation (Algorithm 1's Gram-Schmidt step applied
 * twice): h = V^T w; w -= V h; h2 = V^T w; w -= V h2; h += h2;
 * beta = ||w||.  V: device, j columns of length n with leading dimension
 * ldv >= n (column k at V + k*ldv); w: device, n, in/out (NOT normalised);
 * h: host, j entries; beta: host.  j may be 0 (only beta is computed).
 * stream: cudaStream_t as void*.  The call keeps a small per-thread
 * workspace (device partial sums, pinned host staging) that grows with j
 * and lives until the process exits.  Synchronous. */
int cgs2_orthogonalize(const double* V, long ldv, long n, int j, double* w,
                       double* h, double* beta, void* stream);

/* Host-only access to the dense FP64 eigen-solver that the Krylov layer
 * applies to its projected matrix: eigenvalues and unit-norm eigenvectors
 * (the Ritz pairs of H_m, Sec. 3.2.1) and the real Schur form reordered so
 * that the eigenvalues with |lambda| >= thr come first (step 3 of the
 * Krylov-Schur method, Sec. 3.2.2).  A, T, Z, vr, vi: HOST, column-major
 * n x n; wr, wi: host, n.  Eigenvalues are in the diagonal order of the
 * Schur form; column i of vr + i vi is the eigenvector of wr[i] + i wi[i]
 * (vr, vi may be NULL).  is_hessenberg != 0 skips the Hessenberg reduction
 * (A must then be upper Hessenberg).  *p receives the dimension of the
 * leading block of wanted values.  No GPU is involved.  Errors:
 * INVALID_ARG, NUMERICAL. */
int nsstab_dense_eig(int n, const double* A, int is_hessenberg, double* wr, double* wi,
                     double* vr, double* vi);
int nsstab_dense_schur_ordered(int n, const double* A, double thr, double* T, double* Z, int* p);

/* Message describing the calling thread's last error ("" if none). */
const char* nsstab_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NSSTAB_H */
