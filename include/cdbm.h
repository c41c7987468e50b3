/*
 * cdbm.h -- C ABI of the GB300 central-moment discrete Boltzmann (CDBM) library.
 *
 * The library advances the 16 discrete velocity distributions f_i of the CDBM of
 * Lin, Su, Fei and Luo ("Central-moment-based discrete Boltzmann modeling of
 * compressible flows", Sec. 2) on a 2-D grid with hand-written CUDA kernels for
 * sm_103a.  Each time step:
 *   - forms rho, u, T from the conserved moments of f (Sec. 2, after Eq. 7);
 *   - builds f_eq from the prescribed central moments of the Maxwellian with I
 *     extra degrees of freedom (Eqs. 4-7);
 *   - applies BGK relaxation and the NND/minmod transport term of every discrete
 *     velocity (Eqs. 1, 12-20);
 *   - runs two Runge-Kutta stages, one fused kernel each.
 * On demand it extracts rho, u, T and the nonequilibrium quantities Delta*
 * (Eqs. 8-11).
 *
 * Conventions shared by every entry point
 *   - Discrete velocities (Eqs. 2-3): index i = 4g + k, group g = a, b, c, d.
 *     Groups a and c point along the axes in the order (1,0),(0,1),(-1,0),(0,-1);
 *     groups b and d along the diagonals in the order (1,1),(-1,1),(-1,-1),(1,-1);
 *     each vector is scaled by its group speed (diagonals are not normalised).
 *   - Fields are row-major [ny][nx] doubles (x fastest).  A distribution field is
 *     [16][ny][nx] (velocity plane outermost).  Delta* is [12][ny][nx].
 *   - D = 2; K = D + I; gamma = (K + 2) / K; T from rho K T = sum f((v-u)^2 + eta^2).
 *   - Pointer arguments marked "host or device" may point to either kind of memory
 *     (the library tells them apart through unified addressing); a host pointer is
 *     staged through a library-owned device buffer.  Every other pointer is a
 *     device pointer owned by the caller.
 *   - All work is ordered on the context's CUDA stream and is asynchronous unless
 *     an entry point says otherwise.
 *   - Every entry point returns a cdbm_status and never aborts the process.  The
 *     first error a context meets is sticky: later calls return it until the
 *     context is destroyed; cdbm_last_error() gives a one-line description.
 */
#ifndef CDBM_H
#define CDBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cdbm_ctx cdbm_ctx;

typedef enum {
    CDBM_OK = 0,
    CDBM_EINVAL = 1,      /* bad argument (size, step, stability limit, pointer)   */
    CDBM_ESINGULAR = 2,   /* the moment system of the velocity set is singular or  */
                          /* worse conditioned than 1e12                           */
    CDBM_ENOMEM = 3,      /* the allocator returned NULL                           */
    CDBM_ECUDA = 4,       /* a CUDA runtime call failed                            */
    CDBM_ENONPHYS = 5,    /* a kernel met rho <= 0, T <= 0 or a non-finite value   */
    CDBM_ETIMEOUT = 6     /* reserved for a bounded device-side wait that gives up; */
                          /* no kernel here waits in software (block and cluster   */
                          /* barriers only), so no call returns it                 */
} cdbm_status;

typedef enum { CDBM_BC_PERIODIC = 0, CDBM_BC_ZEROGRAD = 1 } cdbm_bc;

/* Grid: nx, ny >= 1 cells of size dx, dy.  Boundary per axis: periodic, or
 * zero-gradient (ghost cells repeat the edge cell).  The paper states no
 * boundary condition; shock tubes use zero-gradient in x. */
typedef struct {
    int nx, ny;
    double dx, dy;
    int bc_x, bc_y;       /* cdbm_bc */
} cdbm_grid;

/* Discrete velocity set, Eqs. (2)-(3): group speeds (v_a, v_b, v_c, v_d) and
 * extra-degree-of-freedom speeds (eta_a, eta_b, eta_c, eta_d). */
typedef struct {
    double v[4];
    double eta[4];
} cdbm_vset;

/* Optional device-memory allocator (for example a caching allocator).  alloc
 * returns device memory of at least `bytes` usable on `stream`, aligned to at
 * least 16 bytes, or NULL (a block that is not so aligned is handed back to free
 * and counts as NULL); free releases it.  With no allocator the library uses cudaMallocAsync/cudaFreeAsync
 * on the context stream. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} cdbm_allocator;

/* Precision of the stored state. */
typedef enum {
    CDBM_FP64 = 0,        /* state, flux, equilibrium and sums in IEEE double      */
    CDBM_FP32_BULK = 1,   /* state f and the NND transport in IEEE single; the     */
                          /* conserved sums, the moment shift and the equilibrium  */
                          /* product in double; f_eq is rounded to single when it  */
                          /* enters the stage update                               */
    CDBM_FP32_DF64 = 2,   /* as CDBM_FP32_BULK, with the sums, moment shift and    */
                          /* equilibrium product in double-float arithmetic (pairs */
                          /* of floats) on the FP32 pipe, with an absolute error   */
                          /* of a few 2^-47 of the reference equilibrium F         */
    CDBM_FP32_DEV = 3     /* everything in IEEE single: the state as its deviation */
                          /* from F and the equilibrium formed from the deviations */
                          /* of the moments from F's (no value of the size of F    */
                          /* enters a difference; the block product compensated;   */
                          /* mass, momentum and energy projected back onto the     */
                          /* cell's), with an error of a few 2^-24 of the          */
                          /* deviation: as accurate as CDBM_FP32_BULK on flows     */
                          /* near the reference state, 2-4x less on strong shocks  */
                          /* (Sod, 10^4 steps: 2.1e-5 relative L2 density error).  */
                          /* Not the FP64 moment shift and product of              */
                          /* CDBM_FP32_BULK                                        */
} cdbm_precision;

/* Time integrator.  The paper names a second-order Runge-Kutta scheme without
 * printing it (Sec. 2): TVD is f1 = f + dt L(f), f <- (f + f1 + dt L(f1)) / 2;
 * MIDPOINT is fh = f + dt/2 L(f), f <- f + dt L(fh). */
typedef enum { CDBM_RK2_TVD = 0, CDBM_RK2_MIDPOINT = 1 } cdbm_rk;

/*
 * cdbm_create -- validates the run and builds a context (Sec. 2, Eqs. 1-7).
 *   grid, vset   : see above (host memory, copied).
 *   I            : extra degrees of freedom, I >= 0 (Eq. 5).
 *   tau, dt      : relaxation time (Eq. 1) and time step, both > 0.
 *   precision    : cdbm_precision.
 *   cuda_stream  : cudaStream_t for all work of the context (NULL = legacy stream).
 *   allocator    : NULL or a cdbm_allocator (copied).
 *   out          : receives the context.
 * The context owns the state f (two [16][ny][nx] buffers) and a few small
 * scratch buffers; the state starts unset until cdbm_init or cdbm_set_state.
 * Errors: CDBM_EINVAL for nx or ny < 1, dx, dy, dt, tau <= 0, I < 0 or non-finite
 * input, a time step beyond the scheme's limits (max_i(|v_ix| dt/dx + |v_iy| dt/dy)
 * > 1, or dt/tau > 2, outside the real stability interval of RK2); CDBM_ESINGULAR
 * when the central-moment matrix at u = 0 (Eq. 6) is singular or has condition
 * number above 1e12; CDBM_ENOMEM; CDBM_ECUDA.  On error *out is NULL.
 */
cdbm_status cdbm_create(const cdbm_grid *grid, const cdbm_vset *vset, double I, double tau,
                        double dt, int precision, void *cuda_stream,
                        const cdbm_allocator *allocator, cdbm_ctx **out);

/* Chooses the Runge-Kutta variant (default CDBM_RK2_TVD). */
cdbm_status cdbm_set_rk(cdbm_ctx *ctx, int rk);

/*
 * cdbm_init -- sets f = f_eq(rho, u, T) in every cell (Eqs. 5-7), time 0.
 * rho, ux, uy, T: [ny][nx], host or device.
 */
cdbm_status cdbm_init(cdbm_ctx *ctx, const double *rho, const double *ux, const double *uy,
                      const double *T);

/*
 * cdbm_step -- advances the state by nsteps >= 0 time steps of Eq. (1): per step two
 * fused Runge-Kutta stage kernels (rho, u, T -> f_eq -> BGK + NND transport of all
 * 16 velocities -> stage update).  Launches are replayed from a CUDA graph.  A 1-D
 * grid (ny = 1) small enough for one thread-block cluster (at most 16 x 64 cells for
 * CDBM_FP64, 16 x 256 for the three single-precision states) instead runs all nsteps
 * in one persistent launch with its state in the cluster's shared memory; the
 * results are the same bit for bit for the single-precision states and the same to
 * rounding for CDBM_FP64, whose cluster kernel splits each cell over four threads.
 * Asynchronous; a non-physical state is reported by the next cdbm_sync.
 */
cdbm_status cdbm_step(cdbm_ctx *ctx, int nsteps);

/* Enables (default) or disables the small-grid paths of cdbm_step for 1-D grids: the
 * persistent cluster kernel, and for CDBM_FP64 tubes of up to 8192 cells the stage
 * kernel that splits each cell over four threads.  Disabled, those grids step with
 * the one-cell-per-thread stage kernel like any other. */
cdbm_status cdbm_set_small_grid_path(cdbm_ctx *ctx, int enable);

/* Enables (default) or disables the row-marching stage kernels on 2-D grids, which
 * carry the y differences of a run of rows in shared memory (and, for
 * CDBM_FP32_DF64, advance two columns per thread with packed FP32x2 arithmetic);
 * disabled, every stage runs one cell per thread.  Both give the same results bit
 * for bit; the switch serves cross-checks and timing.  EINVAL for a NULL context. */
cdbm_status cdbm_set_row_marching(cdbm_ctx *ctx, int enable);

/*
 * cdbm_macros -- writes rho, u_x, u_y, T of the current state ([ny][nx] each,
 * host or device; a NULL pointer skips that field).  With any host pointer the
 * call returns after the copy has finished.
 */
cdbm_status cdbm_macros(cdbm_ctx *ctx, double *rho, double *ux, double *uy, double *T);

/*
 * cdbm_tne -- nonequilibrium central moments of the current state, Eqs. (8)-(11):
 * out[k][ny][nx], k = 0..11 = rows 5..16 of Eq. (6) applied to f - f_eq:
 * Delta2 {xx, xy, yy}, Delta31 {x, y}, Delta3 {xxx, xxy, xyy, yyy},
 * Delta42 {xx, xy, yy}.  Computed as the central moments of f about u minus the
 * prescribed central moments of Eq. (7) (equal to M(u) f_eq by the definition of
 * f_eq).  out: host or device (a host copy synchronises the stream).
 */
cdbm_status cdbm_tne(cdbm_ctx *ctx, double *out);

/*
 * cdbm_conserved_sums -- domain totals of rho, rho u_x, rho u_y and
 * sum_i f_i (v_i^2 + eta_i^2) (twice the total energy) into out[4] (host):
 * each velocity plane is summed over the cells in double precision, then the 16
 * plane totals are weighted.  Deterministic (fixed reduction order).  Synchronous.
 */
cdbm_status cdbm_conserved_sums(cdbm_ctx *ctx, double out[4]);

/* Copies the state f ([16][ny][nx] doubles, host or device) and the time out / in;
 * a single-precision state (CDBM_FP32_BULK, CDBM_FP32_DF64, CDBM_FP32_DEV) is widened
 * on the way out and rounded on the way in. */
cdbm_status cdbm_get_state(cdbm_ctx *ctx, double *f, double *t);
cdbm_status cdbm_set_state(cdbm_ctx *ctx, const double *f, double t);

/* Device pointer of the state f ([16][ny][nx], owned by the context, valid until
 * cdbm_destroy; steps update it in place): doubles for CDBM_FP64, floats (the
 * deviation g = f - F from the reference equilibrium F) for CDBM_FP32_BULK,
 * CDBM_FP32_DF64 and CDBM_FP32_DEV. */
cdbm_status cdbm_state_ptr(cdbm_ctx *ctx, void **f);

/* Simulated time (host scalar). */
cdbm_status cdbm_time(const cdbm_ctx *ctx, double *t);

/* ------------------------------------------------------------------------------
 * Adjoint (reverse mode) of the time step, for gradients of a loss of the final
 * state with respect to the initial fields and tau.  Requires CDBM_FP64,
 * CDBM_RK2_TVD and periodic boundaries on every axis with more than one cell.
 * The limiter enters through its subgradient: the derivative of the branch the
 * forward pass took (1 for the argument minmod returned, 0 for the other, 0 when it
 * returned 0).  Pointers are device pointers.
 * ---------------------------------------------------------------------------- */

/* Runs nsteps >= 1 steps like cdbm_step from the current state and records a
 * checkpoint of the state every `every` steps (ceil(nsteps / every) states of
 * [16][ny][nx] doubles, allocated through the context allocator).  The run must be
 * the last thing done to the state before cdbm_adjoint_backward. */
cdbm_status cdbm_adjoint_forward(cdbm_ctx *ctx, int nsteps, int every);

/* Given fbar = dL/df of the state at the end of the recorded run ([16][ny][nx]),
 * writes dL/drho0, dL/du_x0, dL/du_y0, dL/dT0 of the fields the state was
 * initialised from by cdbm_init ([ny][nx] each; NULL skips) and dL/dtau (host
 * scalar; NULL skips).  Each segment between checkpoints is recomputed forward
 * (min(every, nsteps) states held at once, plus as many Runge-Kutta stage-1
 * states when the allocator can provide them; without those the sweep recomputes
 * each stage-1 state), then swept backward through the transposed stages.
 * Synchronous.  Errors: CDBM_EINVAL without a recorded run that ends at the
 * current state; CDBM_ENOMEM. */
cdbm_status cdbm_adjoint_backward(cdbm_ctx *ctx, const double *fbar, double *grad_rho, double *grad_ux,
                                  double *grad_uy, double *grad_T, double *grad_tau);

/* Linearisation of the minmod limiter N = minmod(U_{k+s}, U_k) (Eq. 16) used by
 * cdbm_adjoint_backward.  EXACT is the derivative of the branch the forward pass
 * took, i.e. the exact derivative of the discrete step.  Where the limiter picks the
 * downwind slope beside an upwind pick, that linearisation is anti-diffusive, and on
 * fine grids over thousands of steps the exact adjoint can grow without bound while
 * finite differences of the forward run stay finite (the forward map is then rough
 * at perturbations below ~1e-5).  The two frozen modes are the usual approximate
 * linearisations for that regime: FROZEN_RATIO holds the limiter value
 * phi = N / U_k in [0, 1] fixed (dN = phi dU_k); FROZEN holds N fixed (dN = 0, a
 * first-order upwind linearisation of the transport).  Neither is part of the
 * paper's scheme; they trade exactness for a bounded adjoint. */
typedef enum {
    CDBM_ADJ_LIMITER_EXACT = 0,
    CDBM_ADJ_LIMITER_FROZEN_RATIO = 1,
    CDBM_ADJ_LIMITER_FROZEN = 2
} cdbm_adj_limiter;

/* Selects the limiter linearisation (default CDBM_ADJ_LIMITER_EXACT).  Errors:
 * CDBM_EINVAL for an unknown mode. */
cdbm_status cdbm_adjoint_set_limiter(cdbm_ctx *ctx, int mode);

/* fbar = (d(rho, u_x, u_y, T)/df)^T (rho_bar, ux_bar, uy_bar, T_bar) at the current
 * state (the read-out of cdbm_macros transposed); NULL cotangents count as zero. */
cdbm_status cdbm_macros_vjp(cdbm_ctx *ctx, const double *rho_bar, const double *ux_bar, const double *uy_bar,
                            const double *T_bar, double *fbar);

/* Waits for the context stream and reports a sticky CUDA error or the
 * device-side non-physical flag (CDBM_ENONPHYS). */
cdbm_status cdbm_sync(cdbm_ctx *ctx);

/* One-line description of the sticky error of ctx (NULL ctx: of the last failed
 * cdbm_create or cdbm_step_noalloc on this thread).  Never NULL. */
const char *cdbm_last_error(const cdbm_ctx *ctx);

/* Releases the context and its device memory (stream-ordered).  NULL is a no-op. */
void cdbm_destroy(cdbm_ctx *ctx);

/* ------------------------------------------------------------------------------
 * Batched ensembles of 1-D tubes.  Each tube is an independent Ny = 1 run of Eq. (1)
 * with zero-gradient ends (a shock tube), with its own number of cells, cell size,
 * I and initial state; all tubes share the velocity set, tau and dt.  The tubes are
 * concatenated along x: a batch field is [total_cells] (tube t at cells
 * offset_t .. offset_t + nx_t - 1, offsets in tube order); the state is
 * [16][total_cells].  One persistent kernel advances every tube through all
 * requested steps; a block owns a fixed set of whole tubes, so blocks never wait on
 * one another (block barriers only, between Runge-Kutta stages).  The two-stage TVD
 * scheme is used.  Precision: any cdbm_precision (the single-precision states with a
 * per-tube reference F = f_eq of the tube's mean rho and T).
 * ---------------------------------------------------------------------------- */
typedef struct cdbm_batch cdbm_batch;

/* Validates and builds a batch of ntubes tubes: nx[t] >= 1 cells of size dx[t] > 0
 * and I[t] >= 0 (at most 4 distinct values of I); host arrays, copied.  Errors as
 * cdbm_create (CFL checked per tube along x).  The initial tile is 128 threads per
 * block and 3 blocks per SM. */
cdbm_status cdbm_batch_create(int ntubes, const int *nx, const double *dx, const double *I,
                              const cdbm_vset *vset, double tau, double dt, int precision,
                              void *cuda_stream, const cdbm_allocator *allocator, cdbm_batch **out);

/* f = f_eq(rho, u, T) in every cell of every tube; fields [total_cells], host or
 * device.  Synchronous. */
cdbm_status cdbm_batch_init(cdbm_batch *b, const double *rho, const double *ux, const double *uy,
                            const double *T);

/* Advances every tube by nsteps >= 0 steps: one persistent launch, replayed from a
 * CUDA graph.  Asynchronous; cdbm_batch_sync reports a non-physical state. */
cdbm_status cdbm_batch_step(cdbm_batch *b, int nsteps);

/* Times the candidate tiles (64/128/256 threads per block x 1, 2, 3, 4 or 6 blocks
 * per SM, at most 1024 threads per SM; each with its own
 * longest-first partition of the tubes) over trial_steps steps, keeps
 * the fastest and reports it.  The state is saved before and restored after the
 * trials, and results do not depend on the tile. */
cdbm_status cdbm_batch_autotune(cdbm_batch *b, int trial_steps, int *threads, int *blocks_per_sm);

/* Sets the tile explicitly (threads 64, 128 or 256; blocks_per_sm 1..16). */
cdbm_status cdbm_batch_set_tile(cdbm_batch *b, int threads, int blocks_per_sm);

/* Enables (default) or disables the symmetric kernels.  When every tube starts with
 * u_y = 0 (checked by cdbm_batch_init), each tube's state is mirror-symmetric in y --
 * f_S = f_N, f_SE = f_NE, f_SW = f_NW -- and stays so, since the mirror images move
 * alike along x and j_y = 0 gives them equal equilibria.  The symmetric kernels then
 * compute the 10 distinct velocities only, drop the terms of j_y = 0, and write each
 * result to both mirror planes; their results equal the general kernels' bit for bit
 * (up to the sign of an exact zero).  Disabled, every batch runs the general
 * kernels.  EINVAL for a NULL batch. */
cdbm_status cdbm_batch_set_symmetric(cdbm_batch *b, int enable);

/* rho, u_x, u_y, T of every cell ([total_cells] each, host or device, NULL skips).
 * Synchronous. */
cdbm_status cdbm_batch_macros(cdbm_batch *b, double *rho, double *ux, double *uy, double *T);

/* Total cells and the current tile (threads per block, number of blocks). */
cdbm_status cdbm_batch_info(const cdbm_batch *b, long long *total_cells, int *threads, int *blocks);

/* Waits for the batch's stream; reports a sticky error or CDBM_ENONPHYS. */
cdbm_status cdbm_batch_sync(cdbm_batch *b);
const char *cdbm_batch_last_error(const cdbm_batch *b);
void cdbm_batch_destroy(cdbm_batch *b);

/* Largest grid (nx * ny cells) that cdbm_step_noalloc accepts. */
#define CDBM_NOALLOC_MAX_CELLS 32768

/*
 * cdbm_step_noalloc -- cdbm_step without a context and without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory -- a host code that owns all GPU memory through its own
 * pool and forbids other allocations inside its time loop, a plug-in that is handed
 * device buffers but no allocator, or a loop where cudaMalloc's implicit device
 * synchronisation is not acceptable.
 *   grid, vset, I, tau, dt : as for cdbm_create, with the same validation.
 *   f            : device pointer to the caller's state [16][ny][nx] (for example from
 *                  cdbm_get_state or an equilibrium the caller built), advanced in
 *                  place by nsteps >= 0 two-stage TVD Runge-Kutta steps.  The result
 *                  matches cdbm_step's on the same state to rounding (within 1e-12
 *                  relative max-norm): both apply the same per-cell operations, but
 *                  on a short 1-D grid cdbm_step may run them in its cluster kernel,
 *                  whose compiled arithmetic can round differently.  On 2-D grids
 *                  both run the same stage kernels and agree bit for bit.
 *   cuda_stream  : stream for the work (NULL = legacy stream).
 * Scratch: the stage-1 buffer and the error flag live in one fixed device array of
 * the library (16 * CDBM_NOALLOC_MAX_CELLS doubles plus 256 bytes, i.e. 4 MiB), which
 * every GPU that loads the library holds until the process exits.  The call makes no
 * cudaMalloc/cudaFree or other allocating call.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, with the device current).  All
 * calls on a device share the array and it keeps the last call's contents (the flag
 * is cleared at the start of each call), so calls that overlap on the GPU -- on
 * different streams or host threads -- race and must be serialised by the caller.
 * Synchronous: every call ends by copying the flag to the host and waiting for its
 * stream, so it cannot be called while a stream is being captured into a CUDA graph.
 * Errors: CDBM_EINVAL (as
 * cdbm_create, f NULL, nsteps < 0, or nx * ny > CDBM_NOALLOC_MAX_CELLS),
 * CDBM_ESINGULAR, CDBM_ECUDA, CDBM_ENONPHYS (the state went non-physical; f holds the
 * result of the last step).  Messages go to cdbm_last_error(NULL).
 */
cdbm_status cdbm_step_noalloc(const cdbm_grid *grid, const cdbm_vset *vset, double I, double tau,
                              double dt, double *f, int nsteps, void *cuda_stream);

/* ------------------------------------------------------------------------------
 * Diagnostics.  The paper has no counterpart: each runs one device building block,
 * or one hardware rate probe, on its own, so that tests can bound a building block
 * against IEEE arithmetic and the benchmark can measure the rate that bounds the
 * FP64 stage kernels in the same process.  Both are asynchronous on cuda_stream
 * (NULL = legacy stream); messages go to cdbm_last_error(NULL).
 * ---------------------------------------------------------------------------- */

/* y[k] = 1 / x[k] for 0 <= k < n, by the reciprocal the kernels use for 1 / rho
 * (the hardware estimate refined by one cubic Newton-Raphson step).  x, y: device
 * arrays of n doubles; x positive, finite and normal (subnormal inputs are flushed
 * to zero by the estimate).  Errors: CDBM_EINVAL (n < 0, NULL pointer with n > 0),
 * CDBM_ECUDA. */
cdbm_status cdbm_diag_rcp64(const double *x, double *y, long long n, void *cuda_stream);

/* FP64 fused multiply-add probe: blocks x threads threads each run 8 independent
 * chains of `iters` dependent FMAs and write one double to out (device,
 * blocks * threads doubles, caller-owned).  *flops (host, may be NULL) receives the
 * flop count, 2 per FMA; the caller times the launch with events on cuda_stream.
 * Errors: CDBM_EINVAL (NULL out, blocks < 1, threads not a multiple of 32 in
 * [32, 1024], iters < 1), CDBM_ECUDA. */
cdbm_status cdbm_diag_fp64_fma(double *out, int blocks, int threads, int iters, void *cuda_stream,
                               double *flops);

#ifdef __cplusplus
}
#endif

#endif /* CDBM_H */
