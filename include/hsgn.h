/*
 * hsgn.h -- C ABI of the GB300 (sm_103a) library for the semi-implicit IMEX
 * time step of the hyperbolic Serre-Green-Naghdi (hSGN) equations in 1D.
 *
 * Method: E. Macca, W. Boscheri, M. Ricchiuto, "Semi-implicit strategies for
 * the Serre-Green-Naghdi equations in hyperbolic form" (arXiv 2510.07539).
 * The state of an instance is U = (h, q = h u, m = h eta, r = h w) on a
 * uniform grid of n cells (Sec. 2.2, eq. (hSGN_eq)); one step is the two-stage
 * IMEX Runge-Kutta scheme of Sec. 3.2 (eq. (tableau), efficient form), each
 * stage being the fully-discrete semi-implicit update of Sec. 4.2 (eq.
 * (GN_hyp_eq_semi_fully_discrete)): explicit Rusanov fluxes with linear
 * reconstruction (Sec. 4.1), a symmetric tridiagonal system for the depth
 * (cyclic when periodic), and the back-substitution for q, h eta, h w.
 *
 * Conventions shared by every entry point:
 *  - Return value: HSGN_OK (0) or one of the HSGN_ERR_* codes below. No entry
 *    point throws, aborts or prints.
 *  - Arrays are contiguous FP64 with n elements, 8-byte aligned. Unless a
 *    description says otherwise a pointer may address device memory, pinned
 *    host memory or pageable host memory (copies use cudaMemcpyDefault).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it; functions that say "synchronises"
 *    wait for the stream before returning.
 *  - Errors found on the device (non-positive depth, beta <= 0 or a
 *    non-positive pivot, non-finite values) are accumulated in a device error
 *    word and reported by the next synchronising call (hsgn_run, hsgn_check,
 *    hsgn_get_state), which also clears the word. After such an error the
 *    state is undefined until the next hsgn_set_state.
 *  - No call is thread-safe on one handle; distinct handles are independent.
 */
#ifndef HSGN_H
#define HSGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HSGN_OK = 0,
    HSGN_ERR_INVALID_ARG = 1,       /* bad size, pointer, flag or parameter */
    HSGN_ERR_CUDA = 2,              /* a CUDA runtime call failed */
    HSGN_ERR_NONPOSITIVE_DEPTH = 3, /* a depth used as a divisor was <= 0 */
    HSGN_ERR_NOT_COERCIVE = 4,      /* beta <= 0 or a non-positive pivot */
    HSGN_ERR_NONFINITE = 5,         /* NaN or Inf produced */
    HSGN_ERR_UNIMPLEMENTED = 6,     /* entry point or flag not built yet */
    HSGN_ERR_OUT_OF_MEMORY = 7,
    HSGN_ERR_TRUNCATION = 8         /* windowed depth solve: the coupling of the depth
                                     * system decays too slowly for the window overlap
                                     * (time step too large); HSGN_EXACT_SOLVE solves
                                     * it without truncation */
};

/* boundary conditions (reading of the paper, which states none):
 * periodic = indices wrap, cyclic matrix; transmissive = zero-order ghost
 * copies of every per-cell quantity, Neumann end rows. */
#define HSGN_BC_PERIODIC 0
#define HSGN_BC_TRANSMISSIVE 1

/* flags of hsgn_create */
#define HSGN_FP64 0x0          /* every operation in FP64 */
#define HSGN_MIXED 0x1         /* fluxes, coefficients and the depth solve in FP32
                                * on increments; state, base-state differences and
                                * the accumulation in FP64 (with HSGN_EXACT_SOLVE)
                                * or double-float pairs (below); the depth is
                                * updated in flux form (mass conserved to the
                                * rounding of the state).
                                * One launch per stage: each CTA solves the depth
                                * system of its tile on a window that overlaps the
                                * neighbouring tiles by 64 rows and drops the
                                * coupling beyond it (the depth matrix is strictly
                                * diagonally dominant, so that coupling decays
                                * geometrically; each CTA checks the decay bound and
                                * reports HSGN_ERR_TRUNCATION when the dropped part
                                * could exceed 2^-30 of the increment). The state
                                * alternates between two device buffers and is held
                                * as double-float pairs (hi + lo, 48-bit significand;
                                * set/get_state convert from and to doubles), so the
                                * stage runs without double-precision instructions.
                                * hsgn_stage is not available in this form. */
#define HSGN_DOUBLE_FLOAT 0x8  /* FP64-class arithmetic on the single-precision
                                * pipe: every value of the stage (state, fluxes,
                                * coefficients, the depth solve and the
                                * back-substitution) is a double-float pair
                                * (hi + lo, 48-bit significand; about 2^-47
                                * relative error per operation), so that one step
                                * stays within 1e-12 of the FP64 scheme while no
                                * double-precision instruction runs. One launch
                                * per stage on overlapping windows as described
                                * under HSGN_MIXED, with the truncation bound
                                * checked against 2^-50 and an overlap of 48 to 96
                                * rows that follows the coupling (hsgn_df_overlap;
                                * HSGN_ERR_TRUNCATION above about CFL_IMEX 7 for
                                * smooth states); increment form, the state
                                * alternating between two device buffers of pairs
                                * (set/get_state convert). Single instances, the
                                * paper's scheme, flat or with HSGN_WELL_BALANCED
                                * (the bottom form in pairs throughout); not
                                * combinable with HSGN_EXACT_SOLVE
                                * (HSGN_ERR_UNIMPLEMENTED), and hsgn_adjoint stays
                                * with the FP64 form. hsgn_stage works in this
                                * form and leaves the state untouched.
                                * HSGN_DOUBLE_FLOAT | HSGN_MIXED is the precision
                                * split with an FP64-class solve: reconstruction,
                                * fluxes, starred increments and coefficients in
                                * FP32; rows, depth solve, back-substitution and
                                * the state accumulation in pairs (flat bottom
                                * only: with HSGN_WELL_BALANCED as well,
                                * HSGN_ERR_UNIMPLEMENTED). */
#define HSGN_EXACT_SOLVE 0x4   /* with HSGN_MIXED: solve the depth system exactly
                                * through the global separator system (three
                                * launches per stage, state updated in place) */

/* Time-stepping scheme (flags & HSGN_SCHEME_MASK). The default is the paper's
 * method; the others are the comparisons it reports or names, FP64 flat bottom
 * only (HSGN_ERR_UNIMPLEMENTED with HSGN_MIXED or HSGN_WELL_BALANCED):
 *   PRINTED  the two-stage IMEX tableau of Sec. 3.2, eq. (tableau)
 *   ARS222   the three-stage ARS(2,2,2) double tableau (explicit first stage)
 *            in the generic stage form of Sec. 3.2
 *   SI1      first-order semi-implicit: one stage of eq.
 *            (GN_hyp_eq_semi_fully_discrete) with tau = dt, no reconstruction
 *   EX_HEUN  explicit hSGN (Sec. 4.4, eq. (GN_hyp_eq_explicit)), Heun's method,
 *            centred linear reconstruction; needs dt <= CFL dx / nu_max with
 *            CFL about 0.4 (hsgn_suggest_dt with that CFL)
 *   EX_EULER explicit hSGN, forward Euler, no reconstruction
 * The explicit schemes treat every wave explicitly: their global Rusanov
 * speed is the spectral radius max(|u| + c), c^2 = g h + (lambda/3) eta^2/h^2,
 * of the step's state, where the semi-implicit schemes use max |u|. */
#define HSGN_SCHEME_PRINTED 0x000
#define HSGN_SCHEME_ARS222 0x100
#define HSGN_SCHEME_SI1 0x200
#define HSGN_SCHEME_EX_HEUN 0x300
#define HSGN_SCHEME_EX_EULER 0x400
#define HSGN_SCHEME_MASK 0x700

#define HSGN_RUSANOV_LOCAL 0x10 /* Rusanov speed max(|u^L|,|u^R|) per face instead
                                 * of the global max |u^n| of the step */
#define HSGN_WELL_BALANCED 0x2  /* variable bottom b(x) (Sec. 2.3, eq. (hSGNb_eq))
                                 * in a well-balanced extension of the flat-bottom
                                 * scheme, which the paper does not derive: the
                                 * (h eta) equation gets the explicit source
                                 * -(3/2) h u b_x, and the pressure jump plus the
                                 * bottom force -(g h + (3/2) p~) b_x enter the
                                 * depth rows and the momentum as face forces
                                 * linearised about U_l, so that a lake at rest
                                 * (u = 0, eta = h, w = 0, h + b constant) stays at
                                 * rest. FP64, HSGN_DOUBLE_FLOAT (every value a
                                 * pair), or HSGN_MIXED on the windowed kernel
                                 * (the bottom held as double-float pairs, the
                                 * free-surface jumps taken from the pairs;
                                 * HSGN_ERR_UNIMPLEMENTED with HSGN_EXACT_SOLVE);
                                 * single instances only. */

typedef struct {
    int64_t n;       /* number of cells, n >= 3 */
    double x_left;   /* domain [x_left, x_right], dx = (x_right - x_left)/n */
    double x_right;
    int32_t bc;      /* HSGN_BC_PERIODIC or HSGN_BC_TRANSMISSIVE */
    int32_t reserved; /* must be 0 */
} hsgn_grid_t;

typedef struct hsgn_s* hsgn_handle_t;

/* Create an instance: grid, gravity g > 0, relaxation parameter lambda >= 0
 * (Sec. 2.2, eq. (hSGN_eq)). `bathymetry`: NULL for a flat bottom, else n
 * bottom elevations b_i at the cell centres (host or device memory, copied
 * during the call; the caller keeps ownership), which requires
 * HSGN_WELL_BALANCED (INVALID_ARG otherwise). HSGN_WELL_BALANCED with NULL
 * runs the well-balanced form over a flat bottom. Allocates the state and
 * workspace on the current device: about 17 doubles per cell in FP64 (19 with
 * a bottom); 80 bytes per cell with HSGN_MIXED (two state buffers of
 * double-float pairs and four single-precision increments; 88 with a bottom);
 * 4 doubles and 16 floats per cell with HSGN_MIXED | HSGN_EXACT_SOLVE.
 * On success *out owns them until hsgn_destroy. */
int hsgn_create(const hsgn_grid_t* grid, double g, double lambda, const double* bathymetry,
                int32_t flags, hsgn_handle_t* out);

/* Copy a state in (U = (h, q, h eta, h w), n values each) and recompute the
 * global Rusanov speed. The caller keeps ownership of the arrays. Does not
 * synchronise; the arrays must stay valid until the stream reaches the copy.
 * With HSGN_MIXED (windowed) the state is held as double-float pairs: arrays
 * in this device's memory are converted directly, host arrays are copied by
 * the copy engines into a device buffer and converted there (pageable host
 * memory makes the copy synchronous with respect to the host). */
int hsgn_set_state(hsgn_handle_t h, const double* depth, const double* q, const double* heta,
                   const double* hw, void* stream);

/* Copy the state out (the pairs of the windowed form are summed exactly into
 * doubles). Synchronises `stream` only and reports pending device errors. */
int hsgn_get_state(hsgn_handle_t h, double* depth, double* q, double* heta, double* hw,
                   void* stream);

/* hsgn_get_state without the synchronisation: the copy out is enqueued on
 * `stream` and the arrays hold the state once the stream reaches it; pending
 * device errors are reported by the next synchronising call. The windowed form
 * stages the pairs through its idle state buffer, which the next step
 * overwrites: enqueue further steps on the same stream (or synchronise first).
 * Lets a host loop pipeline state in, steps and state out over several
 * handles and streams. */
int hsgn_copy_state_out(hsgn_handle_t h, double* depth, double* q, double* heta, double* hw,
                        void* stream);

/* One IMEX step of size dt > 0 (Sec. 3.2): two implicit stages with
 * tau = gamma dt, gamma = 1 - 1/sqrt(2). Enqueues six kernels; does not
 * synchronise. */
int hsgn_step(hsgn_handle_t h, double dt, void* stream);

/* n_steps >= 0 steps of size dt: one step is captured once per dt into a CUDA
 * graph and replayed. Synchronises and reports pending device errors. */
int hsgn_run(hsgn_handle_t h, double dt, int64_t n_steps, void* stream);

/* Enqueue n_steps >= 0 steps as CUDA-graph replays (same graph as hsgn_run)
 * without synchronising; errors surface at the next synchronising call. */
int hsgn_enqueue(hsgn_handle_t h, double dt, int64_t n_steps, void* stream);

/* Per-kernel timing. While enabled, hsgn_step and hsgn_stage record a CUDA
 * event pair around each kernel launch on the launch stream (graph replays are
 * not timed). hsgn_profile_read waits for the recorded events, adds their
 * elapsed times to ms[kind] and their count to launches[kind] for the
 * HSGN_PROF_KINDS kinds below (either pointer may be NULL), and clears the
 * record when `reset` is non-zero. */
#define HSGN_PROF_ASSEMBLE 0 /* flux + assembly + block elimination kernel */
#define HSGN_PROF_REDUCED 1  /* separator-system solve */
#define HSGN_PROF_BACKSUB 2  /* back-substitution kernel */
#define HSGN_PROF_KINDS 3
int hsgn_profile(hsgn_handle_t h, int32_t enable);
int hsgn_profile_read(hsgn_handle_t h, double* ms, int64_t* launches, int32_t reset);

/* n_steps steps, each with its own time step from the rule of Sec. 5
 * (Sec. 3.3, eq. (eq:MCFL)) applied to the state it starts from:
 * dt = cfl dx / nu_max, reduced to mcfl dx / u_max if the material CFL
 * u_max dt / dx would exceed mcfl (mcfl = 0 disables that test), with
 * nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2) as in hsgn_suggest_dt. The
 * maxima of each new state are folded on the device by the stage that writes
 * it and the next step reads them there, so steps run back to back (one
 * captured graph per state buffer) with no host round trip. *t_advanced
 * (host) receives the sum of the time steps taken. HSGN_DOUBLE_FLOAT forms
 * with the global Rusanov speed only (HSGN_ERR_UNIMPLEMENTED otherwise).
 * Synchronises and reports device errors like hsgn_run. */
int hsgn_run_cfl(hsgn_handle_t h, double cfl, double mcfl, int64_t n_steps, double* t_advanced,
                 void* stream);

/* Window overlap of the HSGN_DOUBLE_FLOAT form (not part of the paper's
 * method: how far the windowed depth solve of Sec. 4.2 must reach). Each
 * window checks that the decay of the depth coupling over its overlap stays
 * under 2^-50, and stage 2 of every step records on the device how many rows
 * of overlap its windows needed. Every synchronising call (hsgn_run,
 * hsgn_run_cfl, hsgn_check, this one) sets the overlap of the steps enqueued
 * after it to that record plus 5 rows, rounded up to a multiple of 8 within
 * [48, 96] (64 while nothing is recorded; longer tiles for a narrower
 * overlap); captured step graphs are re-captured when it changes. A window
 * whose overlap misses the bound all the same (the coupling grew since the
 * record) redoes its tile in pieces with 96 rows, so the overlap changes only
 * the speed; beyond 96 rows the step reports HSGN_ERR_TRUNCATION. A new state
 * (hsgn_set_state) starts with nothing recorded. *rows_needed (host) receives
 * the rows recorded by the last step (0 if none), *overlap the overlap of the
 * next steps. Synchronises the stream. HSGN_ERR_UNIMPLEMENTED for other forms. */
int hsgn_df_overlap(hsgn_handle_t h, int32_t* rows_needed, int32_t* overlap, void* stream);

/* Synchronise the stream and report (and clear) pending device errors. */
int hsgn_check(hsgn_handle_t h, void* stream);

/* Time-step rule of Sec. 5 on the current state: dt = cfl dx / nu_max with
 * nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2); if u_max dt / dx > mcfl then
 * dt = mcfl dx / u_max (mcfl <= 0 disables that test). Synchronises. */
int hsgn_suggest_dt(hsgn_handle_t h, double cfl, double mcfl, double* dt_out, void* stream);

/* One implicit stage S(U_b, U_l, tau) of Sec. 4.2 on caller arrays: base
 * state `base` (the additive old values), linearisation state `lin` (fluxes
 * and coefficients), stage step tau > 0, and Rusanov speed `speed` (ignored
 * with HSGN_RUSANOV_LOCAL). base, lin, out: 4 device pointers each (h, q, m, r),
 * out must not alias base or lin. Uses the handle's grid, parameters and
 * workspace; does not touch its state. Does not synchronise. */
int hsgn_stage(hsgn_handle_t h, const double* const base[4], const double* const lin[4],
               double tau, double speed, double* const out[4], void* stream);

/* Discrete adjoint of a run (the gradient of a gauge misfit).
 *
 * Runs n_steps steps of the paper's scheme (Sec. 3.2) of size dt from the
 * current state and returns
 *   J = 1/2 sum_{s=1..n_steps} sum_g (h_{c_g}^s - d_{s,g})^2 dt
 * in *misfit (host), where h^s is the depth after step s, c_g = gauge_cells[g]
 * (host array of n_gauges cells in [0, n)) and d = gauge_data (host or device,
 * n_steps x n_gauges, row-major). The gradient of J with respect to the
 * initial state goes to grad_state[0..3] (device arrays of n for h, q, h eta,
 * h w; grad_state or any entry may be NULL) and with respect to the bottom to
 * grad_bathymetry (device array of n, may be NULL).
 *
 * The gradient is the exact derivative of the discrete step (every operation
 * of the stage reversed: back-substitution, the depth solve through a second
 * solve with the transposed matrix, rows, face forces, coefficients, starred
 * values, Rusanov fluxes and reconstruction), including the global Rusanov
 * speed max|u| of each step through its first argmax cell. States are stored
 * every checkpoint_every steps and recomputed segment by segment in the
 * reverse sweep (memory: n_steps/checkpoint_every + checkpoint_every + 16
 * states of 4 n doubles, allocated during the call).
 *
 * Requires an FP64 instance created with HSGN_WELL_BALANCED (a NULL bottom
 * gives the flat-bottom case), the paper's scheme and the global Rusanov speed
 * (HSGN_ERR_UNIMPLEMENTED otherwise); the paper has no adjoint. On return the
 * state is the state after n_steps steps. Synchronises. */
int hsgn_adjoint(hsgn_handle_t h, double dt, int64_t n_steps, int64_t n_gauges,
                 const int64_t* gauge_cells, const double* gauge_data, int64_t checkpoint_every,
                 double* const grad_state[4], double* grad_bathymetry, double* misfit,
                 void* stream);

/* ---------------------------------------------------------------------------
 * Batches of independent instances (the batched workload of many 1D problems
 * of uneven length, relaxation parameter and time step). All instances of a
 * batch share g and the boundary condition and are advanced together by the
 * mixed-precision kernels (HSGN_MIXED is implied): one launch per kernel for
 * the whole batch, with the separator systems solved one warp per instance.
 * The state of a batch is the concatenation of the instances' states (packed,
 * instance k occupying cells offset_k .. offset_k + n_k - 1 of every array),
 * exchanged with hsgn_set_state / hsgn_get_state as for a single instance.
 * hsgn_step, hsgn_run and hsgn_enqueue take dt = 0 for a batch: each instance
 * uses the step set by hsgn_batched_set_dt. hsgn_stage, hsgn_suggest_dt and
 * hsgn_adjoint are not available for a batch.
 * ------------------------------------------------------------------------- */

/* count >= 1 instances; per instance: n[k] in [3, 65536] cells on
 * [x_left[k], x_right[k]] and lambda[k] >= 0 (host arrays). */
int hsgn_create_batched(int32_t count, const int64_t* n, const double* x_left,
                        const double* x_right, const double* lambda, double g, int32_t bc,
                        int32_t flags, hsgn_handle_t* out);

/* Per-instance time steps dt[k] > 0 (host array of `count`). Takes effect for
 * steps enqueued after the call; synchronises the device. */
int hsgn_batched_set_dt(hsgn_handle_t h, const double* dt);

/* Per-instance time-step rule of Sec. 5 (as hsgn_suggest_dt) on the current
 * state; dt_out: host array of `count`. Synchronises. */
int hsgn_batched_suggest_dt(hsgn_handle_t h, double cfl, double mcfl, double* dt_out,
                            void* stream);

/* Tiles of a batch (the windowed kernel; HSGN_ERR_UNIMPLEMENTED for a batch
 * created with HSGN_EXACT_SOLVE). variant[k] (host array of `count`) selects
 * the windowed kernel of instance k:
 *   0: 256 threads, 64-row window overlap, tiles of up to 894 rows (default);
 *   1: 128 threads, 64-row overlap, tiles of up to 382 rows (less padding for
 *      short instances);
 *   2: 256 threads, 32-row overlap, tiles of up to 958 rows;
 *   3: 128 threads, 32-row overlap, tiles of up to 446 rows.
 * The narrow overlap (2, 3) needs the depth coupling to decay fast (small
 * CFL numbers); each CTA checks its truncation bound (2^-30) and the next
 * synchronising call reports HSGN_ERR_TRUNCATION when it does not hold. Each
 * variant in use runs as one launch per stage over its instances' tiles.
 * Values outside 0 .. 3 give INVALID_ARG. Synchronises the device; the
 * results of the variants agree to the rounding of the single-precision
 * increments. */
int hsgn_batched_set_tiles(hsgn_handle_t h, const int32_t* variant);

/* The tile variant of every instance (0 .. 3, as hsgn_batched_set_tiles;
 * variant_out: host array of `count`), e.g. after hsgn_batched_autotune.
 * HSGN_ERR_UNIMPLEMENTED for a batch created with HSGN_EXACT_SOLVE. */
int hsgn_batched_get_tiles(hsgn_handle_t h, int32_t* variant_out);

/* Autotuner of the tiles: from the current state (restored exactly after every
 * trial), times `steps` >= 1 steps with every instance on each of the four
 * variants of hsgn_batched_set_tiles in turn (a variant that reports
 * HSGN_ERR_TRUNCATION for this batch and time step is ruled out); from these
 * a cost per tile of each variant gives each instance the variant of smallest
 * predicted cost, and that assignment is timed when it mixes variants. The
 * fastest timed assignment is kept. ms_out (host, 5 doubles, may be NULL): ms
 * per step with every instance on variant 0, 1, 2, 3, then of the per-instance
 * assignment (NaN when not timed or ruled out); choice_out (may be NULL): the
 * variant kept for every instance (0 .. 3), or 4 for the per-instance
 * assignment. HSGN_ERR_TRUNCATION when every variant is ruled out. Needs
 * hsgn_batched_set_dt first (INVALID_ARG otherwise); allocates 32 bytes per
 * cell for the duration of the call; synchronises. */
int hsgn_batched_autotune(hsgn_handle_t h, int32_t steps, double* ms_out, int32_t* choice_out,
                          void* stream);

/* Release everything owned by the handle (NULL is accepted). */
void hsgn_destroy(hsgn_handle_t h);

/* Static, NUL-terminated description of an error code. */
const char* hsgn_error_string(int code);

/* Measured arithmetic peak of the current device, the denominator of the
 * roofline of the arithmetic-bound stage kernels (the paper has no
 * counterpart): independent fused multiply-add chains in single (bits = 32)
 * or double (bits = 64) precision on every SM, timed with CUDA events; a
 * multiply-add counts two operations. *tflops receives TFLOP/s. Allocates a
 * small output buffer on `stream` (stream-ordered) and synchronises. */
int hsgn_fma_peak(int32_t bits, double* tflops, void* stream);

/* ---------------------------------------------------------------------------
 * Tridiagonal component (the depth solve of Sec. 4.2, Delta[hbar] = h^dagger)
 * ------------------------------------------------------------------------- */

/* Bytes of device workspace hsgn_tridiag_solve needs for n rows. */
int hsgn_tridiag_workspace_bytes(int64_t n, size_t* bytes);

/* Solve a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i], i = 0..n-1, n >= 1.
 * periodic != 0: a[0] couples x[n-1] and c[n-1] couples x[0] (cyclic);
 * periodic == 0: a[0] and c[n-1] are ignored. a, b, c, d, x: device pointers;
 * x may alias d. The matrix must be an M-matrix-like, diagonally dominant
 * system (the hSGN depth matrix is); no pivoting is done. A non-positive pivot
 * is reported as HSGN_ERR_NOT_COERCIVE. `workspace` (device, 256-byte aligned,
 * at least hsgn_tridiag_workspace_bytes) is caller-owned scratch.
 * Synchronises and reports device errors. */
int hsgn_tridiag_solve(int64_t n, int32_t periodic, const double* a, const double* b,
                       const double* c, const double* d, double* x, void* workspace,
                       size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Tridiagonal solve without any allocation. The paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc: host loops with a
 * latency budget (cudaMalloc and cudaFree may block and synchronise the device)
 * and programs whose device memory belongs to another allocator (for example
 * PyTorch's caching allocator), which cannot hand raw cudaMalloc'd scratch to a
 * library. It solves the same system as hsgn_tridiag_solve, with the same
 * arguments minus the workspace, and gives the same result.
 *
 * Scratch: one file-scope device array of HSGN_TRIDIAG_NOALLOC_SCRATCH_BYTES
 * (about 6 MiB) inside the library; every GPU that loads the library keeps it
 * until the process exits. Sizes: 1 <= n <= HSGN_TRIDIAG_NOALLOC_MAX_N;
 * larger n returns HSGN_ERR_INVALID_ARG before any device work.
 * Set-up: the first call on each device, with that device current, looks up
 * the device address of the array (cudaGetSymbolAddress); make that first call
 * before any stream capture. The address is kept for the life of the process:
 * cudaDeviceReset, or anything else that destroys the device's primary
 * context, reloads the library's device code at a possibly different address,
 * so do not call this entry point on that device again in the same process
 * after such a reset. All calls share the one array, which keeps the
 * contents of the previous call; the call clears its error word itself, and
 * every other scratch value is written before it is read. Calls that overlap
 * on the GPU (other streams or threads) race on the array and must not be
 * issued. No cudaMalloc, cudaFree or allocating library routine is called.
 * Synchronises `stream` and reports device errors like hsgn_tridiag_solve.
 * --------------------------------------------------------------------------- */
#define HSGN_TRIDIAG_NOALLOC_MAX_N 262144
#define HSGN_TRIDIAG_NOALLOC_SCRATCH_BYTES 6522624 /* 6.2 MiB */
int hsgn_tridiag_solve_noalloc(int64_t n, int32_t periodic, const double* a, const double* b,
                               const double* c, const double* d, double* x, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HSGN_H */
