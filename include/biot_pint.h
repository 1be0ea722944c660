/*
 * biot_pint.h -- C ABI of the GB300 parallel-in-time Biot solver.
 *
 * Method: arxiv 2310.10430, "A Parallel-in-time Method Based on Preconditioner
 * for Biot's Model". The quasi-static two-field Biot model (Sec. 2.1, Eqs.
 * biotsys1-biotsys2) is discretised with stabilised P1-P1 elements and backward
 * Euler (Sec. 2.2, Eq. diseq1), giving one saddle-point system per time step
 * (Eq. fullysystem / axb):
 *
 *     AA x_n = A' x_{n-1} + f^n,   AA = [[A, B], [B^T, -(tau + beta/K) C]],
 *                                  A' = [[0, 0], [B^T, -(beta/K) C]].
 *
 * The inverted time stepping of Algorithms 2-3 (Sec. 3.2) swaps the loops: the
 * outer loop iterates the preconditioned solver, the inner loop runs over the
 * time steps. Every outer iteration ("sweep") forms, for all active time steps
 * at once, the residual r_n = f^n + A' x_{n-1} - AA x_n, applies the block
 * preconditioner P1 (Eq. p1, lower block triangular) or P2 (Eq. p2, block
 * diagonal) built on the approximate Schur complement S = (tau + beta/K) C, and
 * updates x_n with one cycle of the inner Krylov solver K(P, AA, X, b, n_iter).
 *
 * Conventions (all entry points):
 *  - Unknowns are node-interleaved: DOF 3*v + f, f = 0 (u_x), 1 (u_y), 2 (p);
 *    node v = j*(n+1) + i of the structured n x n grid (x fastest).
 *  - Host buffers are owned by the caller; device memory is owned by the
 *    context and released by biot_destroy. Work is stream-ordered on the CUDA
 *    stream given to biot_mesh_create; calls that return host data synchronise
 *    that stream before returning. The context also owns one non-blocking
 *    stream of the highest priority: the block-diagonal preconditioner runs its
 *    solves on A there, concurrently with its solves on S on the caller's
 *    stream, forked from and joined back to the caller's stream by events, so
 *    the ordering seen on the caller's stream is unchanged.
 *  - No C++ exception or exit() crosses the ABI. Every call returns a
 *    biot_status; biot_last_error() gives a one-line message for the last
 *    failure on that context. A call made in the wrong order returns
 *    BIOT_E_STATE and changes nothing.
 *  - A context is not thread safe; distinct contexts are independent.
 */
#ifndef BIOT_PINT_H
#define BIOT_PINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct biot_ctx biot_ctx;

typedef enum {
  BIOT_OK = 0,
  BIOT_E_INVALID = 1,        /* bad argument (null pointer, size, enum) */
  BIOT_E_OOM = 2,            /* device allocation failed */
  BIOT_E_CUDA = 3,           /* CUDA runtime error (message in biot_last_error) */
  BIOT_E_STATE = 4,          /* call made before the step it depends on */
  BIOT_E_NOT_CONVERGED = 5,  /* max_outer sweeps done, tolerance not met; state stays readable */
  BIOT_E_DIVERGED = 6,       /* residual non-finite or grew by more than 1e6 */
  BIOT_E_TIMEOUT = 7         /* a bounded device wait ran out (band-row bulk copy of a block solve) */
} biot_status;

typedef enum {
  BIOT_PRECOND_TRI = 1,      /* P1 = [[A, 0], [B^T, -S]], Eq. (p1) */
  BIOT_PRECOND_DIAG = 2      /* P2 = [[A, 0], [0, -S]],   Eq. (p2) */
} biot_precond_kind;

typedef enum {
  BIOT_FP64 = 0,             /* every kernel in FP64 */
  BIOT_FP32 = 1,             /* FP32 sweep (SpMM, preconditioner, Krylov), FP64 true residual + refinement */
  BIOT_BF16VAL_FP32ACC = 2   /* as BIOT_FP32 with the SpMM matrix values stored in BF16 */
} biot_precision;

typedef enum {
  BIOT_TERZAGHI = 0,         /* consolidation column: top load, drained top, fixed bottom, roller sides */
  BIOT_MMS_TRIG = 1,         /* manufactured cos t cos 3 pi x cos 3 pi y solution, Dirichlet on all sides (Sec. 4.1) */
  BIOT_BARRY_MERCER = 2,     /* point source -0.5 load delta_(a/4, b/4) sin(beta t), beta = (lambda + 2 mu) K / (a b);
                                drained, zero tangential displacement on every side (Sec. 4.2) */
  BIOT_MANDEL = 3            /* quarter domain under a rigid frictionless plate pressed with the force F = load
                                (Sec. 4.3): x = a drained and traction-free, x = 0 and y = 0 symmetry planes
                                (u_x = 0, u_y = 0, no flux), impervious top with u_y constant along x, imposed
                                by the penalty 1e4 (lambda + 2 mu) (u_y(i+1) - u_y(i))^2 / 2 over consecutive top
                                nodes, the force as the traction (0, -F / a); initial state the undrained response
                                of Sec. 4.3 (Skempton B = 1) */
} biot_problem;

typedef enum {
  BIOT_BETA_H2 = 0,          /* beta = h^2 / (4 (lambda + 2 mu)) (dimensionally consistent reading) */
  BIOT_BETA_H = 1,           /* beta = h / (4 (lambda + 2 mu)), as printed in Sec. 2.2 */
  BIOT_BETA_NONE = 2         /* no stabilisation */
} biot_beta_mode;

typedef enum {
  BIOT_SCHED_TOL = 0,        /* retire the oldest active step once its relative residual <= tol */
  BIOT_SCHED_PAPER = 1,      /* every step gets exactly `window` outer iterations (N_thread of Alg. 3) */
  BIOT_SCHED_EAGER = 2       /* as BIOT_SCHED_TOL with every step active from the first sweep (up to the
                                window capacity) instead of step n from sweep n */
} biot_schedule;

typedef struct {
  double E, nu, alpha;       /* Young's modulus, Poisson ratio, Biot-Willis constant (Sec. 2.1) */
  double kappa_const;        /* permeability / viscosity K, used when kappa_elem is NULL */
  const double* kappa_elem;  /* host, nullable: per-triangle K, length 2 n^2, triangle 2(j n + i) lower,
                                2(j n + i) + 1 upper of cell (i, j); copied during biot_assemble */
  double tau;                /* time step */
  int32_t n_t;               /* number of time steps N_t (>= 1) */
  int32_t problem;           /* biot_problem */
  int32_t beta_mode;         /* biot_beta_mode */
  double load;               /* Terzaghi top traction magnitude (traction (0, -load) for t >= tau);
                                Barry & Mercer source amplitude 0.5 load */
  int32_t n_iter;            /* Krylov steps per call of K (1..32) */
  int32_t window;            /* BIOT_SCHED_TOL: max active steps (0 = N_t); BIOT_SCHED_PAPER: iterations per step */
  int32_t schedule;          /* biot_schedule */
  int32_t precision;         /* biot_precision */
} biot_params;

typedef struct {
  int32_t n;                 /* cells per side */
  int32_t n_nodes, n_dof;    /* (n+1)^2, 3 (n+1)^2 */
  int64_t nnz;               /* nonzeros of AA's pattern, 9 (7 n^2 + 6 n + 1) */
  int32_t n_pairs;           /* node adjacency pairs P = 7 n^2 + 6 n + 1 */
  int32_t n_t;               /* time steps (0 before biot_assemble) */
  int32_t window_cap;        /* columns of the device Krylov work buffers */
  int32_t band_u, band_p;    /* half-bandwidths of A (u-ordering 2 v + f) and S (node ordering) */
  int32_t precond;           /* biot_precond_kind set up, 0 if none */
  int32_t precision;         /* biot_precision in use */
  double beta;               /* stabilisation factor actually used */
  int64_t device_bytes;      /* device memory held by the context (multigrid levels: their own) */
  int32_t inner;             /* biot_inner_solver of the block solves */
  int32_t gmg_levels;        /* multigrid levels set up (0: exact block solves) */
  double gmg_lam_u, gmg_lam_p;  /* power-method estimates of lam_max(M^{-1} A), lam_max(M^{-1} S) on level 0 */
} biot_info;

typedef enum {
  BIOT_INNER_EXACT = 0,      /* exact block solves: band Cholesky, or substructured (default) */
  BIOT_INNER_GMG = 1         /* geometric multigrid V-cycles (inexact; FGMRES is flexible) */
} biot_inner_solver;

/* ---- context life cycle ------------------------------------------------- */

/* Create a context for the structured n x n right-triangle mesh of [0,Lx]x[0,Ly]
 * (uniform grid with h = Lx/n, each cell split along its "/" diagonal; Sec. 4,
 * "uniform right triangular grid"). Builds the node adjacency and the int32 CSR
 * pattern of AA on the device. cuda_stream: a cudaStream_t (NULL = legacy
 * default stream). Errors: BIOT_E_INVALID (n < 1, n > 4096, Lx or Ly <= 0, out
 * NULL), BIOT_E_OOM, BIOT_E_CUDA. */
biot_status biot_mesh_create(int32_t n, double Lx, double Ly, void* cuda_stream, biot_ctx** out);

/* Assemble AA, A' (Eq. fullysystem) and the right-hand sides f^n for n = 1..N_t
 * (Eq. axb), apply the Dirichlet data, and set x_0 (Sec. 2.1 initial data).
 * Element-parallel coloured assembly on the device (8 colours, no atomics).
 * Allocates the solution store X[N_dof][N_t+1] and the Krylov work buffers for
 * min(N_t, window) columns (window 0 = N_t). May be called again to reassemble.
 * Errors: BIOT_E_INVALID (null params, E <= 0, nu outside (-1, 0.5), tau <= 0,
 * n_t < 1, n_iter outside 1..32, bad enum, kappa <= 0), BIOT_E_OOM, BIOT_E_CUDA. */
biot_status biot_assemble(biot_ctx* ctx, const biot_params* params);

/* Build the preconditioner of Sec. 3.1: extract A (u-block of AA) and
 * S = (tau + beta/K) C (minus the p-block of AA) as band matrices and factor
 * both by band Cholesky on the device, so that the block solves of P1/P2 are
 * exact up to rounding. Errors: BIOT_E_STATE (before biot_assemble),
 * BIOT_E_INVALID (kind), BIOT_E_CUDA (including a non-positive pivot). */
biot_status biot_precond_setup(biot_ctx* ctx, int32_t kind);

/* Exact block solves by one-level substructuring (an implementation choice; the
 * paper leaves the inner solvers of Sec. 3.1 open). strips = 0: automatic (about 18
 * node columns per strip in FP64 and 10 in the reduced-precision modes, at most
 * sqrt((n + 1) / 1.31) and sqrt((n + 1) / 0.38) strips; none below n = 26 and 13
 * respectively); 1: plain band factorisations of A and S in natural order; k >= 2: the
 * n + 1 node columns are cut by k - 1 separator columns into k strips, each strip's
 * interior is factored along its short side (half-band d (w + 2) - 1 for a strip w nodes
 * wide, d = 2 for A, 1 for S), and the separators' Schur complement
 * A_SS - A_SI A_II^{-1} A_IS (block tridiagonal with d (n + 1) x d (n + 1) blocks) is
 * formed and factored on the device; its solves run as dense block products with the
 * inverted diagonal blocks of the factor (or as band substitutions, whichever biot_tune
 * finds faster). The solves stay exact (block Gaussian elimination); only their cost and
 * rounding order change. Above n = 512 a substructured context builds no natural-order
 * factors (and cannot join biot_batch_solve). Takes effect at the next
 * biot_precond_setup. Errors: BIOT_E_INVALID (strips < 0, or fewer than two node columns
 * per strip: 3 strips > n + 2). */
biot_status biot_set_substructure(biot_ctx* ctx, int32_t strips);

/* Choose how the block solves with A and S of P1/P2 are done (Sec. 3.1 leaves it
 * open); takes effect at the next biot_precond_setup. BIOT_INNER_EXACT (default):
 * band Cholesky / substructured factorisations, exact up to rounding.
 * BIOT_INNER_GMG: `cycles` geometric-multigrid V-cycles per block solve on the
 * nested meshes n, n/2, n/4, ... (Sec. 4 builds its meshes by joining edge
 * midpoints; levels 0 = coarsen while n is even and above 16, else up to
 * `levels` levels while n is even and the coarse mesh keeps two cells), with `smooth` Chebyshev steps before and after each coarse
 * correction (node-block Jacobi, interval [lam/8, 1.1 lam] from 20 power steps),
 * restriction P^T, linear prolongation, coarse operators assembled on the coarse
 * meshes with the element permeability averaged over the four children and the
 * fine beta (the Galerkin operators for P1 on nested meshes), and an exact band
 * solve on the coarsest level. P^{-1} is then inexact; the flexible Krylov cycle
 * still converges to the same solution. Errors: BIOT_E_INVALID (kind; levels 1 or
 * negative, cycles outside 1..16, smooth outside 1..8; a mesh that cannot be
 * coarsened: n odd, or n <= 16 with levels 0). */
biot_status biot_set_inner_solver(biot_ctx* ctx, int32_t kind, int32_t levels, int32_t cycles, int32_t smooth);

/* Run the inverted time stepping (Alg. 3) as windowed snapshot sweeps: at sweep
 * w every active step n uses x_{n-1} and x_n from the state after sweep w-1;
 * step n becomes active at sweep n, which reproduces Alg. 3's iterates
 * X^{n,m}, m = w - n + 1. Tol schedule: the oldest active step retires once its
 * predecessor is retired and |D^{-1/2} r_n| <= tol |D^{-1/2} b_n| (D = |diag AA|);
 * paper schedule: every step gets `window` outer iterations, tol is ignored;
 * eager schedule: the tol schedule with every step (up to the window capacity)
 * active from the first sweep. With precision BIOT_FP32/BF16, the sweep runs in reduced precision as the
 * correction solver of an FP64 iterative refinement on the space-time system.
 * Outputs (nullable): sweeps_done, final_rel_res = relative equilibrated
 * space-time residual |D^{-1/2}(F - calA X)| / |D^{-1/2} F| in FP64.
 * Returns BIOT_E_NOT_CONVERGED after max_outer sweeps without convergence
 * (state readable), BIOT_E_DIVERGED, BIOT_E_STATE (no preconditioner). */
biot_status biot_pint_solve(biot_ctx* ctx, double tol, int32_t max_outer,
                            int32_t* sweeps_done, double* final_rel_res);

/* Change the schedule of later biot_pint_solve calls (biot_schedule) without
 * reassembling, e.g. to continue from a state set by biot_set_state with the
 * eager start. BIOT_SCHED_PAPER keeps the `window` given at assembly as its
 * iterations per step. Errors: BIOT_E_STATE (before biot_assemble),
 * BIOT_E_INVALID (unknown schedule, paper window above the capacity). */
biot_status biot_set_schedule(biot_ctx* ctx, int32_t schedule);

/* Solve `count` independent instances together (batched form of biot_pint_solve).
 * Each context is created, assembled (precision BIOT_FP32 or
 * BIOT_BF16VAL_FP32ACC, window 0 = N_t; all with the same precision and n_iter)
 * and set up (same preconditioner kind) on its own; meshes, material, K field
 * and N_t may differ. Every sweep kernel processes all instances in one launch
 * (device table of per-instance buffers and windows); with use_graph != 0 the
 * FGMRES cycle of a sweep is captured once in a CUDA graph and replayed. Block
 * solves: every context's plain band factors (batched band solves), or, when
 * every context was set up with multigrid block solves (biot_set_inner_solver,
 * the same smoothing steps, one cycle), every instance's V-cycles in the same
 * launches: their levels (of any depth) and coarsest band solves are read from
 * device tables. The FP64 refinement and its tolerance are per instance, as in
 * biot_pint_solve; an instance set to the eager schedule starts eagerly.
 * Work runs on a private stream; the contexts' streams are synchronised first.
 * sweeps_done[count] and final_rel_res[count] (host, nullable) receive each
 * instance's FP32 sweeps and final relative space-time residual. Returns the
 * first failing instance's status (BIOT_E_NOT_CONVERGED, BIOT_E_DIVERGED). */
biot_status biot_batch_solve(biot_ctx* const* ctxs, int32_t count, double tol, int32_t max_outer,
                             int32_t use_graph, int32_t* sweeps_done, double* final_rel_res);

/* One outer iteration (sweep) over the window of steps lo..hi (1 <= lo <= hi <= N_t,
 * hi - lo + 1 <= window_cap): residuals from the current state, one cycle of
 * K = right-preconditioned FGMRES(n_iter) per step, state updated in place.
 * rel_out (host, nullable, length hi - lo + 1) receives the relative residual
 * of each step before the update. This is the unit of work the paper's threads
 * perform in one wave of Alg. 4 (one b^{n_t} + one call of K). */
biot_status biot_sweep(biot_ctx* ctx, int32_t lo, int32_t hi, double* rel_out);

/* Relative equilibrated residuals of steps lo..hi for the current state (no update). */
biot_status biot_residual_norms(biot_ctx* ctx, int32_t lo, int32_t hi, double* rel_out);

/* ---- data exchange ------------------------------------------------------ */

/* Copy x_step (0 <= step <= N_t; step 0 is x_0) to host_out[N_dof]. */
biot_status biot_get_solution(const biot_ctx* ctx, int32_t step, double* host_out);

/* Copy steps lo..hi of the solution store to/from host[(hi-lo+1)][N_dof]
 * (step-major). For end-to-end runs and checkpoint/resume. */
biot_status biot_get_state(const biot_ctx* ctx, int32_t lo, int32_t hi, double* host);
biot_status biot_set_state(biot_ctx* ctx, int32_t lo, int32_t hi, const double* host);

/* Copy the CSR of AA (rowptr[N_dof+1], col[nnz] int32, val[nnz] FP64) and the
 * pressure-pressure entries of A' (ap_pp[P], node-pair order) to the host. Any
 * output may be NULL. nnz_out receives the number of nonzeros. */
biot_status biot_get_csr(const biot_ctx* ctx, int32_t* rowptr, int32_t* col, double* val,
                         double* ap_pp, int64_t* nnz_out);

/* Copy the right-hand sides f^n, n = 0..N_t, to host[(N_t+1)][N_dof] (row 0 is zero). */
biot_status biot_get_rhs(const biot_ctx* ctx, double* host);

/* Compute the window residuals r_n = f^n + A' x_{n-1} - AA x_n, n = lo..hi, of
 * the current state in the context's precision and copy them to
 * host[(hi-lo+1)][N_dof] (step-major). */
biot_status biot_get_residual(biot_ctx* ctx, int32_t lo, int32_t hi, double* host);

/* Apply P^{-1} (the preconditioner set up) to ncols host vectors
 * host_in[ncols][N_dof] -> host_out[ncols][N_dof] on the device (ncols <= window_cap). */
biot_status biot_precond_apply(biot_ctx* ctx, int32_t ncols, const double* host_in, double* host_out);

biot_status biot_get_info(const biot_ctx* ctx, biot_info* out);

/* ---- measurement -------------------------------------------------------- */

/* Kernel classes timed by biot_timing_read. */
typedef enum {
  BIOT_KC_RESIDUAL = 0,      /* fused window residual f^n + A' x_{n-1} - AA x_n */
  BIOT_KC_SPMM = 1,          /* equilibrated AA z of the Arnoldi step */
  BIOT_KC_BAND_SOLVE = 2,    /* band triangular solves of the P1/P2 block solves */
  BIOT_KC_COUNT = 3
} biot_kernel_class;

/* enable != 0: clear previous records and bracket every later launch of the
 * classes above with CUDA events on the context's stream; enable == 0: stop. */
biot_status biot_timing_enable(biot_ctx* ctx, int32_t enable);

/* Sum of the event-measured durations (ms) and number of launches recorded for
 * one kernel class since biot_timing_enable. Synchronises the stream. */
biot_status biot_timing_read(biot_ctx* ctx, int32_t kernel_class, double* total_ms, int64_t* launches);

/* ---- allocation-free variant (the paper has no counterpart) ------------- */

/* Largest window (columns) biot_residual_norms_noalloc accepts. */
#define BIOT_NOALLOC_MAX_COLS 512

/* Window residual norms for callers that cannot allocate device memory.
 *
 * Applications that give all of a GPU's memory to their own pool or arena
 * (a framework's caching allocator, a service with a fixed memory budget) do
 * not let libraries call cudaMalloc or cudaFree: those calls synchronise the
 * device, bypass the pool's accounting and fragment it. This entry point
 * computes exactly what biot_residual_norms computes, without allocating:
 *
 *   R[3v+f][c] = d[3v+f] * (f^n + A' x_{n-1} - AA x_n)[3v+f],  n = lo + c,
 *   rel[c]     = |R[:, c]| / |d .* (f^n + A' x_{n-1})|,          c < ncols,
 *
 * with d = |diag AA|^{-1/2}. All pointers are device memory owned by the
 * caller: the node adjacency (nodeptr[n_nodes+1], nbr[P]: node v's sorted
 * neighbours incl. itself), the CSR of AA (rowptr, values in CSR order, as
 * biot_get_csr returns them), the pressure-pressure entries of A' in
 * node-pair order (ap_pp[P]), dscale[N_dof] = d, the state X and right-hand
 * sides F ([N_dof][ldx], time fastest), and the outputs R ([N_dof][ldr]) and
 * rel[ncols]. Work is ordered on cuda_stream; nothing is synchronised.
 *
 * Scratch: per-block partial sums live in one fixed file-scope device array
 * of 2 x 304 x BIOT_NOALLOC_MAX_COLS doubles (2.5 MB), which every GPU that
 * loads the library holds until the process exits. Every call overwrites the
 * partials it reads, so nothing needs clearing, but all calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. The first call on a device looks up the
 * array's device address and should therefore be made before any stream
 * capture; later calls on a stream that is not capturing look it up again
 * (no allocation), so the entry point keeps working after cudaDeviceReset,
 * while a call on a capturing stream uses the address found by the last
 * earlier call on that device.
 *
 * Errors: BIOT_E_INVALID for a NULL buffer, n_nodes < 1, ncols outside
 * 1..BIOT_NOALLOC_MAX_COLS, lo < 1, ldx < lo + ncols or ldr < ncols;
 * BIOT_E_CUDA for a CUDA error. Messages: biot_last_error(NULL). */
biot_status biot_residual_norms_noalloc(int32_t n_nodes, const int32_t* nodeptr, const int32_t* nbr,
                                        const int32_t* rowptr, const double* val, const double* ap_pp,
                                        const double* dscale, const double* X, const double* F, int32_t ldx,
                                        int32_t lo, int32_t ncols, double* R, int32_t ldr, double* rel,
                                        void* cuda_stream);

/* ---- autotuning ---------------------------------------------------------- */

typedef struct {
  int32_t variant_u, variant_p;         /* chosen band-solve variant for A and for S */
  int32_t tma_u, nb_u, threads_u;       /* its shape: TMA-staged?, rows per block, CTA size */
  int32_t tma_p, nb_p, threads_p;
  double ms_u, ms_p;                    /* forward + backward solve pair, chosen variant */
  double ms_u_default, ms_p_default;    /* same with the default variant */
  int32_t from_cache;                   /* 1 if both choices came from the cache file */
  int32_t strips;                       /* substructured block solves: strips (0: plain band) */
  int32_t variant_sep_u, variant_sep_p; /* substructured: separator variants (variant_*: interiors) */
  double ms_sep_u, ms_sep_p;            /* substructured: the separator pair's part of ms_u, ms_p */
  int32_t spmm_variant;                 /* reduced precision: SpMM shape 0-8 (0: 16-byte vectors, unroll 4,
                                           2 CTAs per SM, 2 x 152 CTAs; 1-5 vary them; 6-7 deal the
                                           nodes out to the grid's warps in turns) */
  double ms_spmm, ms_spmm_default;      /* one SpMM at full window: chosen shape, default shape */
} biot_tuning;

/* Pick the band triangular-solve kernel variant (register-streamed; TMA-staged
 * band rows with 8/16/32-row blocks and 128/256 threads; in FP32 also skewed
 * 32-row block tiles with as many bulk-copy stages as fit; those whose shared
 * memory fits)
 * for A and for S by timing a forward + backward solve pair of each candidate on
 * this context's factors at full window width, in the context's precision.
 * cache_path (nullable): JSON file of earlier choices keyed by precision, block
 * size, half-band and window; read first, rewritten with the new choices.
 * Requires biot_precond_setup. out (nullable) receives the choices and times.
 * With substructured block solves (biot_set_substructure) it times, for A and
 * for S, every fitting in-place variant (TMA-staged split rows with 4 to 32-row blocks,
 * or one row per lane with 1, 2 or 4 warps per CTA) of the strip-parallel interior
 * solves and of the separator solves instead, for the separators also the dense
 * block products (variant 100), keeps the fastest, caches the choices under keys
 * "sub:" + precision, rows, half-band and window, and reports the interior variants,
 * the separator variants, the interior + separator pair times (ms_u, ms_p), their
 * separator parts (ms_sep_u, ms_sep_p) and the strip count. In the reduced-precision
 * modes it also times the SpMM w = D^{-1/2} AA z in each of its shapes (16- or 8-byte
 * vectors per lane, i.e. 4 or 2 columns; neighbour-loop unrolling 1, 2 or 4; registers
 * for 2 to 4 CTAs per SM; grids of 2 to 4 x 152 CTAs) at full window width and keeps
 * the fastest (cache key "spmm:" + precision, rows and window); with multigrid block
 * solves only the SpMM is tuned. */
biot_status biot_tune(biot_ctx* ctx, const char* cache_path, biot_tuning* out);

/* Failure-detection test hook. Every bulk copy of band rows into shared memory is
 * awaited with a bounded spin (clock64 budget, about 2 s by default); when the
 * first wait of a block runs out, the kernel records the failure in the
 * context's device status, lets every copy still in flight land (those drain
 * waits keep the full budget) and returns, and biot_pint_solve then returns
 * BIOT_E_TIMEOUT with the context still usable. This call sets the budget of
 * that first wait on the current device to `cycles` SM clock cycles (a few
 * cycles make it run out on purpose); cycles <= 0 restores the default.
 * Synchronous; affects every context on the device. Errors: BIOT_E_CUDA. */
biot_status biot_debug_set_wait_budget(int64_t cycles);

/* Kernel launches issued by this library since it was loaded (all contexts). */
int64_t biot_launch_count(void);

/* One-line description of the last error on ctx (or of the last failed
 * biot_mesh_create when ctx is NULL). Never NULL. */
const char* biot_last_error(const biot_ctx* ctx);

void biot_destroy(biot_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BIOT_PINT_H */
