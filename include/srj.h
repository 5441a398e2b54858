/*
 * srj.h -- C ABI of libsrj.so: a GB300 (sm_103a) solver for the linear
 * system A u = f on structured grids by Scheduled Relaxation Jacobi (SRJ)
 * with the data-driven per-cycle scheme selection of Islam & Wang,
 * "A data driven heuristic for rapid convergence of Scheduled Relaxation
 * Jacobi schemes" (arXiv:2011.06636).
 *
 * The operator (Sec. 3 1D matrix, Sec. 4.2 2D/3D finite differences,
 * generalised with per-axis and per-cell coefficients):
 *
 *   (A u)_p = sum_a sum_{s=-1,+1} eps_a * kf(p, p + s e_a) / h_a^2
 *                                     * (u_p - u_{p + s e_a})
 *
 * on dim = 1, 2 or 3 axes with zero Dirichlet values outside the interior.
 * kf = 1 for constant coefficients, else the harmonic mean
 * 2 k_p k_q / (k_p + k_q) of the cell coefficients on both sides of a face.
 *
 * One SRJ cycle at scheme level L applies the M = M(L) relaxation factors of
 * App. B / Sec. 2 Eq. (srj-relaxation-parameters) as weighted Jacobi sweeps
 * u <- u + omega D^-1 (f - A u) (Sec. 2, Eq. relaxed-jacobi), then takes the
 * L2 residual norm ||f - A u|| and picks the next level by Sec. 3, Alg. 1.
 *
 * Conventions for every entry point:
 *  - Arrays are dense, interior points only, x fastest:
 *    index = x + n0 * (y + n1 * z).
 *  - Pointers documented as DEVICE must be CUDA device (or managed) memory
 *    of the current device; HOST pointers are ordinary host memory.
 *  - The caller owns every array it passes; the library never frees them and
 *    keeps no reference to f, u or k after the call returns.  The library
 *    owns its workspace (internal padded copies, scheme tables, reduction
 *    scratch, per-cycle trace, CUDA graphs), released by srj_destroy.
 *  - Errors are returned as srj_status codes; no entry point throws, traps
 *    or aborts.  srj_last_error() gives a text for the last failure on a
 *    handle.  A handle is not thread safe; distinct handles are independent.
 *  - Work is queued on the stream given at creation (NULL = legacy default
 *    stream).  srj_solve*, srj_run_levels, srj_residual_norm synchronise
 *    that stream before returning (they return host-side results).
 */
#ifndef SRJ_H
#define SRJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srj_handle srj_handle;

typedef enum srj_status {
    SRJ_OK = 0,
    SRJ_EINVAL = 1,       /* invalid argument (null pointer, size, option) */
    SRJ_ENOMEM = 2,       /* device or host allocation failed */
    SRJ_ECUDA = 3,        /* a CUDA runtime call failed (see srj_last_error) */
    SRJ_ENOTCONV = 4,     /* sweep cap reached before the tolerance */
    SRJ_EDIVERGED = 5,    /* the residual norm became non-finite */
    SRJ_ETIMEOUT = 6,     /* a bounded device-side wait expired (srj_set_wait_limit) */
    SRJ_EUNSUPPORTED = 7  /* valid request the library does not implement */
} srj_status;

/* Per-cycle level selection. */
enum srj_selector {
    SRJ_SEL_HEURISTIC = 0,  /* Sec. 3, Alg. 1: ratio > 0.4 up, 0.2 < ratio < 0.4 down */
    SRJ_SEL_INCREASING = 1, /* Sec. 4: raise the level every cycle */
    SRJ_SEL_FIXED = 2,      /* stay at opts.fixed_level */
    SRJ_SEL_MLP = 3,        /* learned selector (srj_mlp_set_weights) with Alg. 1 as judge:
                               after a picked cycle that did not shrink the residual, or
                               shrank it more slowly per sweep (Sec. 3, Eq.
                               average-convergence-rate) than the latest cycle Alg. 1
                               chose, Alg. 1 takes the next decision */
    SRJ_SEL_JACOBI = 4      /* plain Jacobi, Sec. 2 Eq. (jacobi): omega = 1 every sweep, the
                               comparator of Sec. 4 and Table 3; the residual is tested
                               after every M(fixed_level) sweeps (a "cycle"; level 0:
                               every sweep).  Single-grid handles only. */
};

/* Arithmetic of the sweeps; f and u element types follow it. */
enum srj_precision {
    SRJ_PREC_F64 = 0,   /* FP64 sweeps; f, u are double */
    SRJ_PREC_F32 = 1,   /* FP32 sweeps; f, u are float (roundoff floor ~ kappa*eps32) */
    SRJ_PREC_MIXED = 2  /* FP64 iterative refinement (r = f - A u, u += e in FP64)
                           around FP32-arithmetic inner SRJ on A e = r whose iterate
                           is kept as an unevaluated pair of FP32 values; f, u double */
};

enum srj_tol_kind {
    SRJ_TOL_REL = 0,  /* ||f - A u|| / ||f - A u0|| < tol (Sec. 4.2.3, Eq. relative-residual) */
    SRJ_TOL_ABS = 1,  /* ||f - A u|| < tol (Sec. 4.1) */
    SRJ_TOL_DINF = 2  /* ||u^n - u^(n-1)||_inf < tol, the largest change of one sweep
                         (Sec. 4.2.2, Eq. relative_residual_solution).  Tested after
                         every sweep, so a solve can end inside a cycle; Alg. 1 still
                         reads the L2 residual ratio at each cycle end.  SRJ_PREC_F64
                         and SRJ_PREC_F32 single-problem handles only. */
};

/* Boundary condition of one grid axis (both ends). */
enum srj_bc {
    SRJ_BC_DIRICHLET = 0, /* u = 0 one step outside the n points (Sec. 2, Sec. 4.2.3) */
    SRJ_BC_NEUMANN = 1    /* du/dn = 0 by a mirrored ghost node (Sec. 4.2.2): the n points
                             include both boundary nodes (n >= 2) and the node one step
                             outside takes the value of the node one step inside, so the
                             central difference of du/dx at the boundary vanishes.
                             Constant coefficients, SRJ_PREC_F64 / SRJ_PREC_F32
                             single-problem handles only.  With every axis Neumann, A is
                             singular (constant vectors span its null space) and A u = f
                             needs sum(f) = 0, e.g. the paper's Laplace problem f = 0. */
};

typedef struct srj_grid {
    int32_t dim;   /* 1, 2 or 3 */
    int64_t n[3];  /* points per axis, x first; axes >= dim ignored */
    double h[3];   /* grid spacing per axis; 0 means the unit domain: 1/(n+1) on a
                      Dirichlet axis, 1/(n-1) on a Neumann axis */
    int32_t bc[3]; /* enum srj_bc per axis; zero-initialised = Dirichlet everywhere */
} srj_grid;

typedef struct srj_stencil {
    double eps[3];   /* axis coefficients; 0 means 1 (Poisson) */
    const double *k; /* NULL: constant coefficients.  Else a DEVICE array of the
                        cell coefficient including one ghost layer per axis:
                        (n0+2)(n1+2)(n2+2) doubles (axes >= dim count 1), x
                        fastest, all entries finite and > 0.  Read only during
                        srj_create (face coefficients are derived there). */
    const double *a_diag;   /* NULL, or an explicit symmetric operator replacing the
                               PDE stencil (Sec. 4.1: random symmetric diagonally
                               dominant tridiagonal systems; any dimension):
                               DEVICE array of the n0*n1*n2 diagonal entries A_pp,
                               x fastest, all finite and nonzero.  h, eps and k
                               are then unused (k must be NULL); Dirichlet axes
                               only.  Read only during srj_create. */
    const double *a_off[3]; /* with a_diag: DEVICE arrays (grid size, x fastest) of
                               the couplings A_(p,p+e_a) = A_(p+e_a,p) along each
                               axis a < dim; the entry of a point whose +e_a
                               neighbour lies outside the grid is not read. */
} srj_stencil;

typedef struct srj_opts {
    int32_t selector;       /* enum srj_selector */
    int32_t precision;      /* enum srj_precision */
    int32_t tol_kind;       /* enum srj_tol_kind */
    int32_t level0;         /* level of the first cycle (Sec. 3 uses 0) */
    int32_t fixed_level;    /* level for SRJ_SEL_FIXED */
    int32_t max_level;      /* highest selectable level, <= 24 (0 means 24) */
    int32_t temporal_depth; /* sweeps fused per HBM pass; 0 = library choice.
                               2D constant coefficients: 1 or 2 (F64), 4 or 8
                               (F32), 2 or 4 (MIXED); 3D Dirichlet: 1 or 2
                               (default 2 for MIXED, 1 otherwise; the 3D
                               iterates are the same bit for bit at 1 and 2) */
    int32_t trace_capacity; /* per-cycle records kept (0 means 4096) */
    int64_t max_sweeps;     /* sweep cap per solve (0 means 1000000) */
    double inner_tol;       /* SRJ_PREC_MIXED: floor of the inner solves' relative
                               tolerance; each inner solve aims at the reduction
                               still needed, but not below this (0 means 1e-6) */
} srj_opts;

typedef struct srj_stats {
    int32_t status;      /* srj_status of the solve */
    int32_t final_level; /* level of the last cycle run */
    int64_t sweeps;      /* relaxed Jacobi sweeps = the paper's iterations */
    int64_t cycles;      /* SRJ cycles (for MIXED: summed over inner solves) */
    int64_t outer;       /* MIXED: refinement steps; otherwise 0 */
    int64_t passes;      /* kernel passes over the grid */
    double r0;           /* ||f - A u0||_2 */
    double rn;           /* ||f - A u||_2 at exit (FP64 for F64 and MIXED) */
    double seconds;      /* device time of the solve, CUDA events */
    double inner_seconds; /* device time of the cycle loop alone (the sweep
                             passes with their fused norms and selection;
                             for MIXED summed over the inner solves, without
                             the FP64 outer kernels), CUDA events */
} srj_stats;

/* Library version string (static storage). */
const char *srj_version(void);

/* App. B: number of relaxation factors M of a scheme level, or -1 if the
 * level is outside [0, 24]. */
int32_t srj_level_m(int32_t level);

/* Sec. 2, Eq. (srj-relaxation-parameters): writes the M(level) relaxation
 * factors of a level into the HOST array omega_out (capacity entries), in the
 * order the library applies them within a cycle (Leja order of the Chebyshev
 * roots, largest factor first).  Returns M, or -1 for a bad level or a too
 * small capacity. */
int32_t srj_scheme_omegas(int32_t level, double *omega_out, int32_t capacity);

/* Create a solver for one grid.  grid, stencil and opts are HOST structs
 * (stencil may be NULL: Poisson; opts may be NULL: defaults).  stream is a
 * cudaStream_t (NULL = legacy default stream).  Allocates the device
 * workspace (about 3-6 arrays of the grid size) and the scheme tables on the
 * current device.  On failure *out is NULL and the status says why: a Neumann
 * axis or SRJ_TOL_DINF together with SRJ_PREC_MIXED, variable coefficients or
 * an explicit operator gives SRJ_EUNSUPPORTED; a Neumann axis with fewer than
 * 2 points, or both k and a_diag, SRJ_EINVAL. */
srj_status srj_create(const srj_grid *grid, const srj_stencil *stencil,
                      const srj_opts *opts, void *stream, srj_handle **out);

/* Solve A u = f to tol (kind from opts).  f and u are DEVICE arrays of the
 * grid size with the element type of the precision (double for F64 and
 * MIXED, float for F32); u holds u0 on entry and the result on exit.
 * stats (HOST, may be NULL) receives the counters.  Returns SRJ_OK when
 * converged, SRJ_ENOTCONV / SRJ_EDIVERGED otherwise (u then holds the last
 * iterate). */
srj_status srj_solve(srj_handle *h, const void *f, void *u, double tol,
                     srj_stats *stats);

/* As srj_solve, but f and u are HOST arrays: the host-to-device copies of f
 * and u0 and the device-to-host copy of u are part of the call (and of
 * stats->seconds).  Pinned host memory gives the fastest copies. */
srj_status srj_solve_host(srj_handle *h, const void *f_host, void *u_host,
                          double tol, srj_stats *stats);

/* Run an explicit list of ncycles levels (HOST array) without selection and
 * without a convergence test: for each entry one whole cycle of M(level)
 * sweeps.  f, u as for srj_solve.  rn_out (HOST, ncycles doubles, may be
 * NULL) receives ||f - A u|| after each cycle.  Precision F64 or F32 only. */
srj_status srj_run_levels(srj_handle *h, const void *f, void *u,
                          const int32_t *levels, int64_t ncycles,
                          double *rn_out);

/* ||f - A u||_2 of DEVICE arrays f, u (types as for srj_solve), into *out. */
srj_status srj_residual_norm(srj_handle *h, const void *f, const void *u,
                             double *out);

/* Copy the per-cycle record of the last solve (level and ||f - A u|| after
 * each cycle; for MIXED the inner cycles, rn relative to that inner solve's
 * right-hand side) into HOST arrays of the given capacity.  Returns the
 * number of cycles of the last solve (may exceed capacity) or -1. */
int64_t srj_get_trace(const srj_handle *h, int32_t *levels, double *rn,
                      int64_t capacity);

/* Batched solver: nprob independent 2D constant-coefficient problems of any
 * sizes (grids[i], stencils[i] with k == NULL; stencils may be NULL), solved
 * together in mixed precision (opts->precision must be SRJ_PREC_MIXED): one
 * persistent kernel advances every unfinished problem by one step of its own
 * solve (FP64 residual, inner SRJ pass, FP64 update) per launch, inside one
 * CUDA graph.  grids, stencils: HOST arrays of nprob structs; opts shared by
 * all problems.  The temporal depth (opts->temporal_depth == 0) and the
 * segment height of the persistent kernel are chosen by timing candidates on
 * the first solve (cached in the file named by the environment variable
 * SRJ_AUTOTUNE_CACHE when set).  Workspace: about 20 bytes per grid point
 * plus per-item scratch.  Returns SRJ_EUNSUPPORTED for 1D/3D grids or
 * variable coefficients. */
srj_status srj_create_batched(int32_t nprob, const srj_grid *grids,
                              const srj_stencil *stencils, const srj_opts *opts,
                              void *stream, srj_handle **out);

/* Solve every problem of a batched handle to tol (kind from opts).  f and u
 * are HOST arrays of nprob DEVICE pointers to dense FP64 arrays (f[i], u[i]
 * sized like grids[i]); u[i] holds u0 on entry and the solution on exit.
 * stats: HOST array of nprob srj_stats (may be NULL); stats[i].seconds is the
 * device time of the whole batch.  Returns SRJ_OK if every problem converged,
 * else the first non-OK status. */
srj_status srj_solve_batched(srj_handle *h, const double *const *f, double *const *u,
                             double tol, srj_stats *stats);

/* Learned scheme selector (SRJ_SEL_MLP; not in the paper, which selects
 * with Alg. 1).  A network 12 -> 64 -> 64 -> 25 (ReLU) maps the solver state
 * -- log of the last 8 residual ratios, log10 of the grid size, dimension and
 * the current level -- to the level of the next cycle; Alg. 1 takes over for
 * the next decision whenever a picked cycle did not shrink the residual.
 * Parameters: 6617 values W1 (64x12), b1, W2 (64x64), b2, W3 (25x64), b3,
 * row-major, as BF16 bit patterns.
 *
 * srj_mlp_set_weights: copy the BF16 weights (HOST array of count == 6617)
 * into h (single-grid or batched); required before a solve with SRJ_SEL_MLP. */
srj_status srj_mlp_set_weights(srj_handle *h, const uint16_t *w, int64_t count);

/* Evaluate the selector network on the GPU for n feature rows (HOST arrays:
 * w 6617 BF16, x n*12 floats); writes the argmax level of each row into
 * pick_host (n ints) and, if not NULL, the 25 FP32 logits per row into
 * logits_host.  Uses the current device; allocates and frees its scratch. */
srj_status srj_mlp_forward(const uint16_t *w_host, const float *x_host, int64_t n,
                           int32_t *pick_host, float *logits_host);

/* Train the selector on the GPU: `steps` Adam steps (beta 0.9 / 0.999, eps
 * 1e-8, learning rate lr, moments starting at zero) of mean softmax
 * cross-entropy over minibatches of `batch` (<= 64) samples.  DEVICE arrays:
 * x_dev (n x 12 floats), y_dev (n labels in [0, 25)), order_dev (steps*batch
 * sample indices, the minibatch order), theta_dev (6617 FP32 parameters, in:
 * initial, out: trained).  loss_host (HOST, steps floats, may be NULL)
 * receives the minibatch losses.  Runs on `stream` and synchronises it. */
srj_status srj_mlp_train(const float *x_dev, const int32_t *y_dev, int64_t n,
                         const int32_t *order_dev, int64_t steps, int32_t batch, float lr,
                         float *theta_dev, float *loss_host, void *stream);

/* FP64 residual norm ||f - A u||_2 (constant coefficients; f, u DEVICE
 * dense FP64 arrays of the grid; *out on the HOST) computed without
 * allocating any memory, for callers that cannot call cudaMalloc or cudaFree:
 * code running under a device-memory pool or budget it does not own, or on a
 * path where cudaFree's device-wide synchronisation is unacceptable.  The
 * paper has no counterpart.
 *
 * Its reduction scratch is a fixed device array inside the library (one
 * partial sum per grid row plus a counter, about 512 KB, held by every GPU
 * that loads the library until the process exits), so grids with more than
 * 65536 rows (n1 * n2 > 65536) are rejected with SRJ_EINVAL, as are a
 * negative or non-finite spacing h[a] or coefficient eps[a] (0 selects the
 * default, as in srj_create); variable coefficients (stencil->k or a_diag
 * set) and Neumann axes give SRJ_EUNSUPPORTED.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress with the device
 * current) and caches it; make that first call before any stream capture.
 * The cached address does not survive cudaDeviceReset: do not call this
 * function on a device after resetting it.  Every call clears the counter it
 * needs; all calls on a device share the array, so calls whose work overlaps
 * on the GPU (other streams or host threads) race and must be serialised by
 * the caller.  Work is queued on `stream` (NULL = legacy default), and the
 * call synchronises `stream` before it returns the norm in *out. */
srj_status srj_residual_norm_noalloc(const srj_grid *grid, const srj_stencil *stencil,
                                     const double *f, const double *u, double *out,
                                     void *stream);

/* Geometric multigrid with SRJ smoothing -- an adjacent use of the method:
 * Sec. 1 names Jacobi iteration as the usual multigrid smoother and Sec. 5
 * names SRJ schemes as smoothers that accelerate multigrid.  V-cycles of:
 * nu1 SRJ cycles of scheme level smoother_level (its M(level) factors of Sec. 2,
 * Eq. srj-relaxation-parameters, in the library's order) as pre-smoother, the
 * residual, full-weighting restriction to the grid with (n - 1) / 2 points
 * and twice the spacing per axis (operator rediscretised), the coarse
 * correction by recursion down to one point (solved exactly), linear
 * interpolation of the correction, nu2 cycles as post-smoother.  All FP64.
 * Level 0 (M = 1, omega = 2/3) is the classic damped-Jacobi smoother. */
typedef struct srj_mg_opts {
    int32_t smoother_level; /* scheme level of the smoother, 0..24 (default 1) */
    int32_t nu1, nu2;       /* pre- and post-smoothing cycles (0 means 1 each) */
    int32_t max_cycles;     /* V-cycle cap (0 means 100) */
} srj_mg_opts;

/* Create a multigrid solver.  grid: every axis n = 2^k - 1 with the same k
 * (k >= 1), zero Dirichlet (SRJ_EINVAL otherwise); stencil NULL or constant
 * coefficients eps (k or a_diag give SRJ_EUNSUPPORTED).  opts may be NULL.
 * Allocates about 4 arrays of every grid of the hierarchy (4/3 to 8/7 of the
 * fine grid's 4 arrays) on the current device. */
srj_status srj_mg_create(const srj_grid *grid, const srj_stencil *stencil,
                         const srj_mg_opts *opts, void *stream, srj_handle **out);

/* V-cycles on A u = f until ||f - A u|| / ||f - A u0|| < tol.  f, u: DEVICE
 * dense FP64 arrays of the fine grid (u: u0 in, solution out).  stats (HOST,
 * may be NULL): cycles = V-cycles, sweeps = fine-grid relaxed Jacobi sweeps,
 * passes = kernel launches, r0, rn, seconds.  SRJ_ENOTCONV after max_cycles.
 * The handle must come from srj_mg_create (SRJ_EINVAL otherwise). */
srj_status srj_mg_solve(srj_handle *h, const double *f, double *u, double tol,
                        srj_stats *stats);

/* One record of the Sec. 3 data collection (srj_collect_moves). */
typedef struct srj_move_record {
    double prev_ratio; /* state: ||r|| after / before the previous cycle taken */
    double r_before;   /* ||b - A x|| before the tried cycle */
    double r_after;    /* ||b - A x|| after it; the move's average convergence
                          rate (Sec. 3, Eq. average-convergence-rate) is
                          -log(r_after / r_before) / M(level + action) */
    int32_t level;     /* state: the current scheme level */
    int32_t action;    /* the tried move: -1 decrease, 0 keep, +1 increase */
} srj_move_record;

/* Sec. 3, data collection: trials of the procedure the paper derived Alg. 1
 * from, on the 1D Poisson system of Sec. 3 (Eq. poisson: N = n interior
 * points, h = 1/(n+1), zero Dirichlet values), FP64.  A trial starts from
 * x = 0 with one cycle at level 0; at every step it tries each allowed move
 * (decrease, keep, increase the level, inside [0, max_level]) from the
 * current iterate, one cycle each, records them, and takes one at random (the
 * taken cycle's iterate, level and ratio are the next state); it ends once
 * the taken residual norm is below tol (the paper: 1e-8) or after max_steps
 * steps.  The move of step k of trial t is candidate floor(u * ncand) of the
 * allowed moves in the order decrease, keep, increase, where u = (z >> 11) *
 * 2^-53 and z is SplitMix64's output function (Steele, Lea and Flood, 2014)
 * applied to seed + (t * 2^32 + k + 1) * 0x9E3779B97F4A7C15.
 *
 * f: DEVICE array of n values, or NULL for b = 1 (the paper's choice).  Runs
 * trials trial0 .. trial0 + ntrials - 1; trial trial0 + i writes its records
 * to out[i * 3 * max_steps ...] (DEVICE, ntrials * 3 * max_steps records,
 * caller-owned) and their number to counts[i] (DEVICE, ntrials).  n is
 * limited to 4096 (each trial lives in one CTA's shared memory): SRJ_EINVAL
 * beyond, for ntrials < 1, max_steps < 1, a max_level outside [0, 24] or tol
 * not a positive finite number.  Allocates and frees a small factor table,
 * runs on `stream` and synchronises it. */
srj_status srj_collect_moves(int64_t n, const double *f, double tol, int32_t max_level,
                             uint64_t seed, int64_t trial0, int32_t ntrials, int32_t max_steps,
                             srj_move_record *out, int32_t *counts, void *stream);

/* Failure detection (the paper has no counterpart): the 3D pass waits for
 * every plane it stages in shared memory at most `polls` polls of its
 * mbarrier (default 4194304; a negative value restores the default, 0 makes
 * the first wait give up at once).  A wait that runs out ends the solve with
 * SRJ_ETIMEOUT instead of hanging: the pass still waits, with the default
 * limit, for the copies it has in flight, takes part in the pass's
 * bookkeeping and returns; later passes of the solve exit at once.  After
 * SRJ_ETIMEOUT the contents of u are unspecified; the handle stays usable and
 * the next solve starts from a clean state.  A timeout at the default limit
 * means the copies did not complete: check the CUDA context
 * (cudaDeviceSynchronize) and destroy the handle.  Takes effect from the
 * next solve on h.  Other kernels have no device-side waits. */
srj_status srj_set_wait_limit(srj_handle *h, int64_t polls);

/* Text describing the last failure on h (static storage inside h), or a
 * generic text for h == NULL. */
const char *srj_last_error(const srj_handle *h);

/* Release the handle and all library-owned device memory and graphs. */
srj_status srj_destroy(srj_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* SRJ_H */
