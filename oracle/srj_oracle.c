/*
 * srj_oracle.c -- plain, slow, FP64 CPU oracle for Scheduled Relaxation
 * Jacobi (SRJ) with the data-driven scheme-selection heuristic of
 * Islam & Wang, "A data driven heuristic for rapid convergence of Scheduled
 * Relaxation Jacobi schemes" (arXiv:2011.06636).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  It shares no code, header, table or
 * constant generator with the library under paper_2011_06636_gb300/, and
 * nothing in the product path may call it.  Only tests/, the smoke check and
 * the CPU-baseline leg of bench.py load it.
 *
 * Everything is double precision, written for a reader to check against the
 * paper by eye: no blocking, no fusion, no reordering beyond what the
 * equations state.  Each function cites the passage it follows.
 *
 * Readings of points the paper leaves open:
 *  - within-cycle order of the relaxation factors: Leja order of the
 *    Chebyshev roots, starting from the largest root (largest omega);
 *    Sec. 2 only asks for an order that keeps roundoff under control.
 *  - residual ratio = r_after / r_before (Sec. 3, Alg. 1 thresholds < 1).
 *  - ratio exactly 0.4 or 0.2 keeps the level (Alg. 1 uses strict tests).
 *  - the level is clamped to [0, 24] (App. B lists 25 levels).
 *  - the first cycle runs at level 0; a decision follows every cycle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_LEVEL 24

/* App. B (Table "Relationship between M and scheme level"): scheme level ->
 * number M of relaxation factors in one cycle.  Copied from the paper. */
static const int OR_LEVEL_M[OR_MAX_LEVEL + 1] = {
    1, 2, 3, 5, 7, 10, 14, 19, 26, 35, 47, 63, 84,
    111, 147, 194, 256, 338, 446, 589, 778, 1027, 1356, 1790, 2362};

int oracle_level_m(int level)
{
    if (level < 0 || level > OR_MAX_LEVEL) return -1;
    return OR_LEVEL_M[level];
}

/* Sec. 2, Eq. (transformation): lambda* is the argument where the Chebyshev
 * polynomial T_M equals 3.  For x >= 1, T_M(x) = cosh(M acosh x), so
 * lambda* = cosh(acosh(3) / M). */
double oracle_lambda_star(int M)
{
    return cosh(acosh(3.0) / (double)M);
}

/* Sec. 2, Eq. (srj-relaxation-parameters): omega_j = (lambda*+1) /
 * (2 (lambda* - x_j)) with x_j = cos((2j+1) pi / (2M)), j = 0..M-1, the roots
 * of T_M.  Output in root order (j ascending, so omega descending). */
void oracle_scheme_root_order(int M, double *x_out, double *omega_out)
{
    const double ls = oracle_lambda_star(M);
    for (int j = 0; j < M; ++j) {
        const double xj = cos((2.0 * j + 1.0) * M_PI / (2.0 * M));
        if (x_out) x_out[j] = xj;
        omega_out[j] = (ls + 1.0) / (2.0 * (ls - xj));
    }
}

/* Within-cycle order (reading of Sec. 2, last paragraph): Leja order of the
 * roots x_j on [-1, 1].  The first point is x_0 (largest root); each next
 * point is the unused root that maximises the product of its distances to
 * the roots already chosen, evaluated as a sum of logarithms.  Ties go to the
 * smaller index.  order_out receives the root indices in application order. */
void oracle_leja_order(int M, const double *x, int *order_out)
{
    double *score = (double *)malloc(sizeof(double) * (size_t)M);
    char *used = (char *)calloc((size_t)M, 1);
    for (int j = 0; j < M; ++j) score[j] = 0.0;
    int cur = 0;
    for (int step = 0; step < M; ++step) {
        if (step > 0) {
            int best = -1;
            for (int j = 0; j < M; ++j) {
                if (used[j]) continue;
                if (best < 0 || score[j] > score[best]) best = j;
            }
            cur = best;
        }
        order_out[step] = cur;
        used[cur] = 1;
        for (int j = 0; j < M; ++j)
            if (!used[j]) score[j] += log(fabs(x[j] - x[cur]));
    }
    free(score);
    free(used);
}

/* The relaxation factors of one scheme level, in application order. */
int oracle_level_omegas(int level, double *omega_out)
{
    const int M = oracle_level_m(level);
    if (M < 0) return -1;
    double *x = (double *)malloc(sizeof(double) * (size_t)M);
    double *w = (double *)malloc(sizeof(double) * (size_t)M);
    int *ord = (int *)malloc(sizeof(int) * (size_t)M);
    oracle_scheme_root_order(M, x, w);
    oracle_leja_order(M, x, ord);
    for (int i = 0; i < M; ++i) omega_out[i] = w[ord[i]];
    free(x);
    free(w);
    free(ord);
    return M;
}

/* Sec. 2, Eq. (amplification-M-scheme): G_M(lambda) =
 * prod_i [(1 - omega_i) + omega_i lambda]. */
double oracle_amplification(int M, const double *omega, double lambda)
{
    double g = 1.0;
    for (int i = 0; i < M; ++i) g *= (1.0 - omega[i]) + omega[i] * lambda;
    return g;
}

/* ------------------------------------------------------------------------
 * The linear system A u = f on a structured grid.
 *
 * dim in {1,2,3}; n[a] points on axis a (x is axis 0 and varies fastest in
 * memory).  bc[a] = 0: zero Dirichlet values one step outside the n interior
 * points; bc[a] = 1: homogeneous Neumann, the n points are all nodes including
 * both boundary nodes and the ghost node one step outside mirrors the node one
 * step inside (Sec. 4.2.2, second-order central difference with ghost nodes).
 * Operator (Sec. 3, 1D matrix; Sec. 4.2.2/4.2.3 for 2D/3D, extended with an
 * axis coefficient eps[a] and an optional cell coefficient k):
 *
 *   (A u)_p = sum_a sum_{s=-1,+1} eps[a] * kf(p, p+s e_a) / h[a]^2
 *                                * (u_p - u_{p+s e_a})
 *
 * kf = 1 when k is NULL; otherwise kf is the harmonic mean
 * 2 k_p k_q / (k_p + k_q) of the two cells sharing the face.  k is stored with
 * one ghost layer on every axis < dim, i.e. dims (n[a]+2), x fastest.
 * ------------------------------------------------------------------------ */
typedef struct {
    int dim;
    long n[3];
    double h[3];
    double eps[3];
    const double *k; /* NULL or (n0+2)(n1+2)(n2+2) cell values incl. ghosts */
    int bc[3];       /* per axis: 0 zero Dirichlet, 1 homogeneous Neumann by a
                        mirrored ghost node (Sec. 4.2.2): u_{-1} = u_1,
                        u_n = u_{n-2}, the grid points including both ends */
    /* Explicit symmetric operator (Sec. 4.1, random symmetric diagonally
     * dominant tridiagonal systems, extended to 2D/3D five/seven-point
     * patterns): when adiag is not NULL, A_pp = adiag[p] and
     * A_{p,p+e_a} = A_{p+e_a,p} = aoff[a][p]; entries coupling to a point
     * outside the grid are ignored; h, eps, k and bc are not used. */
    const double *adiag;
    const double *aoff[3];
} oracle_problem;

static long or_npts(const oracle_problem *P)
{
    long t = 1;
    for (int a = 0; a < P->dim; ++a) t *= P->n[a];
    return t;
}

static double or_kcell(const oracle_problem *P, const long c[3])
{
    /* c holds interior coordinates, possibly -1 or n[a] (ghost) */
    long kn[3], idx = 0, stride = 1;
    for (int a = 0; a < 3; ++a) kn[a] = (a < P->dim) ? P->n[a] + 2 : 1;
    for (int a = 0; a < 3; ++a) {
        long ca = (a < P->dim) ? c[a] + 1 : 0;
        idx += ca * stride;
        stride *= kn[a];
    }
    return P->k[idx];
}

static double or_face(const oracle_problem *P, const long p[3], int a, int s)
{
    if (!P->k) return 1.0;
    long q[3] = {p[0], p[1], p[2]};
    q[a] += s;
    const double kp = or_kcell(P, p), kq = or_kcell(P, q);
    return 2.0 * kp * kq / (kp + kq);
}

/* Value of u at the neighbour of interior point p (linear index i) one step
 * s = -1 or +1 along axis a.  Outside the grid: zero for a Dirichlet axis;
 * for a Neumann axis the ghost node mirrors the node one step inside, so the
 * central difference of du/dx at the boundary node vanishes (Sec. 4.2.2). */
static double or_neighbour(const oracle_problem *P, const double *u,
                           const long p[3], long i, int a, int s)
{
    long stride = 1;
    for (int b = 0; b < a; ++b) stride *= P->n[b];
    const long qa = p[a] + s;
    if (qa < 0 || qa >= P->n[a]) {
        if (P->bc[a] != 1) return 0.0;
        return u[i - s * stride]; /* mirror: u_{-1} = u_1, u_n = u_{n-2} */
    }
    return u[i + s * stride];
}

/* linear index of point p (x fastest) */
static long or_index(const oracle_problem *P, const long p[3])
{
    return p[0] + P->n[0] * (p[1] + (P->dim > 1 ? P->n[1] : 1) * p[2]);
}

/* diagonal entry D_p of A (Sec. 2, splitting A = D + L + U) */
static double or_diag(const oracle_problem *P, const long p[3])
{
    if (P->adiag) return P->adiag[or_index(P, p)];
    double d = 0.0;
    for (int a = 0; a < P->dim; ++a) {
        const double c = P->eps[a] / (P->h[a] * P->h[a]);
        d += c * (or_face(P, p, a, -1) + or_face(P, p, a, +1));
    }
    return d;
}

/* (A u)_p for the interior point p with linear index i */
static double or_apply_at(const oracle_problem *P, const double *u,
                          const long p[3], long i)
{
    double acc = 0.0;
    if (P->adiag) {
        acc = P->adiag[i] * u[i];
        for (int a = 0; a < P->dim; ++a) {
            long stride = 1;
            for (int b = 0; b < a; ++b) stride *= P->n[b];
            if (p[a] + 1 < P->n[a]) acc += P->aoff[a][i] * u[i + stride];
            if (p[a] > 0) acc += P->aoff[a][i - stride] * u[i - stride];
        }
        return acc;
    }
    for (int a = 0; a < P->dim; ++a) {
        const double c = P->eps[a] / (P->h[a] * P->h[a]);
        for (int s = -1; s <= 1; s += 2)
            acc += c * or_face(P, p, a, s) * (u[i] - or_neighbour(P, u, p, i, a, s));
    }
    return acc;
}

/* Loop bounds: axes beyond dim have a single position. */
static long or_extent(const oracle_problem *P, int a)
{
    return a < P->dim ? P->n[a] : 1;
}

void oracle_apply_A(const oracle_problem *P, const double *u, double *Au)
{
    long i = 0;
    for (long z = 0; z < or_extent(P, 2); ++z)
        for (long y = 0; y < or_extent(P, 1); ++y)
            for (long x = 0; x < or_extent(P, 0); ++x, ++i) {
                const long p[3] = {x, y, z};
                Au[i] = or_apply_at(P, u, p, i);
            }
}

void oracle_diagonal(const oracle_problem *P, double *D)
{
    long i = 0;
    for (long z = 0; z < or_extent(P, 2); ++z)
        for (long y = 0; y < or_extent(P, 1); ++y)
            for (long x = 0; x < or_extent(P, 0); ++x, ++i) {
                const long p[3] = {x, y, z};
                D[i] = or_diag(P, p);
            }
}

/* ||f - A u||_2 : the L2 residual norm of Sec. 3 and Eq. (relative-residual) */
double oracle_residual_norm(const oracle_problem *P, const double *u, const double *f)
{
    double sum = 0.0;
    long i = 0;
    for (long z = 0; z < or_extent(P, 2); ++z)
        for (long y = 0; y < or_extent(P, 1); ++y)
            for (long x = 0; x < or_extent(P, 0); ++x, ++i) {
                const long p[3] = {x, y, z};
                const double r = f[i] - or_apply_at(P, u, p, i);
                sum += r * r;
            }
    return sqrt(sum);
}

/* One weighted Jacobi sweep, Sec. 2, Eq. (relaxed-jacobi):
 *   x' = omega [B_J x + D^-1 b] + (1 - omega) x,  B_J = -D^-1 (L + U),
 * which is x' = x + omega D^-1 (b - A x).  Out of place. */
void oracle_sweep(const oracle_problem *P, const double *u_in, const double *f,
                  double omega, double *u_out)
{
    const long nx = or_extent(P, 0), ny = or_extent(P, 1), nz = or_extent(P, 2);
    /* Every point is independent (out of place), so the rows may run on
     * several host threads; the pragma only acts in the OpenMP build used to
     * time the CPU baseline and changes no result. */
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y) {
            long i = (z * ny + y) * nx;
            for (long x = 0; x < nx; ++x, ++i) {
                const long p[3] = {x, y, z};
                const double r = f[i] - or_apply_at(P, u_in, p, i);
                u_out[i] = u_in[i] + omega * r / or_diag(P, p);
            }
        }
}

/* Apply a list of relaxation factors in order (a partial or whole cycle). */
void oracle_sweeps(const oracle_problem *P, double *u, const double *f,
                   const double *omega, long count)
{
    const long N = or_npts(P);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N);
    for (long s = 0; s < count; ++s) {
        oracle_sweep(P, u, f, omega[s], tmp);
        memcpy(u, tmp, sizeof(double) * (size_t)N);
    }
    free(tmp);
}

/* As oracle_sweeps, but after every sweep takes ||x^n - x^{n-1}||_inf
 * (Sec. 4.2.2, Eq. relative_residual_solution) and stops after the first
 * sweep where it falls below dtol.  Returns the number of sweeps done. */
long oracle_sweeps_dinf(const oracle_problem *P, double *u, const double *f,
                        const double *omega, long count, double dtol, int *reached)
{
    const long N = or_npts(P);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N);
    long s = 0;
    *reached = 0;
    while (s < count) {
        oracle_sweep(P, u, f, omega[s], tmp);
        double dmax = 0.0;
        for (long i = 0; i < N; ++i) {
            const double d = fabs(tmp[i] - u[i]);
            if (!(d <= dmax)) dmax = d; /* a NaN change is kept: never below dtol */
        }
        memcpy(u, tmp, sizeof(double) * (size_t)N);
        s += 1;
        if (dmax < dtol) {
            *reached = 1;
            break;
        }
    }
    free(tmp);
    return s;
}

/* Sec. 3, Alg. 1 (the data-driven heuristic), with the readings listed at the
 * top of this file.  rule 0 = heuristic, 1 = increasing (Sec. 4, the brute
 * force comparator that raises the level every cycle), 2 = fixed level. */
int oracle_next_level(int rule, double ratio, int level)
{
    if (rule == 1) return level < OR_MAX_LEVEL ? level + 1 : level;
    if (rule == 2) return level;
    if (ratio > 0.4) return level < OR_MAX_LEVEL ? level + 1 : level;
    if (ratio < 0.4 && ratio > 0.2) return level > 0 ? level - 1 : level;
    return level;
}

/* Full SRJ solve (Sec. 3 data-collection loop and Sec. 4 experiments):
 *   r0 = ||f - A u0||; level = level0; repeat { M sweeps of the level's
 *   scheme; rn = ||f - A u||; ratio = rn / r_prev; stop if converged;
 *   level = Alg. 1(ratio, level) }.
 * tol_kind 0 = relative (Eq. relative-residual), 1 = absolute L2 norm,
 * 2 = ||x^n - x^{n-1}||_inf < tol after some sweep (Sec. 4.2.2; tested every
 * sweep, so the solve can stop inside a cycle).
 * Returns 0 converged, 1 sweep cap reached, 2 non-finite residual.
 * Trace arrays (may be NULL) receive per-cycle level, M and rn; at most
 * trace_cap cycles are recorded but the count returned in *cycles_out is the
 * true one. */
int oracle_srj_solve(const oracle_problem *P, const double *f, double *u,
                     double tol, int tol_kind, int rule, int level0,
                     long max_sweeps, long *sweeps_out, long *cycles_out,
                     double *r0_out, double *rn_out, int *trace_level,
                     double *trace_rn, long trace_cap)
{
    double *omega = (double *)malloc(sizeof(double) * 2362);
    const double r0 = oracle_residual_norm(P, u, f);
    double rprev = r0, rn = r0;
    int level = level0;
    long sweeps = 0, cycles = 0;
    int status = 1;
    if (r0_out) *r0_out = r0;
    if ((tol_kind != 2 && r0 == 0.0) || (tol_kind == 1 && r0 < tol)) {
        status = 0;
        goto done;
    }
    while (sweeps < max_sweeps) {
        const int M = oracle_level_omegas(level, omega);
        if (tol_kind == 2) {
            int reached = 0;
            sweeps += oracle_sweeps_dinf(P, u, f, omega, M, tol, &reached);
            if (reached) {
                rn = oracle_residual_norm(P, u, f);
                status = 0;
                break;
            }
        } else {
            oracle_sweeps(P, u, f, omega, M);
            sweeps += M;
        }
        rn = oracle_residual_norm(P, u, f);
        if (cycles < trace_cap) {
            if (trace_level) trace_level[cycles] = level;
            if (trace_rn) trace_rn[cycles] = rn;
        }
        cycles += 1;
        const double ratio = rn / rprev;
        rprev = rn;
        if (!isfinite(rn)) {
            status = 2;
            break;
        }
        if (tol_kind != 2 && (tol_kind == 0 ? rn / r0 : rn) < tol) {
            status = 0;
            break;
        }
        level = oracle_next_level(rule, ratio, level);
    }
done:
    if (sweeps_out) *sweeps_out = sweeps;
    if (cycles_out) *cycles_out = cycles;
    if (rn_out) *rn_out = rn;
    free(omega);
    return status;
}

/* Run an explicit list of levels (no selection): for parity of cycles.
 * rn_out[c] receives the residual norm after cycle c. */
void oracle_srj_run_levels(const oracle_problem *P, const double *f, double *u,
                           const int *levels, long ncycles, double *rn_out)
{
    double *omega = (double *)malloc(sizeof(double) * 2362);
    for (long c = 0; c < ncycles; ++c) {
        const int M = oracle_level_omegas(levels[c], omega);
        oracle_sweeps(P, u, f, omega, M);
        if (rn_out) rn_out[c] = oracle_residual_norm(P, u, f);
    }
    free(omega);
}

/* Plain (unrelaxed) Jacobi, Sec. 2 Eq. (jacobi): omega = 1 every sweep; the
 * residual is tested every check_every sweeps.  Returns 0 converged, 1 cap. */
int oracle_jacobi_solve(const oracle_problem *P, const double *f, double *u,
                        double tol, int tol_kind, long check_every,
                        long max_sweeps, long *sweeps_out, double *rn_out)
{
    const double r0 = oracle_residual_norm(P, u, f);
    const double one = 1.0;
    long sweeps = 0;
    double rn = r0;
    int status = 1;
    if (r0 == 0.0 && tol_kind != 2) status = 0;
    while (status != 0 && sweeps < max_sweeps) {
        if (tol_kind == 2) {
            int reached = 0;
            oracle_sweeps_dinf(P, u, f, &one, 1, tol, &reached);
            sweeps += 1;
            if (reached) status = 0;
            continue;
        }
        for (long s = 0; s < check_every; ++s) oracle_sweeps(P, u, f, &one, 1);
        sweeps += check_every;
        rn = oracle_residual_norm(P, u, f);
        if ((tol_kind == 0 ? rn / r0 : rn) < tol) status = 0;
    }
    if (sweeps_out) *sweeps_out = sweeps;
    if (rn_out) *rn_out = rn;
    return status;
}

/* Thomas algorithm: direct solve of a tridiagonal system
 *   a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,  i = 0..N-1
 * (a_0 and c_{N-1} unused).  Textbook forward elimination / back
 * substitution without pivoting; valid for the diagonally dominant matrices
 * of Sec. 3 and Sec. 4.2.1. */
void oracle_thomas(long N, const double *a, const double *b, const double *c,
                   const double *d, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * (size_t)N);
    double *dp = (double *)malloc(sizeof(double) * (size_t)N);
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (long i = 1; i < N; ++i) {
        const double m = b[i] - a[i] * cp[i - 1];
        cp[i] = (i < N - 1) ? c[i] / m : 0.0;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x[N - 1] = dp[N - 1];
    for (long i = N - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

/* ------------------------------------------------------------------------
 * Geometric multigrid with SRJ smoothing: an adjacent use of the method
 * (Sec. 1: Jacobi iteration is the usual multigrid smoother; Sec. 5: SRJ
 * schemes used as smoothers accelerate multigrid).  Textbook V-cycle:
 * nu1 SRJ cycles of one scheme level as pre-smoother, the residual,
 * full-weighting restriction to the grid with (n - 1) / 2 points and twice
 * the spacing per axis (the operator rediscretised there), the coarse
 * correction by recursion, (bi/tri)linear interpolation of the correction,
 * nu2 cycles as post-smoother.  On the one-point coarsest grid A u = f is
 * solved exactly, u = f / D.  Constant coefficients, zero Dirichlet values,
 * n = 2^k - 1 points on every axis with the same k.
 * ------------------------------------------------------------------------ */
static void or_mg_coarse(const oracle_problem *Pf, oracle_problem *Pc)
{
    *Pc = *Pf;
    for (int a = 0; a < Pf->dim; ++a) {
        Pc->n[a] = (Pf->n[a] - 1) / 2;
        Pc->h[a] = 2.0 * Pf->h[a];
    }
}

/* Full weighting: coarse point c sits on fine point 2c + 1 per axis; its value
 * is the sum over the 3^dim fine points around it with weight
 * prod_a (1/2 on the axis of c, 1/4 one step off). */
void oracle_mg_restrict(const oracle_problem *Pf, const double *rf,
                        const oracle_problem *Pc, double *fc)
{
    const long nf0 = Pf->n[0], nf1 = Pf->dim > 1 ? Pf->n[1] : 1;
    const int r1 = Pf->dim > 1 ? 1 : 0, r2 = Pf->dim > 2 ? 1 : 0;
    long i = 0;
    for (long z = 0; z < or_extent(Pc, 2); ++z)
        for (long y = 0; y < or_extent(Pc, 1); ++y)
            for (long x = 0; x < or_extent(Pc, 0); ++x, ++i) {
                double acc = 0.0;
                for (int dz = -r2; dz <= r2; ++dz)
                    for (int dy = -r1; dy <= r1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const long fx = 2 * x + 1 + dx;
                            const long fy = r1 ? 2 * y + 1 + dy : 0;
                            const long fz = r2 ? 2 * z + 1 + dz : 0;
                            double w = dx == 0 ? 0.5 : 0.25;
                            if (r1) w *= dy == 0 ? 0.5 : 0.25;
                            if (r2) w *= dz == 0 ? 0.5 : 0.25;
                            acc += w * rf[fx + nf0 * (fy + nf1 * fz)];
                        }
                fc[i] = acc;
            }
}

/* Linear interpolation per axis: a fine point 2c + 1 takes the coarse value
 * c; a fine point 2c takes half of coarse c - 1 and half of coarse c (zero
 * outside the coarse grid).  The interpolated correction is added to uf. */
void oracle_mg_prolong_add(const oracle_problem *Pc, const double *ec,
                           const oracle_problem *Pf, double *uf)
{
    const long nc0 = Pc->n[0], nc1 = Pc->dim > 1 ? Pc->n[1] : 1;
    long i = 0;
    for (long z = 0; z < or_extent(Pf, 2); ++z)
        for (long y = 0; y < or_extent(Pf, 1); ++y)
            for (long x = 0; x < or_extent(Pf, 0); ++x, ++i) {
                long cx[2], cy[2], cz[2];
                double wx[2], wy[2], wz[2];
                int mx, my, mz;
                /* coarse neighbours and weights per axis */
                if (x % 2 == 1) { cx[0] = x / 2; wx[0] = 1.0; mx = 1; }
                else { cx[0] = x / 2 - 1; cx[1] = x / 2; wx[0] = wx[1] = 0.5; mx = 2; }
                if (Pf->dim < 2) { cy[0] = 0; wy[0] = 1.0; my = 1; }
                else if (y % 2 == 1) { cy[0] = y / 2; wy[0] = 1.0; my = 1; }
                else { cy[0] = y / 2 - 1; cy[1] = y / 2; wy[0] = wy[1] = 0.5; my = 2; }
                if (Pf->dim < 3) { cz[0] = 0; wz[0] = 1.0; mz = 1; }
                else if (z % 2 == 1) { cz[0] = z / 2; wz[0] = 1.0; mz = 1; }
                else { cz[0] = z / 2 - 1; cz[1] = z / 2; wz[0] = wz[1] = 0.5; mz = 2; }
                double acc = 0.0;
                for (int c = 0; c < mz; ++c)
                    for (int b = 0; b < my; ++b)
                        for (int a = 0; a < mx; ++a) {
                            if (cx[a] < 0 || cx[a] >= nc0) continue;
                            if (Pf->dim > 1 && (cy[b] < 0 || cy[b] >= nc1)) continue;
                            if (Pf->dim > 2 && (cz[c] < 0 || cz[c] >= Pc->n[2])) continue;
                            acc += wx[a] * wy[b] * wz[c] * ec[cx[a] + nc0 * (cy[b] + nc1 * cz[c])];
                        }
                uf[i] += acc;
            }
}

/* One V-cycle on A u = f (u updated in place). */
void oracle_mg_vcycle(const oracle_problem *P, double *u, const double *f,
                      int level, int nu1, int nu2)
{
    const long N = or_npts(P);
    if (N == 1) {
        const long p[3] = {0, 0, 0};
        u[0] = f[0] / or_diag(P, p);
        return;
    }
    double omega[2362];
    const int M = oracle_level_omegas(level, omega);
    for (int c = 0; c < nu1; ++c) oracle_sweeps(P, u, f, omega, M);
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    oracle_apply_A(P, u, r);
    for (long i = 0; i < N; ++i) r[i] = f[i] - r[i];
    oracle_problem Pc;
    or_mg_coarse(P, &Pc);
    const long Nc = or_npts(&Pc);
    double *fc = (double *)malloc(sizeof(double) * (size_t)Nc);
    double *ec = (double *)calloc((size_t)Nc, sizeof(double));
    oracle_mg_restrict(P, r, &Pc, fc);
    oracle_mg_vcycle(&Pc, ec, fc, level, nu1, nu2);
    oracle_mg_prolong_add(&Pc, ec, P, u);
    for (int c = 0; c < nu2; ++c) oracle_sweeps(P, u, f, omega, M);
    free(r);
    free(fc);
    free(ec);
}

/* V-cycles until ||f - A u|| / ||f - A u0|| < tol; rn_trace (may be NULL,
 * capacity max_cycles) receives the norm after each V-cycle.  Returns 0 when
 * converged, 1 otherwise. */
int oracle_mg_solve(const oracle_problem *P, const double *f, double *u, double tol,
                    int level, int nu1, int nu2, long max_cycles, long *cycles_out,
                    double *r0_out, double *rn_out, double *rn_trace)
{
    const double r0 = oracle_residual_norm(P, u, f);
    double rn = r0;
    long c = 0;
    int status = r0 == 0.0 ? 0 : 1;
    while (status != 0 && c < max_cycles) {
        oracle_mg_vcycle(P, u, f, level, nu1, nu2);
        rn = oracle_residual_norm(P, u, f);
        if (rn_trace) rn_trace[c] = rn;
        c += 1;
        if (rn / r0 < tol) status = 0;
    }
    if (cycles_out) *cycles_out = c;
    if (r0_out) *r0_out = r0;
    if (rn_out) *rn_out = rn;
    return status;
}

/* ------------------------------------------------------------------------
 * Sec. 3 data collection (the procedure the heuristic of Alg. 1 was read
 * from).  A trial starts from x = 0 and applies one cycle at level 0; the
 * residual ratio after / before it and the level form the state.  Each later
 * step tries every allowed move from the current iterate -- decrease, keep,
 * increase the level, inside [0, max_level] -- one cycle each, and records
 * for each the state (previous ratio, current level), the move and the
 * residual norms before and after its cycle (its average convergence rate is
 * -log(after / before) / M, Eq. average-convergence-rate).  One of the tried
 * moves is then taken at random: its iterate, level and ratio become the next
 * state.  The trial ends once the taken iterate's residual norm is below tol
 * (the paper uses 1e-8), or after max_steps steps.
 *
 * The random move comes from a counter-based generator: the output function
 * of SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to the counter value
 * seed + (index + 1) * 0x9E3779B97F4A7C15, index = trial * 2^32 + step; the
 * move is candidate floor(u * ncand), u = (output >> 11) * 2^-53, computed
 * in integers.
 * ------------------------------------------------------------------------ */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int oracle_pick(uint64_t seed, long trial, long step, int ncand)
{
    const uint64_t index = ((uint64_t)trial << 32) + (uint64_t)step;
    const uint64_t bits = oracle_splitmix64(seed, index) >> 11;
    return (int)((bits * (uint64_t)ncand) >> 53);
}

/* One trial.  Records go to the arrays at positions 0 .. *nrec_out - 1
 * (capacity 3 * max_steps); the levels taken after the first cycle go to
 * taken_levels (capacity max_steps + 1, may be NULL).  Returns the number of
 * steps made. */
long oracle_collect_moves(const oracle_problem *P, const double *f, double tol, int max_level,
                          uint64_t seed, long trial, long max_steps, double *prev_ratio,
                          int *level, int *action, double *r_before, double *r_after,
                          long *nrec_out, int *taken_levels)
{
    const long N = or_npts(P);
    double *u = (double *)calloc((size_t)N, sizeof(double));
    double *w[3];
    for (int c = 0; c < 3; ++c) w[c] = (double *)malloc(sizeof(double) * (size_t)N);
    double *omega = (double *)malloc(sizeof(double) * 2362);
    const double r0 = oracle_residual_norm(P, u, f);
    /* the first cycle, at level 0 */
    int M = oracle_level_omegas(0, omega);
    oracle_sweeps(P, u, f, omega, M);
    double rcur = oracle_residual_norm(P, u, f);
    double prev = r0 > 0.0 ? rcur / r0 : 0.0;
    int L = 0;
    if (taken_levels) taken_levels[0] = 0;
    long nrec = 0, step = 0;
    for (; step < max_steps && !(rcur < tol); ++step) {
        int cand_level[3], cand_action[3], ncand = 0;
        double rc[3];
        for (int a = -1; a <= 1; ++a) {
            const int c = L + a;
            if (c < 0 || c > max_level) continue;
            memcpy(w[ncand], u, sizeof(double) * (size_t)N);
            M = oracle_level_omegas(c, omega);
            oracle_sweeps(P, w[ncand], f, omega, M);
            rc[ncand] = oracle_residual_norm(P, w[ncand], f);
            cand_level[ncand] = c;
            cand_action[ncand] = a;
            prev_ratio[nrec] = prev;
            level[nrec] = L;
            action[nrec] = a;
            r_before[nrec] = rcur;
            r_after[nrec] = rc[ncand];
            ++nrec;
            ++ncand;
        }
        const int k = oracle_pick(seed, trial, step, ncand);
        memcpy(u, w[k], sizeof(double) * (size_t)N);
        prev = rc[k] / rcur;
        rcur = rc[k];
        L = cand_level[k];
        (void)cand_action;
        if (taken_levels) taken_levels[step + 1] = L;
    }
    *nrec_out = nrec;
    free(u);
    for (int c = 0; c < 3; ++c) free(w[c]);
    free(omega);
    return step;
}
