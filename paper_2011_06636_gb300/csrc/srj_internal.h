// srj_internal.h -- declarations shared by the translation units of libsrj.so.
//
// Internal data layout (all working arrays are library-owned):
//   padded layout: index = x + pitch * y + plane * z, pitch = round_up(nx, 32)
//   elements, plane = pitch * ny.  Columns x in [nx, pitch) are zero and stay
//   zero (they act as the x = nx Dirichlet ghost column).  Points outside the
//   interior are zero (Dirichlet).  1D grids use ny = nz = 1, 2D nz = 1.
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is looked up at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/srj.h"

namespace srj {

constexpr int kMaxLevel = 24;
// Mixed precision: each inner solve after the first starts this many levels
// below the level the previous one ended at.  Measured on the 4096^2 Poisson
// solve: 0 -> 28 680 sweeps, 1 -> 30 470, 3 -> 32 853, 5 -> 31 858 (the
// correction's residual is dominated by the same smooth modes the previous
// inner solve was working on, so restarting lower only repeats the climb).
constexpr int kInnerCarry = 0;
constexpr int kNumLevels = 25;
// Polls of a bounded device-side wait (the 3D pass waiting for a staged plane)
// before it gives up and ends the solve with SRJ_ETIMEOUT; copies in flight
// are then still drained with this limit.
constexpr long long kDefaultWaitLimit = 1LL << 22;
constexpr int kTotalOmegas = 9710;  // sum of M over the 25 levels
constexpr int kBatchLayouts = 3;    // item layouts of the batched solve
// The factor tables end with kJacobiOnes factors omega = 1 (at offset
// kTotalOmegas): every pass of a plain-Jacobi solve reads its factors there.
constexpr int kJacobiOnes = 8;
constexpr int kTableOmegas = kTotalOmegas + kJacobiOnes;

// App. B table (scheme level -> M) and the offset of each level's factors in
// the concatenated factor table.  Defined in schemes.cpp.
extern const int kLevelM[kNumLevels];
int level_offset(int level);
// Sec. 2 Eq. (srj-relaxation-parameters) + Leja order; fills out[kTotalOmegas].
void build_omega_table(double *out);
int scheme_omegas(int level, double *out, int capacity);

// Selector values used on the device (srj_selector plus internal ones).
enum DevSelector : int32_t {
    DSEL_HEURISTIC = 0,
    DSEL_INCREASING = 1,
    DSEL_FIXED = 2,
    DSEL_MLP = 3,
    DSEL_JACOBI = 4,   // plain Jacobi (omega = 1), residual every M(fixed_level) sweeps
    DSEL_SCHEDULE = 5  // explicit level list (srj_run_levels)
};

// Status values of a device-side solve.
enum DevStatus : int32_t {
    DST_RUNNING = 0,
    DST_CONVERGED = 1,
    DST_NOTCONV = 2,
    DST_DIVERGED = 3,
    DST_STALLED = 4,  // inner solve of mixed precision: a cycle raised the residual
    DST_DONE = 5,     // explicit schedule finished
    DST_TIMEOUT = 6   // a bounded device-side wait ran out (SRJ_ETIMEOUT)
};

// Per-solve state in device memory.  The host writes the whole struct (the
// settings and the initial values) before each solve; afterwards it is written
// only by the last CTA of each pass (finish in kernels_generic.cu) and read by
// every CTA at the start of a pass.  Keeping the settings here (not in kernel
// arguments) lets one instantiated CUDA graph serve every solve on a handle.
struct DevState {
    // settings of this solve
    double tol;
    long long max_sweeps;
    int32_t tol_kind;     // srj_tol_kind
    int32_t selector;     // DevSelector
    int32_t fixed_level;
    int32_t max_level;
    int32_t stall_stop;   // 1: stop when a cycle's ratio >= 1 (inner of MIXED)
    int32_t nsched;       // DSEL_SCHEDULE: number of scheduled cycles
    long long wait_limit; // polls a bounded device-side wait makes before it gives up
    // running state
    int32_t level;        // level of the cycle in progress
    int32_t k;            // sweeps of the current cycle already done
    int32_t cur;          // ping-pong buffer holding the current iterate
    int32_t status;       // DevStatus
    int32_t phase;        // 0: initial residual r0 not yet taken
    int32_t trace_base;   // first trace slot of this solve
    long long sweeps, cycles, passes;
    double r0, rprev, rn;
    unsigned int ticket;  // CTAs finished in the current pass
    unsigned int pad1;
    // learned selector: history of log ratios (most recent first) and counters
    float hist[8];
    int32_t nhist;
    int32_t mlp_last;       // 1 when the current cycle's level was the network's pick
    int32_t mlp_fallbacks;  // cycles whose level came from Alg. 1 after a failed pick
    double alg1_rate;       // average convergence rate of the latest cycle Alg. 1 chose
    int32_t dim;
    double npoints;
    double dlast;  // SRJ_TOL_DINF: ||u^n - u^(n-1)||_inf of the latest sweep
};

// Static per-handle pointers passed by value to the pass kernels.
struct SolveCfg {
    const int32_t *sched;  // DSEL_SCHEDULE level list
    int32_t *trace_level;
    double *trace_rn;
    int32_t trace_cap;
    int32_t use_cond;      // 1 when launched inside a conditional while node
    cudaGraphConditionalHandle cond;
    const uint16_t *mlp_w;  // learned selector weights, BF16 (mlp.cuh)
};

// Grid geometry and constant coefficients.
struct GridGeo {
    int32_t dim;
    int32_t nx, ny, nz;
    long long pitch, plane;
    double cx, cy, cz;  // eps_a / h_a^2
    double diag;        // 2 (cx + cy + cz) for constant coefficients
    int32_t neu;        // bit a set: axis a has mirrored-ghost Neumann ends (Sec. 4.2.2)
    int32_t pad;
    // 1 / diag and c_a / diag, divided once on the host (FP64 division is
    // slow on the device and the kernels need them per thread)
    double invdiag, acx, acy, acz;
};

// Sets the axis coefficients of g and the values derived from them.
inline void geo_set_coefficients(GridGeo &g, double cx, double cy, double cz) {
    g.cx = cx;
    g.cy = cy;
    g.cz = cz;
    g.diag = 2.0 * (cx + cy + cz);
    g.invdiag = 1.0 / g.diag;
    g.acx = cx / g.diag;
    g.acy = cy / g.diag;
    g.acz = cz / g.diag;
}

enum Prec : int32_t { PREC_F64 = 0, PREC_F32 = 1, PREC_DF = 2 };

// Buffers of one iterate pair plus right-hand side, typeless.
//   F64: f = double*, u = double*;  F32: float*;  DF: f float*, u = hi float*,
//   ulo = lo float*.
struct IterBufs {
    const void *f;
    void *u[2];
    void *ulo[2];
    // variable coefficients (nullptr for constant): face weights eps*kf/h^2 on
    // the +x, +y, +z face of each cell and 1/D, in the padded layout, element
    // type double for F64, float for F32 / DF.
    const void *wx, *wy, *wz, *invd;
};

struct PassLaunch {
    GridGeo geo;
    IterBufs bufs;
    DevState *st;
    double *partials;      // one FP64 slot per CTA
    int partials_cap;
    const double *w64;     // device factor tables (kTotalOmegas)
    const float *w32;
    SolveCfg cfg;
    int lvl_m[kNumLevels];    // App. B: M of each level
    int lvl_off[kNumLevels];  // offset of each level's factors in w64 / w32
    int dinf;                 // 1: sweep passes also reduce max |u' - u| (SRJ_TOL_DINF)
    int tail_only;            // 1: the one-sweep 3D pass runs beside the two-sweep one
};

// Launch helpers implemented in kernels_generic.cu.  Each returns the CUDA
// error of the launch (cudaSuccess when queued).
struct GenericPlan {
    dim3 grid, block;
    int zchunk;    // z planes per thread (3D), rows per thread (2D)
    void *kernel;  // __global__ entry for graph nodes
    int smem;      // dynamic shared memory bytes
    int plane3d;   // 1: the 3D plane-streaming kernel (kernels_plane3d.cu)
};
// 3D Dirichlet passes: plane-streaming kernel with a cp.async ring of z planes
// (kernels_plane3d.cu); same grid and partial count as the generic 3D pass.
struct Plane3dPlan {
    dim3 grid, block;
    int zchunk;
    void *kernel;
    int smem;
};
Plane3dPlan plane3d_plan(int prec, const GridGeo &g, bool vark);
cudaError_t plane3d_prepare(int prec, bool vark);
// TMA tensor maps of the arrays the 3D pass stages (iterate pair hi / lo,
// rhs, face weights, 1/D), encoded once per handle.
struct Plane3dMaps {
    CUtensorMap u[2], ulo[2], f, wx, wy, wz, invd;
};
cudaError_t plane3d_encode(int prec, bool vark, const GridGeo &g, const IterBufs &b,
                           Plane3dMaps *m, bool two_sweep = false);
// Two sweeps per pass (kernels_plane3d.cu): the passes of a cycle that do two
// sweeps; the one-sweep pass (tail_only) does the rest.  Maps encoded with
// two_sweep = true.
Plane3dPlan plane3d2_plan(int prec, const GridGeo &g, bool vark, int num_sms);
cudaError_t plane3d2_prepare(int prec, bool vark);
GenericPlan generic_plan(int prec, const GridGeo &g, bool vark);
int generic_partials_needed(const GridGeo &g);
// maps: the handle's tensor maps, required when the plan is the 3D
// plane-streaming pass (GenericPlan::plane3d), else unused.
cudaError_t generic_pass_launch(int prec, bool vark, const PassLaunch &a, cudaStream_t s,
                                const struct Plane3dMaps *maps);
cudaError_t add_generic_pass_node(int prec, bool vark, const PassLaunch &a, cudaGraph_t body,
                                  const struct Plane3dMaps *maps);

// Whole solve of a small grid in one CTA (kernels_small.cu): the dynamic
// shared memory it needs, 0 when the grid does not fit.
int small_solve_smem(int prec, bool vark, const GridGeo &g);
cudaError_t small_solve_launch(int prec, bool vark, const PassLaunch &a, cudaStream_t s);

// Temporally blocked 2D constant-coefficient pass (kernels_wave2d.cu).
struct Wave2dPlan {
    int T;        // sweeps fused per pass
    void *entry;  // __global__ entry
    int smem;     // dynamic shared memory bytes
    int block, grid;
    int nstrips, nsegs, R, nitems;
};
int wave2d_depth(int prec, int requested);
Wave2dPlan wave2d_plan(int prec, int T, const GridGeo &g, int num_sms);
cudaError_t wave2d_prepare(int prec, int T);
cudaError_t wave2d_launch(const Wave2dPlan &p, const PassLaunch &a, cudaStream_t s);
cudaError_t add_wave2d_node(const Wave2dPlan &p, const PassLaunch &a, cudaGraph_t body);

// Batched persistent solve of many 2D constant-coefficient problems
// (kernels_batched.cu).  The problems are cut into items (strip x row segment)
// in kBatchLayouts layouts of decreasing segment height; each launch uses one
// layout for every problem, chosen at the end of the previous launch from the
// items the unfinished problems have (tall segments while the problems fill
// the GPU, short ones once a few large problems remain and the length of an
// item sets the time of a pass).  Per problem: immutable geometry and buffers ...
struct BatchProb {
    GridGeo geo;
    IterBufs inner;   // f = FP32 inner rhs, u[2] / ulo[2] = FP32-pair iterates (padded)
    const double *f;  // user arrays (dense FP64), set per solve
    double *u;
    // item decomposition of each layout (segment heights R, largest first)
    int nstrips;
    int nsegs[kBatchLayouts], R[kBatchLayouts], nitems[kBatchLayouts], item_base[kBatchLayouts];
};
// ... and a state machine OUTER -> INNER -> UPDATE -> OUTER ... -> DONE.
struct BatchState {
    DevState in;  // state of the current inner SRJ solve
    int32_t phase, outer, carry, result, final_level, pad;
    double r0, rn;  // FP64 outer residual norms
    long long sweeps, cycles, passes;
    unsigned int ticket, pad1;
};
struct BatchLaunch {
    const BatchProb *probs;
    BatchState *states;
    const int32_t *item_prob[kBatchLayouts];  // problem of every item (problem-major order)
    double *partials;          // one slot per item (of the largest layout)
    unsigned int *ndone;
    int nprob, total_items[kBatchLayouts];
    // layout choice: ctl[0] the layout of the running launch, ctl[1] the CTAs
    // that finished it; active[l]: items of the unfinished problems in layout l
    int32_t *ctl;
    long long *active;
    int resident_warps;  // warps the grid keeps resident
    int fixed_layout;    // >= 0: every launch uses this layout (autotuning)
    const double *w64;
    int lvl_m[kNumLevels], lvl_off[kNumLevels];
    double tol, inner_tol;
    long long max_sweeps;
    int max_outer, tol_kind, selector, max_level, fixed_level;
    int stall_stop;  // 0 while autotuning: inner solves never end, u is untouched
    SolveCfg cfg;
};
int batched_outw(int T);
int batched_smem(int T);
int batched_grid(int T, int num_sms);
cudaError_t batched_prepare(int T);
cudaError_t batched_launch(int T, int num_sms, const BatchLaunch &b, cudaStream_t s);
cudaError_t add_batched_node(int T, int num_sms, const BatchLaunch &b, cudaGraph_t body);

// Whole-grid helpers (kernels_generic.cu).
// FP64 outer residual of the mixed-precision path on dense user arrays:
// writes r into the padded FP32 inner right-hand side, ||r||^2 partials and a
// last-CTA total into *out_norm2 (with its own ticket counter).
struct OuterArgs {
    GridGeo geo;
    const double *f, *u;  // dense user arrays
    double *u_out;        // dense user array (update)
    float *r32;           // padded inner rhs
    const float *ehi[2], *elo[2];  // padded inner iterate pair
    const DevState *inner;         // inner solve state (selects ehi[cur])
    const double *wx, *wy, *wz, *invd;  // FP64 face weights (padded) or null
    double *partials;
    unsigned int *ticket;
    double *out_norm2;
};
cudaError_t outer_residual_launch(const OuterArgs &a, cudaStream_t s);
cudaError_t outer_update_launch(const OuterArgs &a, cudaStream_t s);
int outer_partials_needed(const GridGeo &g);

// Dense <-> padded copies (kernels_generic.cu).  copy_out picks the padded
// buffer holding the iterate from st->cur on the device.
cudaError_t copy_in_launch(int prec, const GridGeo &g, const void *dense, void *padded,
                           cudaStream_t s);
cudaError_t copy_out_launch(int prec, const GridGeo &g, const DevState *st, void *const *pads,
                            void *dense, cudaStream_t s);

// Face weights of an explicit symmetric operator (kernels_generic.cu):
// w_a = -A_(p,p+e_a) (zero where the neighbour is outside), invd = 1 / A_pp.
cudaError_t explicit_faces_launch(const GridGeo &g, const double *adiag,
                                  const double *const *aoff, double *wx, double *wy,
                                  double *wz, double *invd, float *wx32, float *wy32,
                                  float *wz32, float *invd32, cudaStream_t s);

// Face weights of the variable-coefficient operator (kernels_generic.cu).
cudaError_t vark_faces_launch(const GridGeo &g, const double *k, double *wx,
                              double *wy, double *wz, double *invd,
                              float *wx32, float *wy32, float *wz32,
                              float *invd32, cudaStream_t s);

// Multigrid with SRJ smoothing (kernels_mg.cu): dense x-fastest FP64 arrays,
// constant coefficients, zero Dirichlet values.
struct MgGeo {
    int dim;
    int nx, ny, nz;
    double cx, cy, cz;  // eps_a / h_a^2 (0 for axes >= dim)
    double diag;        // 2 (cx + cy + cz)
};
int mg_partials_needed();
cudaError_t mg_sweep_launch(const MgGeo &g, const double *u, double *uo, const double *f,
                            double omega, cudaStream_t s);
// r (may be null) = f - A u; partials (may be null): per-CTA sums of r^2, their
// count in *nparts
cudaError_t mg_residual_launch(const MgGeo &g, const double *u, const double *f, double *r,
                               double *partials, int *nparts, cudaStream_t s);
cudaError_t mg_sum_launch(const double *partials, int n, double *out, cudaStream_t s);
cudaError_t mg_restrict_launch(const MgGeo &gf, const double *r, const MgGeo &gc, double *fc,
                               cudaStream_t s);
cudaError_t mg_prolong_launch(const MgGeo &gc, const double *ec, const MgGeo &gf, double *u,
                              cudaStream_t s);

}  // namespace srj
