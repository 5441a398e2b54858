// api.cu -- the extern "C" entry points of libsrj.so (declared in
// include/srj.h) and the host-side orchestration:
//
//  * srj_create derives the geometry, uploads the scheme tables (Sec. 2,
//    App. B) and allocates the workspace.
//  * One SRJ solve is one launch of a CUDA graph made of a conditional WHILE
//    node whose body is a single pass kernel.  The pass kernels update a
//    device-resident state (cycle position, residual history, level chosen by
//    Alg. 1) and the last CTA of the final pass clears the loop condition, so
//    a whole solve -- thousands of passes -- runs without the host.
//  * SRJ_PREC_MIXED runs FP64 iterative refinement on the host side around
//    that graph: FP64 r = f - A u, inner SRJ on A e = r with FP32 arithmetic
//    on an FP32-pair iterate, FP64 u += e.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "srj_internal.h"

using namespace srj;

struct srj_handle {
    GridGeo geo{};
    int user_prec = SRJ_PREC_F64;  // srj_precision
    int kprec = PREC_F64;          // precision of the pass kernels
    bool vark = false;
    srj_opts opts{};
    cudaStream_t stream = nullptr;
    long long npts = 0;    // dense interior points
    long long padded = 0;  // padded elements (plane * nz)
    size_t esize = 8;      // user element size

    // scheme tables
    double *w64 = nullptr;
    float *w32 = nullptr;
    // iterate buffers (padded).  F64/F32: F, U[2].  MIXED: R32 (as F), E hi/lo.
    void *F = nullptr;
    void *U[2] = {nullptr, nullptr};
    void *Ulo[2] = {nullptr, nullptr};
    // variable coefficients
    double *wx64 = nullptr, *wy64 = nullptr, *wz64 = nullptr, *invd64 = nullptr;
    float *wx32 = nullptr, *wy32 = nullptr, *wz32 = nullptr, *invd32 = nullptr;
    // state, reductions, trace, schedule
    DevState *st = nullptr;
    DevState *h_st = nullptr;  // pinned
    double *partials = nullptr;
    int partials_cap = 0;
    int32_t *trace_level = nullptr;
    double *trace_rn = nullptr;
    int trace_cap = 0;
    int32_t *sched = nullptr;
    // mixed-precision outer
    double *opartials = nullptr;
    unsigned int *oticket = nullptr;
    double *onorm2 = nullptr;
    double *h_onorm2 = nullptr;  // pinned
    // dense device staging for srj_solve_host
    void *dF = nullptr, *dU = nullptr;
    // graph of the device-driven cycle loop
    bool host_loop = false;  // SRJ_LAUNCH=host: passes launched by a host loop
    bool use_wave = false;   // 2D constant coefficients: temporally blocked passes
    int small_smem = 0;      // > 0: the grid fits one CTA's shared memory (kernels_small.cu)
    Plane3dMaps *p3maps = nullptr;  // TMA tensor maps of the 3D pass (host copy)
    bool use_p3d2 = false;          // 3D: two sweeps per pass (plane3d2_kernel)
    Plane3dMaps *p3maps2 = nullptr; // its tensor maps (one box shape)
    Wave2dPlan wplan{};
    int num_sms = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evl0 = nullptr, evl1 = nullptr;  // around the cycle loop
    long long wait_limit = kDefaultWaitLimit;     // srj_set_wait_limit
    long long last_cycles = 0;
    std::string err;
    struct BatchData *batch = nullptr;  // srj_create_batched handles only
    struct MgData *mg = nullptr;        // srj_mg_create handles only
    uint16_t *mlp_w = nullptr;          // learned selector weights (BF16, 6617)
    bool mlp_loaded = false;
};

// Workspace and schedule of a batched handle.
struct BatchData {
    int nprob = 0;
    std::vector<BatchProb> probs;  // host copy of the descriptors
    std::vector<long long> npts;
    BatchProb *dprobs = nullptr;
    BatchState *dstates = nullptr;
    BatchState *hstates = nullptr;  // pinned
    int32_t *item_prob[kBatchLayouts] = {};
    double *partials = nullptr;
    int items_cap[kBatchLayouts] = {};
    unsigned int *ndone = nullptr;
    int32_t *ctl = nullptr;        // layout of the running launch, CTAs done with it
    long long *active = nullptr;   // items of the unfinished problems, per layout
    int partials_cap = 0;
    float *arena = nullptr;  // all inner buffers: per problem r32, hi0, hi1, lo0, lo1
    size_t arena_floats = 0;
    int T = 4, R = 64, total_items[kBatchLayouts] = {};
    bool tuned = false;
    double graph_tol = -1.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Hierarchy and the captured V-cycle of a multigrid handle.
struct MgData {
    int nlev = 0;
    std::vector<MgGeo> geo;  // level 0 = fine grid
    std::vector<double *> U0, U1, F, R;
    std::vector<double> omegas;  // the smoother's factors (one SRJ cycle)
    int nu1 = 1, nu2 = 1, max_cycles = 100;
    double *partials = nullptr, *norm2 = nullptr;
    double *h_norm2 = nullptr;  // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;  // private stream the V-cycle is captured on
    long long fine_sweeps = 0, launches = 0;  // per V-cycle
};

namespace {

const char *kVersion = "srj-gb300 0.1 (sm_103a)";

srj_status fail(srj_handle *h, srj_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

#define CK(call)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return fail(h, SRJ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    const cudaError_t e = cudaMalloc((void **)p, bytes);
    // a failed allocation also sets the runtime's last-error state, which a
    // later launch check (cudaGetLastError) would report as its own failure:
    // the failure is returned here, so clear it
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

// pinned host memory, with the same error handling as dalloc
template <typename T>
cudaError_t halloc(T **p, size_t bytes) {
    *p = nullptr;
    const cudaError_t e = cudaMallocHost((void **)p, bytes);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

PassLaunch make_launch(srj_handle *h, bool inner) {
    PassLaunch a{};
    a.geo = h->geo;
    a.bufs.f = h->F;
    a.bufs.u[0] = h->U[0];
    a.bufs.u[1] = h->U[1];
    a.bufs.ulo[0] = h->Ulo[0];
    a.bufs.ulo[1] = h->Ulo[1];
    if (h->vark) {
        const bool f64 = h->kprec == PREC_F64;
        a.bufs.wx = f64 ? (const void *)h->wx64 : (const void *)h->wx32;
        a.bufs.wy = f64 ? (const void *)h->wy64 : (const void *)h->wy32;
        a.bufs.wz = f64 ? (const void *)h->wz64 : (const void *)h->wz32;
        a.bufs.invd = f64 ? (const void *)h->invd64 : (const void *)h->invd32;
    }
    (void)inner;
    a.dinf = h->opts.tol_kind == SRJ_TOL_DINF;
    a.st = h->st;
    a.partials = h->partials;
    a.partials_cap = h->partials_cap;
    a.w64 = h->w64;
    a.w32 = h->w32;
    a.cfg.sched = h->sched;
    a.cfg.trace_level = h->trace_level;
    a.cfg.trace_rn = h->trace_rn;
    a.cfg.trace_cap = h->trace_cap;
    a.cfg.use_cond = 0;
    a.cfg.mlp_w = h->mlp_w;
    for (int l = 0; l < kNumLevels; ++l) {
        a.lvl_m[l] = kLevelM[l];
        a.lvl_off[l] = level_offset(l);
    }
    return a;
}

// Graph: WHILE(cond) { pass kernel }.  Built once per handle.
constexpr int kPassNodes = 4;  // generic pass nodes per iteration of the solve loop

// Kernel-node parameters of the 3D passes with two sweeps per pass: the
// two-sweep kernel and the one-sweep kernel in its tail role (a cycle's last
// single sweep, the residual).  args must outlive the use of the params.
struct P3d2Params {
    PassLaunch tail;
    int z2 = 0, z1 = 0;
    void *args2[3], *args1[3];
    cudaKernelNodeParams two{}, one{};
};
cudaError_t p3d2_params(srj_handle *h, const PassLaunch &a, P3d2Params &q) {
    const Plane3dPlan p2 = plane3d2_plan(h->kprec, h->geo, h->vark, h->num_sms);
    const GenericPlan p1 = generic_plan(h->kprec, h->geo, h->vark);
    cudaError_t e = plane3d2_prepare(h->kprec, h->vark);
    if (e == cudaSuccess) e = plane3d_prepare(h->kprec, h->vark);
    q.tail = a;
    q.tail.tail_only = 1;
    q.z2 = p2.zchunk;
    q.z1 = p1.zchunk;
    q.args2[0] = (void *)&a;
    q.args2[1] = (void *)&q.z2;
    q.args2[2] = (void *)h->p3maps2;
    q.args1[0] = (void *)&q.tail;
    q.args1[1] = (void *)&q.z1;
    q.args1[2] = (void *)h->p3maps;
    q.two.func = p2.kernel;
    q.two.gridDim = p2.grid;
    q.two.blockDim = p2.block;
    q.two.sharedMemBytes = p2.smem;
    q.two.kernelParams = q.args2;
    q.one.func = p1.kernel;
    q.one.gridDim = p1.grid;
    q.one.blockDim = p1.block;
    q.one.sharedMemBytes = p1.smem;
    q.one.kernelParams = q.args1;
    return e;
}

cudaError_t p3d2_launch_pair(srj_handle *h, const PassLaunch &a, cudaStream_t s) {
    P3d2Params q;
    cudaError_t e = p3d2_params(h, a, q);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernel(q.two.func, q.two.gridDim, q.two.blockDim, q.two.kernelParams,
                         q.two.sharedMemBytes, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(q.one.func, q.one.gridDim, q.one.blockDim, q.one.kernelParams,
                            q.one.sharedMemBytes, s);
}

srj_status build_graph(srj_handle *h) {
    if (h->exec) return SRJ_OK;
    CK(cudaGraphCreate(&h->graph, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, h->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, h->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    PassLaunch a = make_launch(h, true);
    a.cfg.use_cond = 1;
    a.cfg.cond = cond;
    if (h->use_wave) {
        CK(wave2d_prepare(h->kprec, h->wplan.T));
        CK(add_wave2d_node(h->wplan, a, body));
    } else if (h->use_p3d2) {
        // two (two-sweep pass, tail pass) pairs per evaluation of the condition
        P3d2Params q;
        CK(p3d2_params(h, a, q));
        cudaGraphNode_t prev = nullptr, nd;
        for (int i = 0; i < 2; ++i) {
            CK(cudaGraphAddKernelNode(&nd, body, prev ? &prev : nullptr, prev ? 1 : 0, &q.two));
            prev = nd;
            CK(cudaGraphAddKernelNode(&nd, body, &prev, 1, &q.one));
            prev = nd;
        }
    } else {
        CK(add_generic_pass_node(h->kprec, h->vark, a, body, h->p3maps));
        // one-sweep passes are short: chain copies of the pass node so that
        // the conditional node is evaluated once per kPassNodes passes (a pass
        // that starts after the end of the solve exits at once)
        size_t nn = 0;
        CK(cudaGraphGetNodes(body, nullptr, &nn));
        if (nn == 1) {
            cudaGraphNode_t prev;
            CK(cudaGraphGetNodes(body, &prev, &nn));
            cudaKernelNodeParams kp{};
            CK(cudaGraphKernelNodeGetParams(prev, &kp));
            for (int i = 1; i < kPassNodes; ++i) {
                cudaGraphNode_t nd;
                CK(cudaGraphAddKernelNode(&nd, body, &prev, 1, &kp));
                prev = nd;
            }
        }
    }
    CK(cudaGraphInstantiate(&h->exec, h->graph, 0));
    return SRJ_OK;
}

// Run the device-driven cycle loop until the solve state leaves RUNNING.
// Default: one launch of the graph (conditional WHILE around the pass kernel).
// With SRJ_LAUNCH=host (profilers cannot see kernels inside conditional
// graphs) the same pass kernel is launched directly in batches of 64 and the
// state is polled after each batch; passes issued after the end exit at once.
srj_status run_loop(srj_handle *h) {
    if (h->small_smem > 0 && !h->host_loop) {  // the whole solve in one CTA
        PassLaunch a = make_launch(h, true);
        CK(small_solve_launch(h->kprec, h->vark, a, h->stream));
        return SRJ_OK;
    }
    if (!h->host_loop) {
        CK(cudaGraphLaunch(h->exec, h->stream));
        return SRJ_OK;
    }
    PassLaunch a = make_launch(h, true);
    for (;;) {
        for (int i = 0; i < 64; ++i) {
            if (h->use_wave) CK(wave2d_launch(h->wplan, a, h->stream));
            else if (h->use_p3d2) CK(p3d2_launch_pair(h, a, h->stream));
            else CK(generic_pass_launch(h->kprec, h->vark, a, h->stream, h->p3maps));
        }
        DevState *probe = h->h_st;
        CK(cudaMemcpyAsync(probe, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (probe->status != DST_RUNNING) return SRJ_OK;
    }
}

// run_loop bracketed by the loop events; loop_ms() reads their interval once
// the stream has passed the second one.
srj_status run_loop_timed(srj_handle *h) {
    CK(cudaEventRecord(h->evl0, h->stream));
    const srj_status s = run_loop(h);
    if (s != SRJ_OK) return s;
    CK(cudaEventRecord(h->evl1, h->stream));
    return SRJ_OK;
}

double loop_seconds(srj_handle *h) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->evl0, h->evl1) != cudaSuccess) return 0.0;
    return ms * 1e-3;
}

void init_state(srj_handle *h, DevState &s, double tol, int tol_kind, int selector,
                int level0, long long max_sweeps, int stall_stop, int nsched, int trace_base) {
    std::memset(&s, 0, sizeof(s));
    s.tol = tol;
    s.tol_kind = tol_kind;
    s.selector = selector;
    s.fixed_level = h->opts.fixed_level;
    s.max_level = h->opts.max_level;
    s.max_sweeps = max_sweeps;
    s.stall_stop = stall_stop;
    s.nsched = nsched;
    s.level = level0;
    s.trace_base = trace_base;
    s.status = DST_RUNNING;
    s.dim = h->geo.dim;
    s.npoints = (double)h->npts;
    s.wait_limit = h->wait_limit;
}

srj_status status_of(int dst) {
    switch (dst) {
        case DST_CONVERGED:
        case DST_DONE:
            return SRJ_OK;
        case DST_DIVERGED:
            return SRJ_EDIVERGED;
        case DST_TIMEOUT:
            return SRJ_ETIMEOUT;
        default:
            return SRJ_ENOTCONV;
    }
}

// Plain F64 / F32 solve on DEVICE dense arrays (timed by the caller's events).
srj_status solve_plain(srj_handle *h, const void *f, void *u, double tol, int selector,
                       int level0, int nsched, srj_stats *stats) {
    srj_status s = build_graph(h);
    if (s != SRJ_OK) return s;
    cudaStream_t st = h->stream;
    CK(copy_in_launch(h->kprec, h->geo, f, h->F, st));
    CK(copy_in_launch(h->kprec, h->geo, u, h->U[0], st));
    init_state(h, *h->h_st, tol, h->opts.tol_kind, selector, level0, h->opts.max_sweeps, 0,
               nsched, 0);
    CK(cudaMemcpyAsync(h->st, h->h_st, sizeof(DevState), cudaMemcpyHostToDevice, st));
    s = run_loop_timed(h);
    if (s != SRJ_OK) return s;
    void *pads[2] = {h->U[0], h->U[1]};
    CK(copy_out_launch(h->kprec, h->geo, h->st, pads, u, st));
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const DevState &r = *h->h_st;
    h->last_cycles = r.cycles;
    if (stats) {
        stats->inner_seconds = loop_seconds(h);
        stats->status = status_of(r.status);
        stats->final_level = r.level;
        stats->sweeps = r.sweeps;
        stats->cycles = r.cycles;
        stats->outer = 0;
        stats->passes = r.passes;
        stats->r0 = r.r0;
        stats->rn = r.rn;
    }
    const srj_status result = status_of(r.status);
    if (h->opts.tol_kind == SRJ_TOL_DINF && stats) {
        // the per-sweep test can end a solve inside a cycle, after the last
        // cycle-end residual: take ||f - A u|| of the final iterate
        const DevState fin = r;
        init_state(h, *h->h_st, 1.0, SRJ_TOL_REL, DSEL_HEURISTIC, 0, 0, 0, 0, 0);
        h->h_st->cur = fin.cur;
        CK(cudaMemcpyAsync(h->st, h->h_st, sizeof(DevState), cudaMemcpyHostToDevice, st));
        PassLaunch a = make_launch(h, false);
        CK(generic_pass_launch(h->kprec, h->vark, a, st, h->p3maps));
        CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats->rn = h->h_st->r0;
    }
    return result;
}

// FP64 iterative refinement around FP32-arithmetic inner SRJ solves.
srj_status solve_mixed(srj_handle *h, const double *f, double *u, double tol, srj_stats *stats) {
    srj_status s = build_graph(h);
    if (s != SRJ_OK) return s;
    cudaStream_t st = h->stream;
    OuterArgs oa{};
    oa.geo = h->geo;
    oa.f = f;
    oa.u = u;
    oa.u_out = u;
    oa.r32 = (float *)h->F;
    oa.ehi[0] = (const float *)h->U[0];
    oa.ehi[1] = (const float *)h->U[1];
    oa.elo[0] = (const float *)h->Ulo[0];
    oa.elo[1] = (const float *)h->Ulo[1];
    oa.inner = h->st;
    oa.wx = h->wx64;
    oa.wy = h->wy64;
    oa.wz = h->wz64;
    oa.invd = h->invd64;
    oa.partials = h->opartials;
    oa.ticket = h->oticket;
    oa.out_norm2 = h->onorm2;

    const long long kInnerCap = 200000;  // sweeps of one inner solve
    const long long max_sweeps = h->opts.max_sweeps;
    long long sweeps = 0, cycles = 0, passes = 0, outer = 0;
    double r0 = 0.0, rn = 0.0;
    int level = h->opts.level0, final_level = level;
    int result = DST_NOTCONV;
    int trace_base = 0;
    double inner_s = 0.0;
    const size_t ebytes = (size_t)h->padded * sizeof(float);
    for (;;) {
        CK(outer_residual_launch(oa, st));
        CK(cudaMemcpyAsync(h->h_onorm2, h->onorm2, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (outer > 0) {  // fold in the inner solve that just finished
            const DevState &r = *h->h_st;
            inner_s += loop_seconds(h);
            sweeps += r.sweeps;
            cycles += r.cycles;
            passes += r.passes;
            final_level = r.level;
            level = r.level - kInnerCarry > 0 ? r.level - kInnerCarry : 0;
            trace_base += (int)r.cycles;
            if (r.status == DST_DIVERGED || r.status == DST_TIMEOUT) {
                result = r.status;
                break;
            }
        }
        rn = std::sqrt(*h->h_onorm2);
        if (outer == 0) r0 = rn;
        if (!std::isfinite(rn)) {
            result = DST_DIVERGED;
            break;
        }
        const double test = h->opts.tol_kind == SRJ_TOL_ABS ? rn : (r0 > 0 ? rn / r0 : 0.0);
        if (rn == 0.0 || test < tol) {
            result = DST_CONVERGED;
            break;
        }
        if (sweeps >= max_sweeps || outer >= 200) {
            result = DST_NOTCONV;
            break;
        }
        CK(cudaMemsetAsync(h->U[0], 0, ebytes, st));
        CK(cudaMemsetAsync(h->Ulo[0], 0, ebytes, st));
        // the inner solve aims at the reduction still needed (with margin 2),
        // but not below the FP32-pair accuracy floor opts.inner_tol
        const double target = h->opts.tol_kind == SRJ_TOL_ABS ? tol : tol * r0;
        double eta = 0.5 * target / rn;
        if (eta < h->opts.inner_tol) eta = h->opts.inner_tol;
        if (eta > 0.5) eta = 0.5;
        const long long inner_cap = max_sweeps - sweeps < kInnerCap ? max_sweeps - sweeps
                                                                    : kInnerCap;
        init_state(h, *h->h_st, eta, SRJ_TOL_REL, h->opts.selector, level, inner_cap, 1, 0,
                   trace_base);
        CK(cudaMemcpyAsync(h->st, h->h_st, sizeof(DevState), cudaMemcpyHostToDevice, st));
        s = run_loop_timed(h);
        if (s != SRJ_OK) return s;
        CK(outer_update_launch(oa, st));
        CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
        outer += 1;
    }
    h->last_cycles = cycles;
    if (stats) {
        stats->status = status_of(result);
        stats->final_level = final_level;
        stats->sweeps = sweeps;
        stats->cycles = cycles;
        stats->outer = outer;
        stats->passes = passes;
        stats->r0 = r0;
        stats->rn = rn;
        stats->inner_seconds = inner_s;
    }
    return status_of(result);
}

// ------------------------------------------------------------------ batched
// Item tables for temporal depth T and segment height R (problem-major).
srj_status batch_layout(srj_handle *h, int T, int R) {
    BatchData *B = h->batch;
    const int outw = batched_outw(T);
    // segment heights of the layouts: the tuned one, then a quarter and an
    // eighth of it (at least 4 rows)
    int Rl[kBatchLayouts] = {R, R / 4, R / 8};
    for (int l = 1; l < kBatchLayouts; ++l)
        if (Rl[l] < 4) Rl[l] = 4;
    std::vector<int32_t> owner[kBatchLayouts];
    int base[kBatchLayouts] = {};
    for (int p = 0; p < B->nprob; ++p) {
        BatchProb &P = B->probs[p];
        P.nstrips = (P.geo.nx + outw - 1) / outw;
        for (int l = 0; l < kBatchLayouts; ++l) {
            P.R[l] = Rl[l] < P.geo.ny ? Rl[l] : P.geo.ny;
            P.nsegs[l] = (P.geo.ny + P.R[l] - 1) / P.R[l];
            P.nitems[l] = P.nstrips * P.nsegs[l];
            P.item_base[l] = base[l];
            for (int i = 0; i < P.nitems[l]; ++i) owner[l].push_back(p);
            base[l] += P.nitems[l];
        }
    }
    B->T = T;
    B->R = R;
    int most = 0;
    for (int l = 0; l < kBatchLayouts; ++l) {
        B->total_items[l] = base[l];
        if (base[l] > most) most = base[l];
        if (base[l] > B->items_cap[l]) {
            dfree(B->item_prob[l]);
            B->item_prob[l] = nullptr;
            if (dalloc(&B->item_prob[l], (size_t)base[l] * sizeof(int32_t)) != cudaSuccess)
                return fail(h, SRJ_ENOMEM, "batched item tables");
            B->items_cap[l] = base[l];
        }
        CK(cudaMemcpyAsync(B->item_prob[l], owner[l].data(), (size_t)base[l] * sizeof(int32_t),
                           cudaMemcpyHostToDevice, h->stream));
    }
    if (most > B->partials_cap) {
        dfree(B->partials);
        B->partials = nullptr;
        if (dalloc(&B->partials, (size_t)most * sizeof(double)) != cudaSuccess)
            return fail(h, SRJ_ENOMEM, "batched partials");
        B->partials_cap = most;
    }
    CK(cudaMemcpyAsync(B->dprobs, B->probs.data(), B->probs.size() * sizeof(BatchProb),
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SRJ_OK;
}

// Warps the batched grid keeps resident (the layout choice compares item
// counts against it).
int batch_resident_warps(srj_handle *h) {
    return batched_grid(h->batch->T, h->num_sms) * (h->batch->T >= 4 ? 8 : 6);
}

BatchLaunch batch_args(srj_handle *h, double tol, bool tuning) {
    BatchData *B = h->batch;
    BatchLaunch b{};
    b.probs = B->dprobs;
    b.states = B->dstates;
    for (int l = 0; l < kBatchLayouts; ++l) {
        b.item_prob[l] = B->item_prob[l];
        b.total_items[l] = B->total_items[l];
    }
    b.ctl = B->ctl;
    b.active = B->active;
    b.resident_warps = batch_resident_warps(h);
    b.fixed_layout = tuning ? 0 : -1;
    b.partials = B->partials;
    b.ndone = B->ndone;
    b.nprob = B->nprob;
    b.w64 = h->w64;
    for (int l = 0; l < kNumLevels; ++l) {
        b.lvl_m[l] = kLevelM[l];
        b.lvl_off[l] = level_offset(l);
    }
    b.tol = tol;
    b.inner_tol = tuning ? -1.0 : h->opts.inner_tol;
    b.max_sweeps = tuning ? (1LL << 60) : h->opts.max_sweeps;
    b.max_outer = 200;
    b.tol_kind = h->opts.tol_kind;
    b.selector = h->opts.selector;
    b.max_level = h->opts.max_level;
    b.fixed_level = h->opts.fixed_level;
    b.stall_stop = tuning ? 0 : 1;
    b.cfg.trace_cap = 0;
    b.cfg.mlp_w = h->mlp_w;
    return b;
}

srj_status batch_reset(srj_handle *h) {
    BatchData *B = h->batch;
    for (int p = 0; p < B->nprob; ++p) {
        BatchState &S = B->hstates[p];
        std::memset(&S, 0, sizeof(S));
        S.phase = 0;  // outer residual first
        S.carry = h->opts.level0;
        S.result = DST_RUNNING;
    }
    CK(cudaMemcpyAsync(B->dstates, B->hstates, (size_t)B->nprob * sizeof(BatchState),
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(B->ndone, 0, sizeof(unsigned int), h->stream));
    // every problem active: the first launch takes the tallest layout whose
    // items cover the resident warps
    long long act[kBatchLayouts];
    int32_t ctl[2] = {kBatchLayouts - 1, 0};
    for (int l = 0; l < kBatchLayouts; ++l) act[l] = B->total_items[l];
    for (int l = kBatchLayouts - 1; l >= 0; --l)
        if (act[l] >= batch_resident_warps(h)) ctl[0] = l;
    CK(cudaMemcpyAsync(B->active, act, sizeof(act), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(B->ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemsetAsync(B->arena, 0, B->arena_floats * sizeof(float), h->stream));
    return SRJ_OK;
}

// Choose (T, R) by timing a window of batched launches on the real problems.
// During tuning the inner solves never end (tolerance < 0, no stall stop), so
// no UPDATE step runs and the caller's u is only read.
srj_status batch_autotune(srj_handle *h) {
    BatchData *B = h->batch;
    std::string key;
    {
        char buf[64];
        snprintf(buf, sizeof buf, "n%d", B->nprob);
        key = buf;
        unsigned long long hsh = 1469598103934665603ULL;
        for (const BatchProb &P : B->probs) {
            hsh = (hsh ^ (unsigned long long)P.geo.nx) * 1099511628211ULL;
            hsh = (hsh ^ (unsigned long long)P.geo.ny) * 1099511628211ULL;
        }
        snprintf(buf, sizeof buf, "-%016llx", hsh);
        key += buf;
    }
    const char *cache = std::getenv("SRJ_AUTOTUNE_CACHE");
    if (cache) {
        FILE *fp = std::fopen(cache, "r");
        if (fp) {
            char k[128];
            int T, R;
            while (std::fscanf(fp, "%127s %d %d", k, &T, &R) == 3) {
                if (key == k) {
                    std::fclose(fp);
                    srj_status s = batch_layout(h, T, R);
                    if (s == SRJ_OK) B->tuned = true;
                    return s;
                }
            }
            std::fclose(fp);
        }
    }
    const int Ts[2] = {2, 4};
    const int Rs[3] = {32, 64, 128};
    double best = -1.0;
    int bestT = 4, bestR = 64;
    for (int T : Ts) {
        if (h->opts.temporal_depth && T != h->opts.temporal_depth) continue;
        CK(batched_prepare(T));
        for (int R : Rs) {
            srj_status s = batch_layout(h, T, R);
            if (s != SRJ_OK) return s;
            s = batch_reset(h);
            if (s != SRJ_OK) return s;
            BatchLaunch b = batch_args(h, 1e-300, true);
            for (int i = 0; i < 4; ++i) CK(batched_launch(T, h->num_sms, b, h->stream));
            CK(cudaMemcpyAsync(B->hstates, B->dstates, (size_t)B->nprob * sizeof(BatchState),
                               cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            std::vector<long long> before(B->nprob);
            for (int p = 0; p < B->nprob; ++p) before[p] = B->hstates[p].in.sweeps;
            CK(cudaEventRecord(h->ev0, h->stream));
            for (int i = 0; i < 12; ++i) CK(batched_launch(T, h->num_sms, b, h->stream));
            CK(cudaEventRecord(h->ev1, h->stream));
            CK(cudaMemcpyAsync(B->hstates, B->dstates, (size_t)B->nprob * sizeof(BatchState),
                               cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
            double lups = 0.0;
            for (int p = 0; p < B->nprob; ++p)
                lups += (double)(B->hstates[p].in.sweeps - before[p]) * (double)B->npts[p];
            const double rate = ms > 0 ? lups / ms : 0.0;
            if (rate > best) {
                best = rate;
                bestT = T;
                bestR = R;
            }
        }
    }
    srj_status s = batch_layout(h, bestT, bestR);
    if (s != SRJ_OK) return s;
    B->tuned = true;
    if (cache) {
        FILE *fp = std::fopen(cache, "a");
        if (fp) {
            std::fprintf(fp, "%s %d %d\n", key.c_str(), bestT, bestR);
            std::fclose(fp);
        }
    }
    return SRJ_OK;
}

srj_status batch_build_graph(srj_handle *h, double tol) {
    BatchData *B = h->batch;
    if (B->exec && B->graph_tol == tol) return SRJ_OK;
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        cudaGraphDestroy(B->graph);
        B->exec = nullptr;
        B->graph = nullptr;
    }
    CK(batched_prepare(B->T));
    CK(cudaGraphCreate(&B->graph, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, B->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, B->graph, nullptr, nullptr, 0, &np));
    BatchLaunch b = batch_args(h, tol, false);
    b.cfg.use_cond = 1;
    b.cfg.cond = cond;
    CK(add_batched_node(B->T, h->num_sms, b, np.conditional.phGraph_out[0]));
    CK(cudaGraphInstantiate(&B->exec, B->graph, 0));
    B->graph_tol = tol;
    return SRJ_OK;
}

}  // namespace

extern "C" {

const char *srj_version(void) { return kVersion; }

int32_t srj_level_m(int32_t level) {
    if (level < 0 || level > kMaxLevel) return -1;
    return kLevelM[level];
}

int32_t srj_scheme_omegas(int32_t level, double *omega_out, int32_t capacity) {
    return scheme_omegas(level, omega_out, capacity);
}

srj_status srj_create(const srj_grid *grid, const srj_stencil *stencil, const srj_opts *opts,
                      void *stream, srj_handle **out) {
    srj_handle *h = nullptr;
    if (out) *out = nullptr;
    if (!grid || !out) return SRJ_EINVAL;
    if (grid->dim < 1 || grid->dim > 3) return SRJ_EINVAL;
    int neu = 0;
    for (int a = 0; a < grid->dim; ++a) {
        if (grid->n[a] < 1 || grid->n[a] > (1LL << 30) || grid->h[a] < 0 ||
            !std::isfinite(grid->h[a]))
            return SRJ_EINVAL;
        if (grid->bc[a] != SRJ_BC_DIRICHLET && grid->bc[a] != SRJ_BC_NEUMANN) return SRJ_EINVAL;
        if (grid->bc[a] == SRJ_BC_NEUMANN) {
            if (grid->n[a] < 2) return SRJ_EINVAL;
            neu |= 1 << a;
        }
    }
    const bool expl = stencil && stencil->a_diag;
    if (expl) {
        if (stencil->k) return SRJ_EINVAL;
        for (int a = 0; a < grid->dim; ++a)
            if (!stencil->a_off[a]) return SRJ_EINVAL;
    }
    if (neu || (opts && opts->tol_kind == SRJ_TOL_DINF)) {
        // mirrored ghosts and the per-sweep change test live in the one-sweep
        // pass kernel, for constant coefficients and one-level arithmetic
        if ((stencil && (stencil->k || expl)) || (opts && opts->precision == SRJ_PREC_MIXED))
            return SRJ_EUNSUPPORTED;
    }
    h = new (std::nothrow) srj_handle();
    if (!h) return SRJ_ENOMEM;
    srj_opts o{};
    if (opts) o = *opts;
    if (o.max_level == 0) o.max_level = kMaxLevel;
    if (o.trace_capacity == 0) o.trace_capacity = 4096;
    if (o.max_sweeps == 0) o.max_sweeps = 1000000LL;
    if (o.inner_tol == 0) o.inner_tol = 1e-6;
    auto bad = [&](const char *m) {
        delete h;
        (void)m;
        return SRJ_EINVAL;
    };
    if (o.selector < 0 || o.selector > SRJ_SEL_JACOBI) return bad("selector");
    if (o.precision < 0 || o.precision > SRJ_PREC_MIXED) return bad("precision");
    if (o.tol_kind != SRJ_TOL_REL && o.tol_kind != SRJ_TOL_ABS && o.tol_kind != SRJ_TOL_DINF)
        return bad("tol_kind");
    if (o.max_level < 0 || o.max_level > kMaxLevel) return bad("max_level");
    if (o.level0 < 0 || o.level0 > o.max_level) return bad("level0");
    if (o.fixed_level < 0 || o.fixed_level > o.max_level) return bad("fixed_level");
    if (o.trace_capacity < 0 || o.max_sweeps < 0 || o.inner_tol < 0 || o.temporal_depth < 0)
        return bad("negative option");
    h->opts = o;
    h->stream = (cudaStream_t)stream;
    h->user_prec = o.precision;
    h->kprec = o.precision == SRJ_PREC_F64 ? PREC_F64
                                            : (o.precision == SRJ_PREC_F32 ? PREC_F32 : PREC_DF);
    h->esize = o.precision == SRJ_PREC_F32 ? 4 : 8;

    GridGeo &g = h->geo;
    g.dim = grid->dim;
    g.nx = (int)grid->n[0];
    g.ny = grid->dim > 1 ? (int)grid->n[1] : 1;
    g.nz = grid->dim > 2 ? (int)grid->n[2] : 1;
    double hh[3], ee[3];
    for (int a = 0; a < 3; ++a) {
        const long long na = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
        // unit domain: n interior points (Dirichlet) or n nodes incl. both ends (Neumann)
        const bool na_neu = (neu >> a) & 1;
        hh[a] = (a < grid->dim && grid->h[a] > 0)
                    ? grid->h[a]
                    : 1.0 / (double)(na_neu ? na - 1 : na + 1);
        const double e = stencil ? stencil->eps[a] : 0.0;
        if (e < 0 || !std::isfinite(e)) return bad("eps");
        ee[a] = e > 0 ? e : 1.0;
    }
    geo_set_coefficients(g, ee[0] / (hh[0] * hh[0]), g.dim > 1 ? ee[1] / (hh[1] * hh[1]) : 0.0,
                         g.dim > 2 ? ee[2] / (hh[2] * hh[2]) : 0.0);
    g.neu = neu;
    g.pitch = ((long long)g.nx + 31) / 32 * 32;
    g.plane = g.pitch * g.ny;
    h->npts = (long long)g.nx * g.ny * g.nz;
    h->padded = g.plane * g.nz;
    h->vark = stencil && (stencil->k || stencil->a_diag);

    // scheme tables
    std::vector<double> w(kTableOmegas, 1.0);  // the scheme factors, then the Jacobi ones
    build_omega_table(w.data());
    std::vector<float> wf(kTableOmegas);
    for (int i = 0; i < kTableOmegas; ++i) wf[i] = (float)w[i];
#define ALLOC(ptr, bytes)                                      \
    do {                                                       \
        if (dalloc(&(ptr), (bytes)) != cudaSuccess) {          \
            srj_destroy(h);                                    \
            return SRJ_ENOMEM;                                 \
        }                                                      \
    } while (0)
    ALLOC(h->w64, kTableOmegas * sizeof(double));
    ALLOC(h->w32, kTableOmegas * sizeof(float));
    const size_t kb = h->kprec == PREC_F64 ? 8 : 4;
    ALLOC(h->F, h->padded * kb);
    ALLOC(h->U[0], h->padded * kb);
    ALLOC(h->U[1], h->padded * kb);
    if (h->kprec == PREC_DF) {
        ALLOC(h->Ulo[0], h->padded * 4);
        ALLOC(h->Ulo[1], h->padded * 4);
    }
    if (h->vark) {
        ALLOC(h->wx64, h->padded * 8);
        ALLOC(h->wy64, h->padded * 8);
        ALLOC(h->wz64, h->padded * 8);
        ALLOC(h->invd64, h->padded * 8);
        ALLOC(h->wx32, h->padded * 4);
        ALLOC(h->wy32, h->padded * 4);
        ALLOC(h->wz32, h->padded * 4);
        ALLOC(h->invd32, h->padded * 4);
    }
    ALLOC(h->st, sizeof(DevState));
    ALLOC(h->mlp_w, 6617 * sizeof(uint16_t));
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) !=
                cudaSuccess ||
            h->num_sms <= 0)
            h->num_sms = 152;
    }
    h->use_wave = (g.dim == 2) && !h->vark && !neu && o.tol_kind != SRJ_TOL_DINF;
    {
        const char *lm = std::getenv("SRJ_LAUNCH");
        h->host_loop = lm && std::strcmp(lm, "host") == 0;
    }
    h->small_smem = small_solve_smem(h->kprec, h->vark, g);
    h->partials_cap = generic_partials_needed(g);
    if (h->use_wave) {
        h->wplan = wave2d_plan(h->kprec, wave2d_depth(h->kprec, o.temporal_depth), g, h->num_sms);
        if (h->wplan.grid > h->partials_cap) h->partials_cap = h->wplan.grid;
    }
    ALLOC(h->partials, (size_t)h->partials_cap * sizeof(double));
    h->trace_cap = o.trace_capacity > 0 ? o.trace_capacity : 1;
    ALLOC(h->trace_level, (size_t)h->trace_cap * sizeof(int32_t));
    ALLOC(h->trace_rn, (size_t)h->trace_cap * sizeof(double));
    ALLOC(h->sched, (size_t)h->trace_cap * sizeof(int32_t));
    if (h->user_prec == SRJ_PREC_MIXED) {
        ALLOC(h->opartials, (size_t)outer_partials_needed(g) * sizeof(double));
        ALLOC(h->oticket, sizeof(unsigned int));
        ALLOC(h->onorm2, sizeof(double));
    }
#undef ALLOC
    if (halloc(&h->h_st, sizeof(DevState)) != cudaSuccess ||
        halloc(&h->h_onorm2, sizeof(double)) != cudaSuccess) {
        srj_destroy(h);
        return SRJ_ENOMEM;
    }
    cudaStream_t s = h->stream;
    srj_status rc = SRJ_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && rc == SRJ_OK) {
            rc = SRJ_ECUDA;
            h->err = std::string(what) + ": " + cudaGetErrorString(e);
        }
    };
    ck(cudaMemcpyAsync(h->w64, w.data(), kTableOmegas * sizeof(double), cudaMemcpyHostToDevice, s),
       "upload w64");
    ck(cudaMemcpyAsync(h->w32, wf.data(), kTableOmegas * sizeof(float), cudaMemcpyHostToDevice, s),
       "upload w32");
    // padding columns must read as zero; iterate buffers start at zero
    for (void *p : {h->F, h->U[0], h->U[1]}) ck(cudaMemsetAsync(p, 0, h->padded * kb, s), "memset");
    for (void *p : {h->Ulo[0], h->Ulo[1]})
        if (p) ck(cudaMemsetAsync(p, 0, h->padded * 4, s), "memset");
    ck(cudaMemsetAsync(h->st, 0, sizeof(DevState), s), "memset");
    if (h->oticket) ck(cudaMemsetAsync(h->oticket, 0, sizeof(unsigned int), s), "memset");
    if (h->vark) {
        for (void *p : {(void *)h->wx64, (void *)h->wy64, (void *)h->wz64, (void *)h->invd64})
            ck(cudaMemsetAsync(p, 0, h->padded * 8, s), "memset");
        for (void *p : {(void *)h->wx32, (void *)h->wy32, (void *)h->wz32, (void *)h->invd32})
            ck(cudaMemsetAsync(p, 0, h->padded * 4, s), "memset");
        if (stencil->a_diag) {
            const double *aoff[3] = {stencil->a_off[0], g.dim > 1 ? stencil->a_off[1] : nullptr,
                                     g.dim > 2 ? stencil->a_off[2] : nullptr};
            ck(explicit_faces_launch(g, stencil->a_diag, aoff, h->wx64, h->wy64, h->wz64,
                                     h->invd64, h->wx32, h->wy32, h->wz32, h->invd32, s),
               "explicit operator");
        } else {
            ck(vark_faces_launch(g, stencil->k, h->wx64, h->wy64, h->wz64, h->invd64, h->wx32,
                                 h->wy32, h->wz32, h->invd32, s),
               "face weights");
        }
    }
    if (g.dim == 3 && g.neu == 0 && rc == SRJ_OK) {  // the 3D pass stages planes by TMA
        h->p3maps = new (std::nothrow) Plane3dMaps();
        if (!h->p3maps) {
            srj_destroy(h);
            return SRJ_ENOMEM;
        }
        const PassLaunch a = make_launch(h, false);
        ck(plane3d_encode(h->kprec, h->vark, g, a.bufs, h->p3maps), "tensor maps");
        // two sweeps per pass: on request (temporal depth 2), and by default
        // for the FP32-pair inner sweeps of mixed precision (measured on the
        // 512^3 variable-k solve: 4.16 s against 4.38 s with one sweep per
        // pass; the same sweeps and bit-identical iterates); the per-sweep
        // change test of SRJ_TOL_DINF needs every sweep's own pass
        const int d3 = o.temporal_depth ? o.temporal_depth : (h->kprec == PREC_DF ? 2 : 1);
        h->use_p3d2 = d3 == 2 && o.tol_kind != SRJ_TOL_DINF;
        if (h->use_p3d2) {
            h->p3maps2 = new (std::nothrow) Plane3dMaps();
            if (!h->p3maps2) {
                srj_destroy(h);
                return SRJ_ENOMEM;
            }
            ck(plane3d_encode(h->kprec, h->vark, g, a.bufs, h->p3maps2, true), "tensor maps");
        }
    }
    ck(cudaEventCreate(&h->ev0), "event");
    ck(cudaEventCreate(&h->ev1), "event");
    ck(cudaEventCreate(&h->evl0), "event");
    ck(cudaEventCreate(&h->evl1), "event");
    ck(cudaStreamSynchronize(s), "create sync");
    if (rc != SRJ_OK) {
        srj_destroy(h);
        return rc;
    }
    *out = h;
    return SRJ_OK;
}

srj_status srj_solve(srj_handle *h, const void *f, void *u, double tol, srj_stats *stats) {
    if (!h) return SRJ_EINVAL;
    if (h->mg) return fail(h, SRJ_EINVAL, "srj_solve: multigrid handle (use srj_mg_solve)");
    if (h->opts.selector == SRJ_SEL_MLP && !h->mlp_loaded)
        return fail(h, SRJ_EINVAL, "srj_solve: learned selector without weights");
    if (!f || !u || !(tol > 0) || !std::isfinite(tol))
        return fail(h, SRJ_EINVAL, "srj_solve: null array or tol not a positive finite number");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    CK(cudaEventRecord(h->ev0, h->stream));
    srj_status s;
    if (h->user_prec == SRJ_PREC_MIXED)
        s = solve_mixed(h, (const double *)f, (double *)u, tol, stats);
    else
        s = solve_plain(h, f, u, tol, h->opts.selector, h->opts.level0, 0, stats);
    if (s == SRJ_ECUDA || s == SRJ_EINVAL) return s;
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (stats) stats->seconds = ms * 1e-3;
    return s;
}

srj_status srj_solve_host(srj_handle *h, const void *f_host, void *u_host, double tol,
                          srj_stats *stats) {
    if (!h) return SRJ_EINVAL;
    if (h->mg) return fail(h, SRJ_EINVAL, "srj_solve_host: multigrid handle");
    if (h->opts.selector == SRJ_SEL_MLP && !h->mlp_loaded)
        return fail(h, SRJ_EINVAL, "srj_solve_host: learned selector without weights");
    if (!f_host || !u_host) return fail(h, SRJ_EINVAL, "srj_solve_host: null array");
    const size_t bytes = (size_t)h->npts * h->esize;
    if (!h->dF) {
        if (dalloc(&h->dF, bytes) != cudaSuccess || dalloc(&h->dU, bytes) != cudaSuccess)
            return fail(h, SRJ_ENOMEM, "srj_solve_host: staging allocation");
    }
    if (stats) std::memset(stats, 0, sizeof(*stats));
    CK(cudaEventRecord(h->ev0, h->stream));
    CK(cudaMemcpyAsync(h->dF, f_host, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->dU, u_host, bytes, cudaMemcpyHostToDevice, h->stream));
    srj_status s;
    if (h->user_prec == SRJ_PREC_MIXED)
        s = solve_mixed(h, (const double *)h->dF, (double *)h->dU, tol, stats);
    else
        s = solve_plain(h, h->dF, h->dU, tol, h->opts.selector, h->opts.level0, 0, stats);
    if (s == SRJ_ECUDA || s == SRJ_EINVAL) return s;
    CK(cudaMemcpyAsync(u_host, h->dU, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (stats) stats->seconds = ms * 1e-3;
    return s;
}

srj_status srj_run_levels(srj_handle *h, const void *f, void *u, const int32_t *levels,
                          int64_t ncycles, double *rn_out) {
    if (!h) return SRJ_EINVAL;
    if (h->mg) return fail(h, SRJ_EINVAL, "srj_run_levels: multigrid handle");
    if (!f || !u || !levels || ncycles < 1)
        return fail(h, SRJ_EINVAL, "srj_run_levels: bad arguments");
    if (h->user_prec == SRJ_PREC_MIXED)
        return fail(h, SRJ_EUNSUPPORTED, "srj_run_levels: F64 or F32 precision only");
    if (ncycles > h->trace_cap)
        return fail(h, SRJ_EINVAL, "srj_run_levels: more cycles than trace_capacity");
    long long total = 0;
    for (int64_t c = 0; c < ncycles; ++c) {
        if (levels[c] < 0 || levels[c] > kMaxLevel)
            return fail(h, SRJ_EINVAL, "srj_run_levels: level outside [0, 24]");
        total += kLevelM[levels[c]];
    }
    // next_level() reads sched[cycles] after cycle `cycles` completes
    CK(cudaMemcpyAsync(h->sched, levels, (size_t)ncycles * sizeof(int32_t),
                       cudaMemcpyHostToDevice, h->stream));
    const long long saved = h->opts.max_sweeps;
    h->opts.max_sweeps = total + 1;
    srj_stats stats{};
    srj_status s = solve_plain(h, f, u, -1.0, DSEL_SCHEDULE, levels[0], (int)ncycles, &stats);
    h->opts.max_sweeps = saved;
    if (s == SRJ_ECUDA) return s;
    if (rn_out) {
        CK(cudaMemcpy(rn_out, h->trace_rn, (size_t)ncycles * sizeof(double),
                      cudaMemcpyDeviceToHost));
    }
    return stats.cycles == ncycles ? SRJ_OK : fail(h, s, "srj_run_levels: schedule cut short");
}

srj_status srj_residual_norm(srj_handle *h, const void *f, const void *u, double *out) {
    if (!h) return SRJ_EINVAL;
    if (h->mg) return fail(h, SRJ_EINVAL, "srj_residual_norm: multigrid handle");
    if (!f || !u || !out) return fail(h, SRJ_EINVAL, "srj_residual_norm: null argument");
    if (h->user_prec == SRJ_PREC_MIXED)
        return fail(h, SRJ_EUNSUPPORTED, "srj_residual_norm: F64 or F32 precision only");
    cudaStream_t st = h->stream;
    CK(copy_in_launch(h->kprec, h->geo, f, h->F, st));
    CK(copy_in_launch(h->kprec, h->geo, u, h->U[0], st));
    init_state(h, *h->h_st, 1.0, SRJ_TOL_REL, DSEL_HEURISTIC, 0, 0, 0, 0, 0);
    CK(cudaMemcpyAsync(h->st, h->h_st, sizeof(DevState), cudaMemcpyHostToDevice, st));
    PassLaunch a = make_launch(h, false);
    CK(generic_pass_launch(h->kprec, h->vark, a, st, h->p3maps));
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = h->h_st->r0;
    return SRJ_OK;
}

int64_t srj_get_trace(const srj_handle *h, int32_t *levels, double *rn, int64_t capacity) {
    if (!h || capacity < 0) return -1;
    const int64_t n = h->last_cycles < capacity ? h->last_cycles : capacity;
    const int64_t m = n < h->trace_cap ? n : h->trace_cap;
    if (m > 0) {
        if (levels &&
            cudaMemcpy(levels, h->trace_level, m * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
            return -1;
        if (rn && cudaMemcpy(rn, h->trace_rn, m * sizeof(double), cudaMemcpyDeviceToHost) !=
                      cudaSuccess)
            return -1;
    }
    return h->last_cycles;
}

srj_status srj_create_batched(int32_t nprob, const srj_grid *grids, const srj_stencil *stencils,
                              const srj_opts *opts, void *stream, srj_handle **out) {
    if (out) *out = nullptr;
    if (!out || !grids || nprob < 1) return SRJ_EINVAL;
    srj_opts o{};
    if (opts) o = *opts;
    if (o.precision != SRJ_PREC_MIXED) return SRJ_EUNSUPPORTED;
    if (o.selector == SRJ_SEL_JACOBI) return SRJ_EUNSUPPORTED;
    if (o.temporal_depth != 0 && o.temporal_depth != 2 && o.temporal_depth != 4)
        return SRJ_EINVAL;
    for (int p = 0; p < nprob; ++p) {
        if (grids[p].dim != 2 || (stencils && (stencils[p].k || stencils[p].a_diag)) ||
            grids[p].bc[0] || grids[p].bc[1])
            return SRJ_EUNSUPPORTED;
        if (grids[p].n[0] < 1 || grids[p].n[1] < 1 || grids[p].n[0] > (1 << 20) ||
            grids[p].n[1] > (1 << 20))
            return SRJ_EINVAL;
    }
    // The scheme tables, options and events come from an ordinary handle on a
    // 1x1 grid; the batch owns its own per-problem workspace.
    srj_grid g1{};
    g1.dim = 2;
    g1.n[0] = g1.n[1] = 1;
    srj_handle *h = nullptr;
    srj_status s = srj_create(&g1, nullptr, &o, stream, &h);
    if (s != SRJ_OK) return s;
    BatchData *B = new (std::nothrow) BatchData();
    if (!B) {
        srj_destroy(h);
        return SRJ_ENOMEM;
    }
    h->batch = B;
    B->nprob = nprob;
    B->probs.resize(nprob);
    B->npts.resize(nprob);
    size_t floats = 0;
    std::vector<size_t> offs(nprob);
    for (int p = 0; p < nprob; ++p) {
        BatchProb &P = B->probs[p];
        std::memset(&P, 0, sizeof(P));
        GridGeo &g = P.geo;
        g.dim = 2;
        g.nx = (int)grids[p].n[0];
        g.ny = (int)grids[p].n[1];
        g.nz = 1;
        const double hx = grids[p].h[0] > 0 ? grids[p].h[0] : 1.0 / (g.nx + 1.0);
        const double hy = grids[p].h[1] > 0 ? grids[p].h[1] : 1.0 / (g.ny + 1.0);
        const double ex = stencils && stencils[p].eps[0] > 0 ? stencils[p].eps[0] : 1.0;
        const double ey = stencils && stencils[p].eps[1] > 0 ? stencils[p].eps[1] : 1.0;
        geo_set_coefficients(g, ex / (hx * hx), ey / (hy * hy), 0.0);
        g.pitch = ((long long)g.nx + 31) / 32 * 32;
        g.plane = g.pitch * g.ny;
        B->npts[p] = (long long)g.nx * g.ny;
        offs[p] = floats;
        floats += 5 * (size_t)g.plane;
    }
    B->arena_floats = floats;
    if (dalloc(&B->arena, floats * sizeof(float)) != cudaSuccess ||
        dalloc(&B->dprobs, (size_t)nprob * sizeof(BatchProb)) != cudaSuccess ||
        dalloc(&B->dstates, (size_t)nprob * sizeof(BatchState)) != cudaSuccess ||
        dalloc(&B->ndone, sizeof(unsigned int)) != cudaSuccess ||
        dalloc(&B->ctl, 2 * sizeof(int32_t)) != cudaSuccess ||
        dalloc(&B->active, kBatchLayouts * sizeof(long long)) != cudaSuccess ||
        halloc(&B->hstates, (size_t)nprob * sizeof(BatchState)) != cudaSuccess) {
        srj_destroy(h);
        return SRJ_ENOMEM;
    }
    for (int p = 0; p < nprob; ++p) {
        BatchProb &P = B->probs[p];
        float *base = B->arena + offs[p];
        const size_t pl = (size_t)P.geo.plane;
        P.inner.f = base;
        P.inner.u[0] = base + pl;
        P.inner.u[1] = base + 2 * pl;
        P.inner.ulo[0] = base + 3 * pl;
        P.inner.ulo[1] = base + 4 * pl;
    }
    s = batch_layout(h, o.temporal_depth ? o.temporal_depth : 4, 64);
    if (s == SRJ_OK && cudaMemsetAsync(B->arena, 0, floats * sizeof(float), h->stream) != cudaSuccess)
        s = SRJ_ECUDA;
    if (s != SRJ_OK) {
        srj_destroy(h);
        return s;
    }
    *out = h;
    return SRJ_OK;
}

srj_status srj_solve_batched(srj_handle *h, const double *const *f, double *const *u, double tol,
                             srj_stats *stats) {
    if (!h) return SRJ_EINVAL;
    BatchData *B = h->batch;
    if (!B) return fail(h, SRJ_EINVAL, "srj_solve_batched: not a batched handle");
    if (h->opts.selector == SRJ_SEL_MLP && !h->mlp_loaded)
        return fail(h, SRJ_EINVAL, "srj_solve_batched: learned selector without weights");
    if (!f || !u || !(tol > 0) || !std::isfinite(tol))
        return fail(h, SRJ_EINVAL, "srj_solve_batched: null arrays or bad tol");
    for (int p = 0; p < B->nprob; ++p) {
        if (!f[p] || !u[p]) return fail(h, SRJ_EINVAL, "srj_solve_batched: null array");
        B->probs[p].f = f[p];
        B->probs[p].u = u[p];
    }
    CK(cudaMemcpyAsync(B->dprobs, B->probs.data(), B->probs.size() * sizeof(BatchProb),
                       cudaMemcpyHostToDevice, h->stream));
    srj_status s = SRJ_OK;
    if (!B->tuned) {
        s = batch_autotune(h);
        if (s != SRJ_OK) return s;
    }
    s = batch_build_graph(h, tol);
    if (s != SRJ_OK) return s;
    CK(cudaEventRecord(h->ev0, h->stream));
    s = batch_reset(h);
    if (s != SRJ_OK) return s;
    CK(cudaGraphLaunch(B->exec, h->stream));
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaMemcpyAsync(B->hstates, B->dstates, (size_t)B->nprob * sizeof(BatchState),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    srj_status worst = SRJ_OK;
    for (int p = 0; p < B->nprob; ++p) {
        const BatchState &S = B->hstates[p];
        const srj_status ps = status_of(S.result);
        if (ps != SRJ_OK && worst == SRJ_OK) worst = ps;
        if (stats) {
            srj_stats &o = stats[p];
            std::memset(&o, 0, sizeof(o));
            o.status = ps;
            o.final_level = S.final_level;
            o.sweeps = S.sweeps;
            o.cycles = S.cycles;
            o.outer = S.outer;
            o.passes = S.passes;
            o.r0 = S.r0;
            o.rn = S.rn;
            o.seconds = ms * 1e-3;
        }
    }
    return worst;
}

srj_status srj_set_wait_limit(srj_handle *h, int64_t polls) {
    if (!h) return SRJ_EINVAL;
    h->wait_limit = polls < 0 ? kDefaultWaitLimit : (long long)polls;
    return SRJ_OK;
}

srj_status srj_mlp_set_weights(srj_handle *h, const uint16_t *w, int64_t count) {
    if (!h) return SRJ_EINVAL;
    if (h->mg) return fail(h, SRJ_EINVAL, "srj_mlp_set_weights: multigrid handle");
    if (!w || count != 6617) return fail(h, SRJ_EINVAL, "srj_mlp_set_weights: need 6617 values");
    CK(cudaMemcpyAsync(h->mlp_w, w, 6617 * sizeof(uint16_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->mlp_loaded = true;
    return SRJ_OK;
}

const char *srj_last_error(const srj_handle *h) {
    if (!h) return "srj: invalid handle";
    return h->err.empty() ? "" : h->err.c_str();
}

srj_status srj_mg_create(const srj_grid *grid, const srj_stencil *stencil,
                         const srj_mg_opts *opts, void *stream, srj_handle **out) {
    if (out) *out = nullptr;
    if (!grid || !out || grid->dim < 1 || grid->dim > 3) return SRJ_EINVAL;
    if (stencil && (stencil->k || stencil->a_diag)) return SRJ_EUNSUPPORTED;
    // every axis n = 2^k - 1 with one k: the hierarchy halves all axes down to
    // a single point
    int k = -1;
    for (int a = 0; a < grid->dim; ++a) {
        const long long n = grid->n[a];
        if (grid->bc[a] != SRJ_BC_DIRICHLET || n < 1 || n > (1LL << 30) || ((n + 1) & n) != 0 ||
            grid->h[a] < 0 || !std::isfinite(grid->h[a]))
            return SRJ_EINVAL;
        int ka = 0;
        while ((1LL << ka) < n + 1) ++ka;
        if (k >= 0 && ka != k) return SRJ_EINVAL;
        k = ka;
    }
    srj_mg_opts o{1, 0, 0, 0};
    if (opts) o = *opts;
    if (o.smoother_level < 0 || o.smoother_level > kMaxLevel || o.nu1 < 0 || o.nu2 < 0 ||
        o.max_cycles < 0)
        return SRJ_EINVAL;
    srj_handle *h = new (std::nothrow) srj_handle();
    if (!h) return SRJ_ENOMEM;
    MgData *m = new (std::nothrow) MgData();
    if (!m) {
        delete h;
        return SRJ_ENOMEM;
    }
    h->mg = m;
    h->stream = (cudaStream_t)stream;
    m->nu1 = o.nu1 > 0 ? o.nu1 : 1;
    m->nu2 = o.nu2 > 0 ? o.nu2 : 1;
    m->max_cycles = o.max_cycles > 0 ? o.max_cycles : 100;
    m->omegas.resize(kLevelM[o.smoother_level]);
    scheme_omegas(o.smoother_level, m->omegas.data(), (int)m->omegas.size());
    MgGeo g{};
    g.dim = grid->dim;
    int n3[3] = {(int)grid->n[0], grid->dim > 1 ? (int)grid->n[1] : 1,
                 grid->dim > 2 ? (int)grid->n[2] : 1};
    double c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < grid->dim; ++a) {
        const double hh = grid->h[a] > 0 ? grid->h[a] : 1.0 / (double)(n3[a] + 1);
        const double e = stencil ? stencil->eps[a] : 0.0;
        if (e < 0 || !std::isfinite(e)) {
            srj_destroy(h);
            return SRJ_EINVAL;
        }
        c[a] = (e > 0 ? e : 1.0) / (hh * hh);
    }
    m->nlev = k;
    for (int l = 0; l < k; ++l) {
        g.nx = n3[0];
        g.ny = n3[1];
        g.nz = n3[2];
        g.cx = c[0];
        g.cy = c[1];
        g.cz = c[2];
        g.diag = 2.0 * (c[0] + c[1] + c[2]);
        m->geo.push_back(g);
        for (int a = 0; a < grid->dim; ++a) {
            n3[a] = (n3[a] - 1) / 2;
            c[a] *= 0.25;  // twice the spacing
        }
    }
    for (int l = 0; l < k; ++l) {
        const size_t bytes =
            sizeof(double) * (size_t)m->geo[l].nx * m->geo[l].ny * m->geo[l].nz;
        double *p[4] = {nullptr, nullptr, nullptr, nullptr};
        for (double *&q : p)
            if (dalloc(&q, bytes) != cudaSuccess) {
                for (double *r : p) dfree(r);
                srj_destroy(h);
                return SRJ_ENOMEM;
            }
        m->U0.push_back(p[0]);
        m->U1.push_back(p[1]);
        m->F.push_back(p[2]);
        m->R.push_back(p[3]);
    }
    if (dalloc(&m->partials, sizeof(double) * mg_partials_needed()) != cudaSuccess ||
        dalloc(&m->norm2, sizeof(double)) != cudaSuccess ||
        halloc(&m->h_norm2, sizeof(double)) != cudaSuccess) {
        srj_destroy(h);
        return SRJ_ENOMEM;
    }
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess) {
        srj_destroy(h);
        return SRJ_ECUDA;
    }
    *out = h;
    return SRJ_OK;
}

}  // extern "C"

namespace {

// Record one V-cycle from level l down (stream capture); the iterate of level
// l is in U0 (cur 0) or U1 (cur 1).  Returns the buffer holding it afterwards.
int mg_record(MgData &m, int l, int cur, cudaStream_t s, cudaError_t &err) {
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    };
    const MgGeo &g = m.geo[l];
    double *U[2] = {m.U0[l], m.U1[l]};
    if (l == m.nlev - 1) {  // one point: u = f / D from u = 0
        ck(mg_sweep_launch(g, U[cur], U[cur ^ 1], m.F[l], 1.0, s));
        m.launches += 1;
        return cur ^ 1;
    }
    auto smooth = [&](int cycles) {
        for (int c = 0; c < cycles; ++c)
            for (double w : m.omegas) {
                ck(mg_sweep_launch(g, U[cur], U[cur ^ 1], m.F[l], w, s));
                cur ^= 1;
                m.launches += 1;
                if (l == 0) m.fine_sweeps += 1;
            }
    };
    smooth(m.nu1);
    ck(mg_residual_launch(g, U[cur], m.F[l], m.R[l], nullptr, nullptr, s));
    ck(mg_restrict_launch(g, m.R[l], m.geo[l + 1], m.F[l + 1], s));
    const MgGeo &gc = m.geo[l + 1];
    ck(cudaMemsetAsync(m.U0[l + 1], 0, sizeof(double) * (size_t)gc.nx * gc.ny * gc.nz, s));
    const int cc = mg_record(m, l + 1, 0, s, err);
    ck(mg_prolong_launch(gc, cc ? m.U1[l + 1] : m.U0[l + 1], g, U[cur], s));
    m.launches += 3;
    smooth(m.nu2);
    return cur;
}

// ||f - A u||^2 of the fine level (in U0) into the pinned host word.
void mg_norm(MgData &m, cudaStream_t s, cudaError_t &err) {
    int np = 0;
    cudaError_t e = mg_residual_launch(m.geo[0], m.U0[0], m.F[0], nullptr, m.partials, &np, s);
    if (e == cudaSuccess) e = mg_sum_launch(m.partials, np, m.norm2, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m.h_norm2, m.norm2, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
}

}  // namespace

extern "C" {

srj_status srj_mg_solve(srj_handle *h, const double *f, double *u, double tol, srj_stats *stats) {
    if (!h) return SRJ_EINVAL;
    MgData *m = h->mg;
    if (!m) return fail(h, SRJ_EINVAL, "srj_mg_solve: not a multigrid handle");
    if (!f || !u || !(tol > 0) || !std::isfinite(tol))
        return fail(h, SRJ_EINVAL, "srj_mg_solve: null array or tol not a positive finite number");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaStream_t s = h->stream;
    const MgGeo &g0 = m->geo[0];
    const size_t bytes = sizeof(double) * (size_t)g0.nx * g0.ny * g0.nz;
    if (!m->exec) {  // capture one V-cycle (ending in U0 of the fine level) + its norm
        // on the handle's private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream
        cudaError_t err = cudaSuccess;
        cudaStream_t cs = m->cap;
        m->launches = 0;
        m->fine_sweeps = 0;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const int fin = mg_record(*m, 0, 0, cs, err);
        if (fin != 0) {
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(m->U0[0], m->U1[0], bytes, cudaMemcpyDeviceToDevice, cs);
            m->launches += 1;
        }
        mg_norm(*m, cs, err);
        m->launches += 2;
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (err != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(h, SRJ_ECUDA, std::string("srj_mg_solve: capture: ") +
                                          cudaGetErrorString(err != cudaSuccess ? err : e2));
        }
        m->graph = graph;
        CK(cudaGraphInstantiate(&m->exec, m->graph, 0));
    }
    CK(cudaEventRecord(h->ev0, s));
    CK(cudaMemcpyAsync(m->F[0], f, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(m->U0[0], u, bytes, cudaMemcpyDeviceToDevice, s));
    cudaError_t err = cudaSuccess;
    mg_norm(*m, s, err);
    CK(err);
    CK(cudaStreamSynchronize(s));
    const double r0 = std::sqrt(*m->h_norm2);
    double rn = r0;
    long long cycles = 0;
    srj_status result = SRJ_ENOTCONV;
    if (!std::isfinite(r0)) result = SRJ_EDIVERGED;
    else if (r0 == 0.0) result = SRJ_OK;
    while (result == SRJ_ENOTCONV && cycles < m->max_cycles) {
        CK(cudaGraphLaunch(m->exec, s));
        CK(cudaStreamSynchronize(s));
        cycles += 1;
        rn = std::sqrt(*m->h_norm2);
        if (!std::isfinite(rn)) result = SRJ_EDIVERGED;
        else if (rn / r0 < tol) result = SRJ_OK;
    }
    CK(cudaMemcpyAsync(u, m->U0[0], bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(h->ev1, s));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (stats) {
        stats->status = result;
        stats->final_level = 0;
        stats->sweeps = cycles * m->fine_sweeps;
        stats->cycles = cycles;
        stats->outer = 0;
        stats->passes = cycles * m->launches;
        stats->r0 = r0;
        stats->rn = rn;
        stats->seconds = ms * 1e-3;
    }
    return result;
}

srj_status srj_destroy(srj_handle *h) {
    if (!h) return SRJ_EINVAL;
    if (MgData *m = h->mg) {
        if (m->exec) cudaGraphExecDestroy(m->exec);
        if (m->graph) cudaGraphDestroy(m->graph);
        for (auto *v : {&m->U0, &m->U1, &m->F, &m->R})
            for (double *p : *v) dfree(p);
        dfree(m->partials);
        dfree(m->norm2);
        if (m->h_norm2) cudaFreeHost(m->h_norm2);
        if (m->cap) cudaStreamDestroy(m->cap);
        delete m;
    }
    if (BatchData *B = h->batch) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        for (void *p : {(void *)B->dprobs, (void *)B->dstates, (void *)B->partials,
                        (void *)B->ndone, (void *)B->arena, (void *)B->ctl, (void *)B->active})
            dfree(p);
        for (int l = 0; l < kBatchLayouts; ++l) dfree(B->item_prob[l]);
        if (B->hstates) cudaFreeHost(B->hstates);
        delete B;
    }
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->evl0) cudaEventDestroy(h->evl0);
    if (h->evl1) cudaEventDestroy(h->evl1);
    for (void *p : {(void *)h->w64, (void *)h->w32, h->F, h->U[0], h->U[1], h->Ulo[0], h->Ulo[1],
                    (void *)h->wx64, (void *)h->wy64, (void *)h->wz64, (void *)h->invd64,
                    (void *)h->wx32, (void *)h->wy32, (void *)h->wz32, (void *)h->invd32,
                    (void *)h->st, (void *)h->partials, (void *)h->trace_level,
                    (void *)h->trace_rn, (void *)h->sched, (void *)h->opartials,
                    (void *)h->oticket, (void *)h->onorm2, h->dF, h->dU, (void *)h->mlp_w})
        dfree(p);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->h_onorm2) cudaFreeHost(h->h_onorm2);
    delete h->p3maps;
    delete h->p3maps2;
    delete h;
    return SRJ_OK;
}

}  // extern "C"
